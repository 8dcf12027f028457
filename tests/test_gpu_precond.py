"""GPU parity of the reference-medium preconditioner (Sec. 5.4) through the C ABI
(`pc_block_precond`) against the oracle, which builds each mode's factor from the weighted
SVD of Eq. weighted_svd_unified with Psi = C_ref^-1 and the transforms from separable Bloch
sums (no FFT).

Tolerances (element-wise, relative to the largest reference entry): complex128 with FP64
transforms 1e-12 (two FFTs and a 3x3 solve in FP64); complex64, and complex128 with complex64
transforms, 5e-5 (two single-precision FFTs of length <= 48 and a 3x3 adjugate solve, each
a few units of 6e-8 times log2 of the length, with margin).
"""

import numpy as np
import pytest

from oracle import oracle as O
from workloads import complex_gaussian, two_phase_sphere
from workloads.materials import TwoPhaseCell

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c128-fp32": 5e-5, "c64": 5e-5}


@pytest.fixture(scope="module")
def pc():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_03599_gb300 as pc
    return pc


class Grid:
    def __init__(self, pc, cell):
        self.pc = pc
        self.h = pc.pc_grid_create(cell.N, cell.C, cell.rho, phase=cell.phase, theta=cell.theta,
                                   a_lat=cell.a_lat)
        C0, rho0, L = pc.pc_grid_units(self.h)
        self.pb = O.problem_from_cell(cell, C0=C0, rho0=rho0, L=L)

    def close(self):
        self.pc.pc_grid_destroy(self.h)


def _gpu_precond(pc, g, block, sigma, r, mode):
    import torch
    td = torch.complex64 if mode == "c64" else torch.complex128
    rd = torch.from_numpy(np.ascontiguousarray(r).reshape(-1)).to(td).cuda()
    zd = torch.empty_like(rd)
    pc.pc_block_precond(g.h, block, sigma, rd, zd, fp32_transforms=(mode == "c128-fp32"))
    torch.cuda.synchronize()
    return zd.cpu().numpy().astype(np.complex128).reshape(3, -1)


def _check(got, ref, tol):
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= tol, err


@pytest.mark.parametrize("mode", ["c128", "c128-fp32", "c64"])
@pytest.mark.parametrize("kappa", [[0.3, -0.1, 0.45], [0.0, 0.0, 0.0]])
@pytest.mark.parametrize("N", [8, 10, 24])
def test_precond_parity_blocks(pc, N, kappa, mode):
    g = Grid(pc, two_phase_sphere(N, 0.35, 1))
    try:
        pc.pc_set_k(g.h, kappa)
        sigma = pc.pc_default_sigma(g.h)
        for b in range(4):
            r = complex_gaussian((3, N ** 3 // 4), 100 + b)
            ref = O.precond_block(g.pb, kappa, b, sigma, r)
            _check(_gpu_precond(pc, g, b, sigma, r, mode), ref, TOL[mode])
    finally:
        g.close()


@pytest.mark.parametrize("mode", ["c128", "c64"])
def test_precond_parity_full_space(pc, mode):
    N = 10
    g = Grid(pc, two_phase_sphere(N, 0.3, 4))
    try:
        kappa = [0.2, 0.45, -0.3]
        pc.pc_set_k(g.h, kappa)
        sigma = pc.pc_default_sigma(g.h)
        r = complex_gaussian((3, N ** 3), 110)
        ref = O.precond_full(g.pb, kappa, sigma, r)
        _check(_gpu_precond(pc, g, -1, sigma, r, mode), ref, TOL[mode])
    finally:
        g.close()


def test_precond_parity_fractional_material_fcc_lattice(pc):
    N = 12
    cell = two_phase_sphere(N, 0.3, 2)
    cell.theta = np.random.default_rng(3).uniform(0, 1, N ** 3).astype(np.float32)
    cell.phase = None
    cell.a_lat = np.array([[0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]]) * 0.03
    g = Grid(pc, cell)
    try:
        kappa = [0.25, 0.5, 0.75]
        pc.pc_set_k(g.h, kappa)
        sigma = pc.pc_default_sigma(g.h)
        for b in (1, 2):
            r = complex_gaussian((3, N ** 3 // 4), 120 + b)
            ref = O.precond_block(g.pb, kappa, b, sigma, r)
            for mode in ("c128", "c64"):
                _check(_gpu_precond(pc, g, b, sigma, r, mode), ref, TOL[mode])
    finally:
        g.close()


@pytest.mark.parametrize("mode", ["c128", "c128-fp32"])
def test_precond_parity_n48_solver_workload(pc, mode):
    """The FP64 band workload's grid (N=48, R=0.35, seed 2), every block, as the solve applies it."""
    N = 48
    g = Grid(pc, two_phase_sphere(N, 0.35, 2))
    try:
        kappa = [0.3, 0.1, 0.2]
        pc.pc_set_k(g.h, kappa)
        sigma = pc.pc_default_sigma(g.h)
        for b in range(4):
            r = complex_gaussian((3, N ** 3 // 4), 130 + b)
            ref = O.precond_block(g.pb, kappa, b, sigma, r)
            _check(_gpu_precond(pc, g, b, sigma, r, mode), ref, TOL[mode])
    finally:
        g.close()


@pytest.mark.parametrize("mode", ["c64", "c128"])
def test_precond_single_modes_n160_precision_workload(pc, mode):
    """Full size, the N=160 precision workload's grid (R=0.3, seed 3): a block Fourier mode
    T_sigma[:, m] u maps to T_sigma[:, m] F(m) u with F(m) from the oracle's weighted SVD,
    at every node.  Tolerance 64 eps (lambda_max(m) + |sigma| rho_ref) / (|sigma| rho_ref):
    rounding of the input and of the transforms is amplified at most by the mode's stiffness
    relative to the shift."""
    N = 160
    g = Grid(pc, two_phase_sphere(N, 0.3, 3))
    eps = 2.0 ** -24 if mode == "c64" else 2.0 ** -53
    modes = [(0, 0, 0), (1, 0, 0), (0, 2, 1)] + ([(5, 7, 33), (37, 71, 150)] if mode == "c128" else [])
    u = np.array([0.4 - 0.2j, 1.1, -0.3j])
    try:
        kappa = [0.3, 0.1, 0.2]
        pc.pc_set_k(g.h, kappa)
        sigma = pc.pc_default_sigma(g.h)
        C_ref, rho_ref = O.reference_medium(g.pb)
        for b in (0, 3):
            for m in modes:
                col = O.block_mode_vector(g.pb.dims, kappa, b, *m)
                F = O.precond_mode_factor(g.pb, kappa, sigma, *m, C_ref, rho_ref)
                ref = np.outer(F @ u, col)
                ratio = 1.0 / (np.linalg.eigvalsh(F).min() * abs(sigma) * rho_ref)
                _check(_gpu_precond(pc, g, b, sigma, np.outer(u, col), mode), ref, 64 * eps * ratio)
    finally:
        g.close()


def test_precond_inverts_homogeneous_operator(pc):
    """On a homogeneous medium (A - sigma M) P r = r with the GPU apply (FP64, N=32: the
    shifted operator's condition number is ~4e4 there, so 1e-9 leaves a wide margin)."""
    import torch
    N = 32
    C = np.diag([180.0, 150.0, 120.0, 40.0, 50.0, 60.0]) * 1e9
    C[0, 1] = C[1, 0] = 50e9
    C[1, 2] = C[2, 1] = 30e9
    cell = TwoPhaseCell(N=N, C=np.stack([C, C]), rho=np.array([3000.0, 3000.0]), phase=None, theta=None,
                        a_lat=np.eye(3))
    g = Grid(pc, cell)
    try:
        pc.pc_set_k(g.h, [0.3, 0.1, 0.2])
        sigma = pc.pc_default_sigma(g.h)
        for b in (-1, 0, 3):
            m = N ** 3 // 4 if b >= 0 else N ** 3
            r = torch.from_numpy(complex_gaussian(3 * m, 140 + b)).cuda()
            z = torch.empty_like(r)
            back = torch.empty_like(r)
            pc.pc_block_precond(g.h, b, sigma, r, z)
            pc.pc_block_apply(g.h, b, z, back, shift=sigma)
            torch.cuda.synchronize()
            err = ((back - r).abs().max() / r.abs().max()).item()
            assert err <= 1e-9, err
    finally:
        g.close()


def test_precond_argument_errors(pc):
    import torch
    N = 8
    g = Grid(pc, two_phase_sphere(N, 0.35, 1))
    try:
        r = torch.zeros(3 * N ** 3 // 4, dtype=torch.complex128, device="cuda")
        z = torch.empty_like(r)
        with pytest.raises(pc.PcError) as e:
            pc.pc_block_precond(g.h, 0, -1.0, r, z)
        assert e.value.code == pc.PC_ESTATE
        pc.pc_set_k(g.h, [0.1, 0.2, 0.3])
        for block, sigma in ((4, -1.0), (-2, -1.0), (0, float("nan")), (0, float("inf"))):
            with pytest.raises(pc.PcError) as e:
                pc.pc_block_precond(g.h, block, sigma, r, z)
            assert e.value.code == pc.PC_EINVAL
        assert pc.lib.pc_block_precond(g.h, 0, pc.PC_C128, 0, -1.0, None, None, None) == pc.PC_EINVAL
        # a zero vector maps to zero, in place as well
        pc.pc_block_precond(g.h, 0, -1.0, r, r)
        torch.cuda.synchronize()
        assert torch.count_nonzero(r).item() == 0
    finally:
        g.close()
