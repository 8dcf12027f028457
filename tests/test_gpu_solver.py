"""GPU parity of the block Fourier transform, the shift-invert PCG and the
Krylov-Schur eigensolver, through the C ABI, against the oracle.

Eigenvalue tolerance 1e-10 relative (the method's FP64 target), for both the
plain FP64 path and the mixed-precision path with FP64 residual refinement.
"""

import numpy as np
import pytest

from oracle import oracle as O
from workloads import complex_gaussian, isotropic_voigt, two_phase_sphere
from workloads.materials import TwoPhaseCell

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_03599_gb300 as pc
    return pc


class Grid:
    def __init__(self, pc, cell):
        self.pc = pc
        self.cell = cell
        self.h = pc.pc_grid_create(cell.N, cell.C, cell.rho, phase=cell.phase, theta=cell.theta,
                                   a_lat=cell.a_lat)
        self.C0, self.rho0, self.L = pc.pc_grid_units(self.h)
        self.pb = O.problem_from_cell(cell, C0=self.C0, rho0=self.rho0, L=self.L)
        self.to_si = self.C0 / (self.rho0 * self.L ** 2)

    def close(self):
        self.pc.pc_grid_destroy(self.h)


# N = 6, 10, 12 run the transform kernels with runtime factors (n = 3, 5, 6), N = 4, 8, 16 the
# compile-time factorisations (n = 2 x 2 ... 4 x 4 with n = 2 on the runtime path)
@pytest.mark.parametrize("N", [4, 6, 8, 10, 12, 16])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_block_fourier_matches_dense_basis(pc, N, dtype):
    import torch
    g = Grid(pc, two_phase_sphere(N, 0.35, 1))
    td = torch.complex128 if dtype == "c128" else torch.complex64
    tol = 1e-12 if dtype == "c128" else 2e-6
    try:
        kappa = [0.3, -0.1, 0.45]
        pc.pc_set_k(g.h, kappa)
        for b in range(4):
            # the library labels modes with kappa reduced into [0, 1) (same operator, fixed labels)
            kr = np.asarray(kappa) - np.floor(kappa)
            T = O.T_sigma_dense((N, N, N), kr, b)  # columns: modes p fastest, then q, then r
            w = complex_gaussian((3, N ** 3 // 4), 20 + b)
            ref = np.stack([T.conj().T @ w[a] for a in range(3)])
            wd = torch.from_numpy(w.reshape(-1)).to(td).cuda()
            out = torch.empty_like(wd)
            pc.pc_block_fourier(g.h, b, 0, wd, out)
            back = torch.empty_like(wd)
            pc.pc_block_fourier(g.h, b, 1, out, back)
            torch.cuda.synchronize()
            got = out.cpu().numpy().astype(np.complex128).reshape(3, -1)
            assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
            assert np.abs(back.cpu().numpy().reshape(3, -1) - w).max() <= tol * np.abs(w).max()
    finally:
        g.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("kappa", [[0.3, 0.1, 0.2], [0.0, 0.0, 0.0]])
@pytest.mark.parametrize("N", [16, 24, 48])
def test_shift_invert_pcg_residual(pc, dtype, kappa, N):
    import torch
    g = Grid(pc, two_phase_sphere(N, 0.35, 2))
    td = torch.complex128 if dtype == "c128" else torch.complex64
    tol = 1e-10 if dtype == "c128" else 1e-5
    try:
        pc.pc_set_k(g.h, kappa)
        sigma = pc.pc_default_sigma(g.h)
        assert sigma < 0
        for b in (0, 3, -1):
            m = N ** 3 // 4 if b >= 0 else N ** 3
            rhs = complex_gaussian((3, m), 30 + b)
            bd = torch.from_numpy(rhs.reshape(-1)).to(td).cuda()
            xd = torch.empty_like(bd)
            info = pc.pc_shift_invert_pcg(g.h, b, sigma, bd, xd, tol=tol, maxit=500)
            assert info["status"] == 0 and info["rel_resid"] <= tol
            x = xd.cpu().numpy().astype(np.complex128).reshape(3, -1)
            Ax = (O.apply_block(g.pb, kappa, b, x, sigma) if b >= 0 else O.apply_full(g.pb, kappa, x, sigma))
            true_rel = np.linalg.norm(rhs - Ax) / np.linalg.norm(rhs)
            assert true_rel <= (10 * tol if dtype == "c128" else 1e-4)
            assert info["iters"] < 200
    finally:
        g.close()


def test_pcg_status_codes(pc):
    import torch
    N = 8
    g = Grid(pc, two_phase_sphere(N, 0.35, 1))
    try:
        kappa = [0.3, 0.1, 0.2]
        pc.pc_set_k(g.h, kappa)
        rhs = torch.from_numpy(complex_gaussian(3 * N ** 3 // 4, 1)).cuda()
        x = torch.empty_like(rhs)
        r = pc.pc_shift_invert_pcg(g.h, 0, pc.pc_default_sigma(g.h), rhs, x, tol=1e-12, maxit=1,
                                   raise_on_fail=False)
        assert r["rc"] == pc.PC_ENOCONV and r["iters"] == 1
        # a shift above the lowest eigenvalue makes the operator indefinite
        lam = O.dense_eigvals(g.pb, kappa, 0)
        r = pc.pc_shift_invert_pcg(g.h, 0, 0.5 * (lam[5] + lam[6]), rhs, x, tol=1e-12, maxit=300,
                                   raise_on_fail=False)
        assert r["rc"] in (pc.PC_EBREAKDOWN, pc.PC_ENOCONV)
        zero = torch.zeros_like(rhs)
        r = pc.pc_shift_invert_pcg(g.h, 0, -1.0, zero, x, tol=1e-10, maxit=10)
        assert r["iters"] == 0 and torch.count_nonzero(x).item() == 0
    finally:
        g.close()


@pytest.mark.parametrize("kappa", [[0.3, 0.1, 0.2], [0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
@pytest.mark.parametrize("mode", ["blocked", "blocked-pre64", "full", "mixed"])
def test_eigs_tiny_vs_dense(pc, kappa, mode):
    """Tiny two-phase cell (N = 8, R = 0.35, seed 1): lowest 12 non-zero eigenvalues.
    blocked-pre64: the FP64 inner PCG with its preconditioner in FP64 too (default: complex64)."""
    g = Grid(pc, two_phase_sphere(8, 0.35, 1))
    try:
        opt = pc.pc_options_default(full_space=int(mode == "full"),
                                    precision=pc.PC_PREC_MIXED if mode == "mixed" else pc.PC_PREC_FP64,
                                    precond_fp32=int(mode != "blocked-pre64"))
        ev, blocks, info = pc.pc_eigs(g.h, kappa, 12, opt=opt)
        dense = O.lowest_nonzero(O.dense_eigvals(g.pb, kappa), 12) * g.to_si
        rel = np.abs(ev - dense) / dense
        assert rel.max() <= 1e-10, rel
        assert info["max_rel_resid"] <= 1e-8
        at_gamma = np.allclose(kappa, 0)
        assert info["zero_modes"] == (12 if at_gamma else 0)
        if mode != "full":
            for b in range(4):  # each reported value is an eigenvalue of its block
                mine = ev[blocks == b]
                if mine.size:
                    db = O.lowest_nonzero(O.dense_eigvals(g.pb, kappa, b), 12) * g.to_si
                    assert np.min(np.abs(mine[:, None] - db[None, :]) / db[None, :], axis=1).max() <= 1e-10
    finally:
        g.close()


def test_eigs_homogeneous_closed_form(pc):
    """A homogeneous cell: eigenvalues = union over modes of eig(B_hat C B_hat^H)/rho, exact fourfold."""
    N = 24
    rng = np.random.default_rng(4)
    G = rng.standard_normal((6, 6))
    C = (G @ G.T + 6 * np.eye(6)) * 1e10
    cell = TwoPhaseCell(N=N, C=np.stack([C, C]), rho=np.array([2000.0, 2000.0]), phase=None, theta=None,
                        a_lat=np.eye(3))
    g = Grid(pc, cell)
    try:
        kappa = [0.21, 0.13, 0.05]
        ev, blocks, info = pc.pc_eigs(g.h, kappa, 20)
        cf = O.homogeneous_spectrum((N,) * 3, kappa, np.eye(3), C / g.C0, 2.0)[:20] * g.to_si
        assert np.abs(ev - cf).max() / cf.max() <= 1e-10
    finally:
        g.close()


def test_eigenvectors_satisfy_pencil(pc):
    import torch
    N = 8
    g = Grid(pc, two_phase_sphere(N, 0.35, 1))
    try:
        kappa = [0.3, 0.1, 0.2]
        nev = 6
        evecs = torch.empty(nev * 3 * N ** 3, dtype=torch.complex128, device="cuda")
        ev, blocks, info = pc.pc_eigs(g.h, kappa, nev, evecs=evecs)
        V = evecs.cpu().numpy().reshape(nev, 3, -1)
        rho = g.pb.node_rho()
        for i in range(nev):
            lam = ev[i] / g.to_si
            Av = O.apply_full(g.pb, kappa, V[i])
            r = Av - lam * rho[None, :] * V[i]
            assert np.linalg.norm(r) <= 1e-8 * abs(lam) * np.linalg.norm(rho[None, :] * V[i])
            assert abs(np.real(np.vdot(V[i], rho[None, :] * V[i])) - 1.0) < 1e-10
    finally:
        g.close()


def test_eigs_argument_errors(pc):
    g = Grid(pc, two_phase_sphere(8, 0.35, 1))
    try:
        with pytest.raises(pc.PcError):
            pc.pc_eigs(g.h, [0, 0, 0], 0)
        with pytest.raises(pc.PcError):
            pc.pc_eigs(g.h, [0, 0, 0], 10 ** 6)
    finally:
        g.close()


@pytest.mark.parametrize("kappa", [[0.5, 0.0, 0.0], [0.0, 0.0, 0.0]])
def test_eigs_n48_preconditioner_precision_neutral(pc, kappa):
    """N = 48 two-phase cell: the FP64 solve with the complex64 preconditioner (flexible CG) and
    with the FP64 preconditioner give the same 20 eigenvalues to 1e-10 relative."""
    g = Grid(pc, two_phase_sphere(48, 0.35, 2))
    try:
        out = {}
        for p32 in (1, 0):
            opt = pc.pc_options_default(precond_fp32=p32)
            ev, _, info = pc.pc_eigs(g.h, kappa, 20, opt=opt)
            assert info["max_rel_resid"] <= 1e-8
            out[p32] = (ev, info["pcg_iters"])
        assert np.abs(out[1][0] - out[0][0]).max() / out[0][0].max() <= 1e-10
        # complex64 rounding of the preconditioner costs at most a few iterations
        assert out[1][1] <= 1.3 * out[0][1]
    finally:
        g.close()
