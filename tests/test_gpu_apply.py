"""GPU parity of the fused block apply against the oracle, through the C ABI.

Tolerances: complex128 (FP64 arithmetic) 1e-12 relative, as the method's FP64
target requires; complex64 (FP32 arithmetic) 2e-6 relative, i.e. about 30 FP32
unit roundoffs (u = 6e-8) for a chain of ~10 dependent rounding stages on
values of the output's magnitude.  Both are checked element by element
against the largest output magnitude and in the 2-norm.
"""

import numpy as np
import pytest

from oracle import oracle as O
from workloads import complex_gaussian, two_phase_sphere

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 2e-6}
KAPPAS = [[0.3, 0.1, 0.2], [0.0, 0.0, 0.0], [0.5, 0.5, 0.5], [1.3, 0.1, -0.8]]


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

    def close(self):
        self.pc.pc_grid_destroy(self.h)


def _gpu_apply(pc, g, block, x, shift, dtype):
    import torch
    td = torch.complex64 if dtype == "c64" else torch.complex128
    xd = torch.from_numpy(np.ascontiguousarray(x.reshape(-1))).to(td).cuda()
    yd = torch.full_like(xd, complex(float("nan"), float("nan")))
    pc.pc_block_apply(g.h, block, xd, yd, shift=shift)
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.complex128).reshape(3, -1)


def _check(y, ref, tol):
    scale = np.abs(ref).max()
    assert np.all(np.isfinite(y))
    assert np.abs(y - ref).max() <= tol * scale
    assert np.linalg.norm(y - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("N", [4, 6, 8, 12, 16])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_block_apply_parity_small(pc, N, dtype):
    g = Grid(pc, two_phase_sphere(N, 0.35, 1))
    try:
        for kappa in KAPPAS:
            pc.pc_set_k(g.h, kappa)
            for block in (0, 1, 2, 3, -1):
                m = N ** 3 // 4 if block >= 0 else N ** 3
                x = complex_gaussian((3, m), 100 + block)
                for shift in (0.0, 0.73):
                    ref = (O.apply_block(g.pb, kappa, block, x, shift) if block >= 0
                           else O.apply_full(g.pb, kappa, x, shift))
                    _check(_gpu_apply(pc, g, block, x, shift, dtype), ref, TOL[dtype])
    finally:
        g.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_block_apply_parity_n48(pc, dtype):
    g = Grid(pc, two_phase_sphere(48, 0.35, 2))
    try:
        kappa = [0.3, 0.1, 0.2]
        pc.pc_set_k(g.h, kappa)
        for block in (0, 3, -1):
            m = 48 ** 3 // 4 if block >= 0 else 48 ** 3
            x = complex_gaussian((3, m), 5)
            ref = (O.apply_block(g.pb, kappa, block, x, 0.5) if block >= 0
                   else O.apply_full(g.pb, kappa, x, 0.5))
            _check(_gpu_apply(pc, g, block, x, 0.5, dtype), ref, TOL[dtype])
    finally:
        g.close()


def test_fractional_material_and_fcc_lattice(pc):
    N = 8
    cell = two_phase_sphere(N, 0.3, 2)
    cell.theta = np.random.default_rng(3).uniform(0, 1, N ** 3).astype(np.float32)
    cell.phase = None
    cell.a_lat = np.array([[0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]]) * 0.03
    g = Grid(pc, cell)
    try:
        kappa = [0.25, 0.5, 0.75]
        pc.pc_set_k(g.h, kappa)
        for block in (0, 2, -1):
            m = N ** 3 // 4 if block >= 0 else N ** 3
            x = complex_gaussian((3, m), 3)
            ref = (O.apply_block(g.pb, kappa, block, x, 0.2) if block >= 0
                   else O.apply_full(g.pb, kappa, x, 0.2))
            for dtype in ("c128", "c64"):
                _check(_gpu_apply(pc, g, block, x, 0.2, dtype), ref, TOL[dtype])
    finally:
        g.close()


def test_full_space_equals_sum_of_blocks(pc):
    import torch
    N = 16
    g = Grid(pc, two_phase_sphere(N, 0.35, 3))
    try:
        pc.pc_set_k(g.h, [0.1, -0.2, 0.35])
        x = torch.from_numpy(complex_gaussian(3 * N ** 3, 1)).cuda()
        y_full = torch.empty_like(x)
        pc.pc_block_apply(g.h, -1, x, y_full)
        y_sum = torch.zeros_like(x)
        for b in range(4):
            xb = torch.empty(3 * N ** 3 // 4, dtype=x.dtype, device="cuda")
            yb = torch.empty_like(xb)
            pc.pc_block_transfer(g.h, b, 0, x, xb)
            pc.pc_block_apply(g.h, b, xb, yb)
            pc.pc_block_transfer(g.h, b, 1, yb, y_sum)
        torch.cuda.synchronize()
        err = (y_full - y_sum).abs().max().item() / y_full.abs().max().item()
        assert err < 1e-14
    finally:
        g.close()


def test_mass_and_transfer(pc):
    import torch
    N = 8
    g = Grid(pc, two_phase_sphere(N, 0.35, 1))
    try:
        x = complex_gaussian((3, N ** 3), 2)
        xd = torch.from_numpy(x.reshape(-1)).cuda()
        rho = g.pb.node_rho()
        for b in range(4):
            idx = O.block_index(g.pb.dims, b)
            xb = torch.empty(3 * idx.size, dtype=xd.dtype, device="cuda")
            pc.pc_block_transfer(g.h, b, 0, xd, xb)
            assert np.array_equal(xb.cpu().numpy().reshape(3, -1), x[:, idx])
            yb = torch.empty_like(xb)
            pc.pc_block_mass(g.h, b, xb, yb)
            assert np.allclose(yb.cpu().numpy().reshape(3, -1), rho[idx][None, :] * x[:, idx],
                               rtol=1e-15, atol=0)
    finally:
        g.close()


def test_apply_argument_errors(pc):
    import torch
    g = Grid(pc, two_phase_sphere(8, 0.35, 1))
    try:
        x = torch.zeros(3 * 128, dtype=torch.complex128, device="cuda")
        with pytest.raises(pc.PcError):  # before pc_set_k
            pc.pc_block_apply(g.h, 0, x, torch.empty_like(x))
        pc.pc_set_k(g.h, [0, 0, 0])
        with pytest.raises(pc.PcError):
            pc.pc_block_apply(g.h, 4, x, torch.empty_like(x))
        with pytest.raises(pc.PcError):  # in place
            pc.pc_block_apply(g.h, 0, x, x)
        pc.pc_block_apply_many(g.h, 0, 0, x, torch.empty_like(x))  # count 0 is a no-op
    finally:
        g.close()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_block_apply_sampled_n160(pc, dtype):
    """Full-size grid of the apply benchmark (N = 160, R = 0.3, seed 3), one launch
    per block (pc_block_apply_many), checked on sampled outputs the oracle computes
    node by node."""
    import torch
    N = 160
    cell = two_phase_sphere(N, 0.3, 3)
    g = Grid(pc, cell)
    try:
        kappa = [0.3, 0.1, 0.2]
        pc.pc_set_k(g.h, kappa)
        nb = N ** 3 // 4
        rng = np.random.default_rng(11)
        X = N // 2
        for b in range(4):
            x = complex_gaussian((3, nb), 7 + b)
            td = torch.complex64 if dtype == "c64" else torch.complex128
            xd = torch.from_numpy(x.reshape(-1)).to(td).cuda()
            yd = torch.empty_like(xd)
            pc.pc_block_apply_many(g.h, b, 1, xd, yd, 0.4)
            torch.cuda.synchronize()
            y = yd.cpu().numpy().astype(np.complex128).reshape(3, -1)
            # random nodes plus the faces and edges of the quarter grid (wrap paths)
            t = rng.integers(0, nb, 1500)
            a = rng.integers(0, X, 300)
            bb = rng.integers(0, X, 300)
            k = rng.integers(0, N, 300)
            faces = np.concatenate([0 + X * (bb + X * k), (X - 1) + X * (bb + X * k),
                                    a + X * (0 + X * k), a + X * ((X - 1) + X * k),
                                    a + X * (bb + X * 0), a + X * (bb + X * (N - 1))])
            ts = np.unique(np.concatenate([t, faces]))
            ref = O.apply_block_at(g.pb, kappa, b, x, ts, 0.4)  # (len, 3)
            got = y[:, ts].T
            scale = np.abs(ref).max()
            assert np.abs(got - ref).max() <= TOL[dtype] * scale
    finally:
        g.close()


def test_register_staged_tma_and_row_kernels_agree(pc):
    """The register-staged kernel (PC_APPLY_KERNEL=legacy, used for odd quarter-grid widths), the
    TMA tile kernel (PC_APPLY_KERNEL=tma), the row-tile kernel (default for complex64 blocks) and
    the two-pass kernels (PC_APPLY_KERNEL=split, default for complex128) give the same operator,
    in both precisions, on a grid where all of them apply."""
    import subprocess
    import sys
    import os
    import tempfile
    code = r'''
import sys, numpy as np, torch
sys.path.insert(0, %r)
import paper_2606_03599_gb300 as pc
from workloads import complex_gaussian, two_phase_sphere
N = 24
cell = two_phase_sphere(N, 0.35, 5)
g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
pc.pc_set_k(g, [0.3, -0.2, 0.1])
out = []
for b in (0, 3, -1):
    m = N ** 3 // 4 if b >= 0 else N ** 3
    for dt in (torch.complex128, torch.complex64):
        x = torch.from_numpy(complex_gaussian(3 * m, 11)).to(dt).cuda()
        y = torch.empty_like(x)
        pc.pc_block_apply(g, b, x, y, 0.3)
        out.append(y.cpu().numpy().astype(np.complex128))
torch.cuda.synchronize()
np.save(sys.argv[1], np.concatenate(out))
'''
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = {}
    tmp = tempfile.mkdtemp()
    for mode in ("legacy", "tma", "row", "split"):
        path = os.path.join(tmp, "kernel_ab_%s.npy" % mode)
        env = dict(os.environ, PC_APPLY_KERNEL=mode)
        subprocess.run([sys.executable, "-c", code % root, path], check=True, env=env)
        res[mode] = np.load(path)
    a = res["legacy"]
    for mode in ("tma", "row", "split"):
        assert np.abs(a - res[mode]).max() <= 2e-6 * np.abs(a).max(), mode
