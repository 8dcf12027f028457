"""The allocation-free apply-with-inner-product entry point against the regular apply.

Some callers cannot let a library allocate device memory (their own pool owns
the GPU, or cudaMalloc's implicit synchronisation is too costly for them);
pc_block_apply_dot_noalloc serves them with scratch in a static device array.
This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test; it also passes on its own.
"""

import numpy as np
import pytest

from workloads import complex_gaussian, two_phase_sphere

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 2e-6}


@pytest.fixture(scope="module")
def pc():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_03599_gb300 as pc
    return pc


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("block", [0, 3, -1])
def test_noalloc_matches_regular_apply_twice(pc, dtype, block):
    import torch
    N = 16
    cell = two_phase_sphere(N, 0.35, 1)
    g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    try:
        pc.pc_set_k(g, [0.3, 0.1, 0.2])
        td = torch.complex128 if dtype == "c128" else torch.complex64
        m = N ** 3 // 4 if block >= 0 else N ** 3
        for call in range(2):  # two calls in a row share the static scratch
            x = torch.from_numpy(complex_gaussian(3 * m, 40 + call)).to(td).cuda()
            y_ref = torch.empty_like(x)
            pc.pc_block_apply(g, block, x, y_ref, shift=0.6)
            y = torch.full_like(x, complex(float("nan"), float("nan")))
            dot = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            pc.pc_block_apply_dot_noalloc(g, block, x, y, dot, shift=0.6)
            torch.cuda.synchronize()
            yr = y_ref.cpu().numpy().astype(np.complex128)
            yn = y.cpu().numpy().astype(np.complex128)
            assert np.abs(yn - yr).max() <= TOL[dtype] * np.abs(yr).max()
            xn = x.cpu().numpy().astype(np.complex128)
            ref_dot = np.real(np.vdot(xn, yr))
            assert abs(dot.item() - ref_dot) <= TOL[dtype] * np.linalg.norm(xn) * np.linalg.norm(yr)
    finally:
        pc.pc_grid_destroy(g)


@pytest.mark.parametrize("N", [186, 254])
def test_noalloc_complex128_full_space_inside_the_limit(pc, N):
    """Full-space complex128 grids inside the documented 2^24-node limit whose default launch
    would need more CTAs than the static scratch holds (4x4 tiles: 2209 at N = 186, 4096 at
    N = 254) are accepted and computed with a smaller launch: y on sampled nodes (random and on
    the Bloch-wrap faces) against the oracle, and *dot against the inner product of the returned
    y with x."""
    import torch
    from oracle import oracle as O
    cell = two_phase_sphere(N, 0.3, 2)
    g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    try:
        kappa = [0.3, 0.1, 0.2]
        pc.pc_set_k(g, kappa)
        C0, rho0, L = pc.pc_grid_units(g)
        pb = O.problem_from_cell(cell, C0=C0, rho0=rho0, L=L)
        n = N ** 3
        xh = complex_gaussian((3, n), 77)
        x = torch.from_numpy(xh.reshape(-1)).cuda()
        y = torch.full_like(x, complex(float("nan"), float("nan")))
        dot = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        pc.pc_block_apply_dot_noalloc(g, -1, x, y, dot, shift=0.4)
        torch.cuda.synchronize()
        yh = y.cpu().numpy().reshape(3, n)
        assert np.isfinite(yh).all()
        rng = np.random.default_rng(5)
        i, j, k = (rng.integers(0, N, 150) for _ in range(3))
        faces = np.concatenate([0 + N * (j + N * k), (N - 1) + N * (j + N * k), i + N * (0 + N * k),
                                i + N * ((N - 1) + N * k), i + N * (j + N * 0), i + N * (j + N * (N - 1))])
        nodes = np.unique(np.concatenate([rng.integers(0, n, 600), faces]))
        ref = O.apply_at_nodes(pb, kappa, xh, nodes, 0.4)
        assert np.abs(yh[:, nodes].T - ref).max() <= 1e-12 * np.abs(ref).max()
        ref_dot = float(np.real(np.vdot(xh.reshape(-1), yh.reshape(-1))))
        assert abs(dot.item() - ref_dot) <= 1e-12 * np.linalg.norm(xh) * np.linalg.norm(yh)
    finally:
        pc.pc_grid_destroy(g)


def test_noalloc_rejects_grids_beyond_the_static_limit(pc):
    import torch
    N = 258  # 258^3 nodes > 2^24
    cell = two_phase_sphere(N, 0.3, 1)
    g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    try:
        pc.pc_set_k(g, [0.1, 0.2, 0.3])
        x = torch.zeros(16, dtype=torch.complex128, device="cuda")
        y = torch.zeros_like(x)
        dot = torch.zeros(1, dtype=torch.float64, device="cuda")
        with pytest.raises(pc.PcError) as ei:
            pc.pc_block_apply_dot_noalloc(g, -1, x, y, dot)
        assert ei.value.code == pc.PC_EINVAL and "static-scratch limit" in str(ei.value)
    finally:
        pc.pc_grid_destroy(g)
