"""Batched band solves over ragged grids and many Bloch vectors (pc_eigs_batch): the batch
returns the eigenvalues pc_eigs returns one Bloch vector at a time, the clones it solves on
apply the same operator, and a spot check against the dense oracle."""

import numpy as np
import pytest

from oracle import oracle as O
from workloads import complex_gaussian, two_phase_sphere
from workloads.kpath import sc_uniform_path

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_03599_gb300 as pc
    return pc


def _grid(pc, N, seed):
    cell = two_phase_sphere(N, 0.3, seed)
    return cell, pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_one_at_a_time(pc, precision):
    prec = pc.PC_PREC_FP64 if precision == "fp64" else pc.PC_PREC_MIXED
    grids = [_grid(pc, N, 30 + i)[1] for i, N in enumerate((16, 24, 32))]
    ks = [sc_uniform_path(12)[i::4][:3] for i in range(3)]
    try:
        opt = pc.pc_options_default(precision=prec, autotune=1)
        evs, blocks, status, info = pc.pc_eigs_batch(grids, ks, 10, opt=opt, workers=3)
        assert info["kpoints"] == 9 and info["failed"] == 0 and info["workers"] == 3
        assert info["max_rel_resid"] <= 1e-8
        for g, kk, ev in zip(grids, ks, evs):
            for k, e in zip(kk, ev):
                ref, _, _ = pc.pc_eigs(g, k, 10, opt=pc.pc_options_default(precision=prec))
                assert np.allclose(e, ref, rtol=1e-10, atol=0)
        assert all((s == 0).all() for s in status)
    finally:
        for g in grids:
            pc.pc_grid_destroy(g)


def test_batch_matches_dense_oracle_n8(pc):
    cell, g = _grid(pc, 8, 5)
    try:
        C0, rho0, L = pc.pc_grid_units(g)
        pb = O.problem_from_cell(cell, C0=C0, rho0=rho0, L=L)
        ks = np.array([[0.3, 0.1, 0.2], [0.5, 0.5, 0.0]])
        evs, _, _, _ = pc.pc_eigs_batch([g], [ks], 8, workers=2)
        for k, ev in zip(ks, evs[0]):
            dense = np.sort(np.concatenate([O.dense_eigvals(pb, k, b) for b in range(4)]))
            dense = dense[dense > 1e-9 * dense.max()][:8] * C0 / (rho0 * L ** 2)
            assert np.allclose(ev, dense, rtol=1e-10, atol=0)
    finally:
        pc.pc_grid_destroy(g)


def test_clone_applies_the_same_operator(pc):
    import torch
    cell, g = _grid(pc, 16, 9)
    h = pc.pc_grid_clone(g)
    try:
        for grid in (g, h):
            pc.pc_set_k(grid, [0.2, -0.1, 0.35])
        x = torch.from_numpy(complex_gaussian(3 * 16 ** 3 // 4, 3)).cuda()
        y0, y1 = torch.empty_like(x), torch.empty_like(x)
        pc.pc_block_apply(g, 2, x, y0, 0.5)
        pc.pc_block_apply(h, 2, x, y1, 0.5)
        torch.cuda.synchronize()
        assert torch.equal(y0, y1)
        assert pc.pc_grid_units(g) == pc.pc_grid_units(h)
    finally:
        pc.pc_grid_destroy(h)
        pc.pc_grid_destroy(g)


def test_batch_rejects_bad_jobs(pc):
    cell, g = _grid(pc, 8, 1)
    try:
        with pytest.raises(pc.PcError):
            pc.pc_eigs_batch([g], [np.zeros((1, 3))], 0)
        with pytest.raises(pc.PcError):
            pc.pc_eigs_batch([], [], 4)
    finally:
        pc.pc_grid_destroy(g)
