"""Mixed precision (complex64 inner PCG, FP64 outer Krylov with FP64 residual
refinement) reproduces the FP64 eigenvalues, on a heterogeneous cell, per band."""

import numpy as np
import pytest

from workloads import two_phase_sphere

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_03599_gb300 as pc
    return pc


@pytest.mark.parametrize("kappa", [[0.25, 0.0, 0.0], [0.5, 0.5, 0.0], [0.0, 0.0, 0.0]])
def test_mixed_matches_fp64_per_band(pc, kappa):
    N = 32
    cell = two_phase_sphere(N, 0.3, 12)
    g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    try:
        ev64, b64, i64 = pc.pc_eigs(g, kappa, 20, opt=pc.pc_options_default(precision=pc.PC_PREC_FP64))
        evmx, bmx, imx = pc.pc_eigs(g, kappa, 20, opt=pc.pc_options_default(precision=pc.PC_PREC_MIXED))
        rel = np.abs(evmx - ev64) / ev64
        assert rel.max() <= 1e-10, rel
        assert imx["max_rel_resid"] <= 1e-8 and i64["max_rel_resid"] <= 1e-8
    finally:
        pc.pc_grid_destroy(g)


def test_blocked_equals_full_space(pc):
    """Merged four-block spectrum = full-space spectrum (Cor. 4.2) on the GPU."""
    N = 24
    cell = two_phase_sphere(N, 0.35, 2)
    g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    try:
        for kappa in ([0.3, 0.1, 0.2], [0.0, 0.0, 0.0]):
            evb, _, _ = pc.pc_eigs(g, kappa, 16)
            evf, _, _ = pc.pc_eigs(g, kappa, 16, opt=pc.pc_options_default(full_space=1))
            assert np.abs(evb - evf).max() / evf.max() <= 1e-10
    finally:
        pc.pc_grid_destroy(g)
