"""The benchmarked N = 48 cell against eigenvalues the oracle alone computed.

tests/golden/arpack_n48.json holds, for the FP64 band workload (two-phase simple-cubic cell,
N = 48, sphere R = 0.35, seed 2) at Gamma, X and kappa = (0.3, 0.1, 0.2), the lowest non-zero
eigenvalues of every parity block from the oracle's ARPACK shift-invert solve with an exact
sparse LU (written by tests/golden/make_arpack_n48.py, which calls only oracle/), and the
merged lowest 20 (Theorem 4.1 / Cor. 4.2).  A true residual bounds each returned eigenvalue's
distance to the spectrum but cannot show that none was skipped; this comparison does.

* pc_eigs (FP64, and mixed precision with FP64 refinement) returns the merged 20, band by band,
  to 1e-10 relative, and each value's source block holds it in the oracle's block spectrum.
* pc_eigs_multi on the three Bloch vectors in lockstep returns the same.
"""

import json
import os

import numpy as np
import pytest

from workloads import config_cell

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "arpack_n48.json")


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        g = json.load(f)
    assert all(p["complete"] for p in g["points"])
    return g


@pytest.fixture(scope="module")
def grid():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_03599_gb300 as pc
    cell = config_cell("fp64")
    h = pc.pc_grid_create(cell.N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    yield pc, h
    pc.pc_grid_destroy(h)


def _check(point, ev, blocks):
    ref = np.array(point["merged"])
    assert ev.shape == ref.shape
    assert np.abs(ev - ref).max() <= 1e-10 * ref.max(), (point["name"], np.abs(ev - ref).max() / ref.max())
    for v, b in zip(ev, blocks):
        spec = np.array(point["blocks"][b])
        assert np.abs(spec - v).min() <= 1e-10 * ref.max(), (point["name"], v, b)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("index", [0, 1, 2])
def test_pc_eigs_equals_the_oracle_arpack_spectrum(golden, grid, precision, index):
    pc, h = grid
    point = golden["points"][index]
    prec = pc.PC_PREC_FP64 if precision == "fp64" else pc.PC_PREC_MIXED
    ev, blocks, info = pc.pc_eigs(h, point["kappa"], golden["nev_merged"], opt=pc.pc_options_default(precision=prec))
    assert info["max_rel_resid"] <= 1e-8
    _check(point, ev, blocks)


def test_pc_eigs_multi_equals_the_oracle_arpack_spectrum(golden, grid):
    pc, h = grid
    ks = np.array([p["kappa"] for p in golden["points"]])
    ev, blocks, infos = pc.pc_eigs_multi(h, ks, golden["nev_merged"],
                                         opt=pc.pc_options_default(precision=pc.PC_PREC_MIXED))
    for i, point in enumerate(golden["points"]):
        assert infos[i]["status"] == pc.PC_OK
        _check(point, ev[i], blocks[i])
