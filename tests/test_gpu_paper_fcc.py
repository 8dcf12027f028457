"""The paper's own FCC example on its 128^3 grid: low-quartz matrix, silicon sphere
(R = a0/4), sub-pixel inclusion fractions, FCC primitive cell (Sec. 7.1), against the grouped
band frequencies the paper prints for its own 128^3 result (tests/golden/paper_table2.json).

Readings (each decided by the printed values, which an independent computation can only
match under one of them):

* The Bloch vectors the paper lists for its FCC path, e.g. X = (0, 1/2, 1/2), are used in its
  computation as Cartesian wave vectors in units of 2 pi / a0, i.e. kappa_l = a_l . k / a0 in
  the reduced coordinates of the library.  Read as reduced coordinates only Gamma and L (the
  two points both readings share) agree with the table.
* At Gamma the paper counts the 12 zero-derivative modes among its bands (they sit at the
  deflation shift d0), so its group G7 (bands 25-28) is the 13th-16th non-zero frequencies.
* The paper's K and U rows are identical in every column although K and U are not
  equivalent for the trigonal quartz matrix under either reading; they are computed and
  printed here but not asserted.

Tolerance 1e-3 relative: the paper does not define which cell a node's inclusion fraction
is taken over (here: the reduced cube of side 1/N centred on the node, 8^3 sub-samples) and
prints 5 significant digits.
"""

import json
import os

import numpy as np
import pytest

from workloads import FCC_POINTS, fcc_lattice, fcc_quartz_silicon_cell
from workloads.materials import FCC_A0

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fcc_quartz_silicon_matches_paper_table():
    import torch
    import paper_2606_03599_gb300 as pc
    assert torch.cuda.is_available()
    with open(os.path.join(HERE, "golden", "paper_table2.json")) as f:
        table = json.load(f)
    N = table["grid"]
    cell = fcc_quartz_silicon_cell(N)
    g = pc.pc_grid_create(N, cell.C, cell.rho, theta=cell.theta, a_lat=cell.a_lat)
    try:
        opt = pc.pc_options_default(tol=1e-8, precision=pc.PC_PREC_MIXED, autotune=1)
        A = fcc_lattice()
        worst = 0.0
        for e in table["entries"]:
            grp = e["group"]
            zero_modes = 12 if e["point"] == "G" else 0
            first = 4 * (grp - 1) - zero_modes  # 0-based index of the group's first non-zero band
            kappa = A.T @ FCC_POINTS[e["point"]] / FCC_A0  # Cartesian (2 pi / a0 units) -> reduced
            ev, _, info = pc.pc_eigs(g, kappa, first + 4, opt=opt)
            assert info["max_rel_resid"] <= 1e-8
            f = np.sqrt(ev) / (2 * np.pi)
            mean = float(np.mean(f[first:first + 4]))
            rel = abs(mean - e["present_hz"]) / e["present_hz"]
            print("%s G%d: %.1f Hz (paper %.4e), relative difference %.2e" % (e["point"], grp, mean,
                                                                            e["present_hz"], rel))
            if e["point"] in ("K", "U"):
                continue
            worst = max(worst, rel)
            assert rel <= 1e-3, (e, mean, rel)
        print("worst relative difference to the paper's 128^3 result (G, X, W, L): %.2e" % worst)
    finally:
        pc.pc_grid_destroy(g)
