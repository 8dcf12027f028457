"""Several Bloch vectors of one grid in one launch (Sec. 6.3: the block subproblems of every Bloch
vector are independent), through the C ABI, against the oracle and against one-at-a-time solves.

* pc_apply_batch_k: items of mixed parity blocks and Bloch slots in one batch equal the oracle's
  block apply at each item's own Bloch vector (complex128 1e-12, complex64 2e-6), for the default
  kernels (one launch for all slots) and for launch shapes that run once per slot.
* pc_eigs_multi: the lowest eigenvalues at four Bloch vectors (Gamma, X, M, a generic vector)
  solved in lockstep equal four pc_eigs calls (1e-10 relative, FP64 and mixed precision), with the
  zero modes deflated at Gamma only and every true residual below the tolerance.
* pc_eigs_batch with lockstep chunks equals pc_eigs per Bloch vector on ragged grids; so do
  lockstep solves of the full space and of a nodewise material.
* Grids whose block transform falls back to the library FFT accept one Bloch vector at a time.
"""

import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import oracle as O
from workloads import complex_gaussian, two_phase_sphere

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KAPPAS = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [0.5, 0.5, 0.0], [0.3, 0.1, 0.2]])


@pytest.fixture(scope="module")
def pc():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_03599_gb300 as pc
    return pc


def _apply_case(pc, N, dtype, tol):
    import torch
    cell = two_phase_sphere(N, 0.35, 4)
    g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    try:
        C0, rho0, L = pc.pc_grid_units(g)
        pb = O.problem_from_cell(cell, C0=C0, rho0=rho0, L=L)
        kap = np.array([[0.3, 0.1, 0.2], [0.0, 0.0, 0.0], [0.7, -0.4, 1.3]])
        pc.pc_set_k_multi(g, kap)
        nb = N ** 3 // 4
        blocks = [0, 3, 1, 2, 2, 0, 1, 3, 0]
        slots = [0, 1, 2, 2, 0, 1, 1, 0, 2]
        shifts = [0.25 * i - 0.5 for i in range(len(blocks))]
        xs, ys, xh = [], [], []
        for i in range(len(blocks)):
            x = complex_gaussian((3, nb), 100 + i)
            xh.append(x)
            xd = torch.from_numpy(x.reshape(-1).astype(dtype)).cuda()
            xs.append(xd)
            ys.append(torch.full_like(xd, complex(float("nan"), float("nan"))))
        pc.pc_apply_batch_k(g, blocks, slots, xs, ys, shifts)
        torch.cuda.synchronize()
        for i in range(len(blocks)):
            ref = O.apply_block(pb, kap[slots[i]], blocks[i], xh[i], shift=shifts[i]).reshape(-1)
            got = ys[i].cpu().numpy()
            err = np.abs(got - ref).max() / np.abs(ref).max()
            assert err <= tol, (i, blocks[i], slots[i], err)
    finally:
        pc.pc_grid_destroy(g)


@pytest.mark.parametrize("N", [8, 12, 16])
def test_apply_batch_k_complex128_matches_oracle(pc, N):
    _apply_case(pc, N, np.complex128, 1e-12)


@pytest.mark.parametrize("N", [8, 12, 16, 32])
def test_apply_batch_k_complex64_matches_oracle(pc, N):
    _apply_case(pc, N, np.complex64, 2e-6)


_CHILD = r"""
import sys
sys.path.insert(0, %r)
import numpy as np, torch
import paper_2606_03599_gb300 as pc
sys.path.insert(0, %r)
from test_gpu_multik import _apply_case
_apply_case(pc, 16, np.complex64, 2e-6)
_apply_case(pc, 12, np.complex128, 1e-12)
print("CHILD-OK")
"""


@pytest.mark.parametrize("kernel", ["tma", "row", "legacy"])
def test_apply_batch_k_per_slot_launch_shapes(kernel):
    # launch shapes with grid-uniform phases run once per run of equal slots
    env = dict(os.environ, PC_APPLY_KERNEL=kernel)
    code = _CHILD % (ROOT, os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "CHILD-OK" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_eigs_multi_equals_one_at_a_time(pc, precision):
    N = 16
    cell = two_phase_sphere(N, 0.35, 2)
    g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    try:
        prec = pc.PC_PREC_FP64 if precision == "fp64" else pc.PC_PREC_MIXED
        opt = pc.pc_options_default(precision=prec)
        assert pc.pc_eigs_multi_max(g) == 32
        ev, bo, infos = pc.pc_eigs_multi(g, KAPPAS, 12, opt=opt)
        # the grid's current Bloch vector is the first one afterwards
        import torch
        x = torch.from_numpy(complex_gaussian((3, N ** 3 // 4), 5).reshape(-1)).cuda()
        y = torch.empty_like(x)
        pc.pc_block_apply(g, 1, x, y)
        C0, rho0, L = pc.pc_grid_units(g)
        pb = O.problem_from_cell(cell, C0=C0, rho0=rho0, L=L)
        ref = O.apply_block(pb, KAPPAS[0], 1, x.cpu().numpy().reshape(3, -1)).reshape(-1)
        assert np.abs(y.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
        for i, k in enumerate(KAPPAS):
            assert infos[i]["status"] == pc.PC_OK
            assert infos[i]["max_rel_resid"] <= 1e-8
            assert infos[i]["zero_modes"] == (12 if i == 0 else 0)
            e1, b1, _ = pc.pc_eigs(g, k, 12, opt=opt)
            assert np.abs(ev[i] - e1).max() <= 1e-10 * e1.max(), (i, ev[i], e1)
            # blocks of degenerate values may swap; the multiset per value must agree
            for v in np.unique(np.round(e1 / e1.max(), 8)):
                sel1 = np.abs(e1 / e1.max() - v) < 1e-8
                sel2 = np.abs(ev[i] / e1.max() - v) < 1e-8
                assert sorted(b1[sel1]) == sorted(bo[i][sel2])
    finally:
        pc.pc_grid_destroy(g)


def test_eigs_multi_matches_dense_at_n8(pc):
    N = 8
    cell = two_phase_sphere(N, 0.35, 1)
    g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    try:
        C0, rho0, L = pc.pc_grid_units(g)
        pb = O.problem_from_cell(cell, C0=C0, rho0=rho0, L=L)
        ev, _, infos = pc.pc_eigs_multi(g, KAPPAS, 12)
        to_si = C0 / (rho0 * L * L)
        for i, k in enumerate(KAPPAS):
            ref = O.lowest_nonzero(O.dense_eigvals(pb, k), 12) * to_si
            assert np.abs(ev[i] - ref).max() <= 1e-10 * ref.max(), (i, ev[i], ref)
    finally:
        pc.pc_grid_destroy(g)


def test_eigs_batch_lockstep_chunks_equal_pc_eigs(pc):
    sizes = [8, 12, 16]
    cells = [two_phase_sphere(N, 0.3, 10 + i) for i, N in enumerate(sizes)]
    grids = [pc.pc_grid_create(c.N, c.C, c.rho, phase=c.phase, a_lat=c.a_lat) for c in cells]
    try:
        ks = np.array([[0.1 * i, 0.05 * i, 0.0] for i in range(6)])
        opt = pc.pc_options_default(precision=pc.PC_PREC_MIXED, kbatch=4)
        evs, _, st, info = pc.pc_eigs_batch(grids, [ks] * 3, 8, opt=opt, workers=2)
        assert info["kpoints"] == 18 and info["failed"] == 0
        for g, ev, s in zip(grids, evs, st):
            assert (s == 0).all()
            for i in (0, 3, 5):
                e1, _, _ = pc.pc_eigs(g, ks[i], 8, opt=pc.pc_options_default(precision=pc.PC_PREC_MIXED))
                assert np.abs(ev[i] - e1).max() <= 1e-10 * e1.max()
    finally:
        for g in grids:
            pc.pc_grid_destroy(g)


def test_fallback_fft_grid_solves_one_vector_at_a_time(pc):
    N = 34  # N/2 = 17: prime above the own transform's factor limit
    cell = two_phase_sphere(N, 0.3, 3)
    g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    try:
        assert pc.pc_eigs_multi_max(g) == 1
        with pytest.raises(pc.PcError) as ei:
            pc.pc_eigs_multi(g, KAPPAS[:2], 4)
        assert ei.value.code == pc.PC_EINVAL
        ev, _, infos = pc.pc_eigs_multi(g, KAPPAS[3:], 4)
        e1, _, _ = pc.pc_eigs(g, KAPPAS[3], 4)
        assert np.abs(ev[0] - e1).max() <= 1e-10 * e1.max()
    finally:
        pc.pc_grid_destroy(g)


def test_eigs_multi_full_space_equals_one_at_a_time(pc):
    """Lockstep solves of the full space (one space per Bloch vector, the preconditioner through the
    four block transforms of each vector's slot) equal pc_eigs per Bloch vector."""
    N = 12
    cell = two_phase_sphere(N, 0.35, 5)
    g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    try:
        opt = pc.pc_options_default(full_space=1)
        ev, bo, infos = pc.pc_eigs_multi(g, KAPPAS, 10, opt=opt)
        for i, k in enumerate(KAPPAS):
            assert infos[i]["status"] == pc.PC_OK and (bo[i] == -1).all()
            e1, _, _ = pc.pc_eigs(g, k, 10, opt=opt)
            assert np.abs(ev[i] - e1).max() <= 1e-10 * e1.max()
    finally:
        pc.pc_grid_destroy(g)


def test_eigs_multi_nodewise_material_equals_one_at_a_time(pc):
    """A nodewise material (two-pass complex128 kernels with per-node stiffness) solved at several
    Bloch vectors in lockstep equals pc_eigs per Bloch vector."""
    from paper_2606_03599_gb300 import autodiff
    N = 12
    cell = two_phase_sphere(N, 0.35, 6)
    C21, rho = autodiff.two_phase_nodewise(cell)
    rng = np.random.default_rng(3)
    rho = rho * (1 + 0.1 * rng.uniform(size=rho.shape))
    g = pc.pc_grid_create_nodewise(N, C21, rho, a_lat=cell.a_lat)
    try:
        ev, _, infos = pc.pc_eigs_multi(g, KAPPAS, 8)
        for i, k in enumerate(KAPPAS):
            assert infos[i]["status"] == pc.PC_OK
            e1, _, _ = pc.pc_eigs(g, k, 8)
            assert np.abs(ev[i] - e1).max() <= 1e-10 * e1.max()
    finally:
        pc.pc_grid_destroy(g)
