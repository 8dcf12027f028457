"""The stencil-launch autotuner: tuned launches keep parity with the oracle, the tuned choice is
reported, persisted to and read back from the PC_TUNE_CACHE file, and eigen-solves with
autotuning give the same eigenvalues."""

import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

from oracle import oracle as O
from workloads import complex_gaussian, two_phase_sphere

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pc():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_03599_gb300 as pc
    return pc


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_tuned_batch_apply_matches_oracle(pc, dtype):
    import torch
    N = 32
    cell = two_phase_sphere(N, 0.35, 7)
    g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    try:
        C0, rho0, L = pc.pc_grid_units(g)
        pb = O.problem_from_cell(cell, C0=C0, rho0=rho0, L=L)
        kappa = [0.3, 0.1, 0.2]
        pc.pc_set_k(g, kappa)
        code = pc.PC_C64 if dtype == "c64" else pc.PC_C128
        pc.pc_autotune(g, code, 2, 8)
        kind, shape, tz, ctas = pc.pc_tuned_config(g, code, 0, 8)
        assert kind in (0, 1, 2, 3, 4) and ctas >= 1 and (kind not in (2, 4) or dtype == "c64")
        td = torch.complex64 if dtype == "c64" else torch.complex128
        nb = N ** 3 // 4
        blocks = [0, 1, 2, 3, 0, 1, 2, 3]
        xs = [torch.from_numpy(complex_gaussian(3 * nb, 100 + i)).to(td).cuda() for i in range(8)]
        ys = [torch.empty_like(x) for x in xs]
        pc.pc_apply_batch(g, blocks, xs, ys, [0.25] * 8)
        torch.cuda.synchronize()
        tol = 2e-6 if dtype == "c64" else 1e-12
        for i in (0, 3, 6):
            ref = O.apply_block(pb, kappa, blocks[i], xs[i].cpu().numpy().astype(np.complex128).reshape(3, nb),
                                shift=0.25)
            got = ys[i].cpu().numpy().astype(np.complex128).reshape(3, nb)
            assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    finally:
        pc.pc_grid_destroy(g)


def test_tune_cache_file_round_trip(pc):
    code = r'''
import sys
sys.path.insert(0, %r)
import paper_2606_03599_gb300 as pc
from workloads import two_phase_sphere
cell = two_phase_sphere(24, 0.35, 3)
g = pc.pc_grid_create(24, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
pc.pc_set_k(g, [0.1, 0.2, 0.3])
if sys.argv[1] == "tune":
    pc.pc_autotune(g, pc.PC_C128, 0, 4)
print(pc.pc_tuned_config(g, pc.PC_C128, 0, 4))
pc.pc_grid_destroy(g)
''' % ROOT
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.json")
        env = dict(os.environ, PC_TUNE_CACHE=path)
        a = subprocess.run([sys.executable, "-c", code, "tune"], env=env, capture_output=True, text=True, check=True)
        lines = open(path).read().splitlines()
        assert len(lines) == 1 and lines[0].startswith('"12,12,24,c128,blocks,phase,cubic,n4,sm')
        b = subprocess.run([sys.executable, "-c", code, "read"], env=env, capture_output=True, text=True, check=True)
        assert a.stdout.strip() == b.stdout.strip()
        assert open(path).read().splitlines() == lines  # reading does not retune


def test_eigs_with_autotune_same_eigenvalues(pc):
    N = 24
    cell = two_phase_sphere(N, 0.35, 2)
    g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    try:
        for prec in (pc.PC_PREC_FP64, pc.PC_PREC_MIXED):
            ev0, _, _ = pc.pc_eigs(g, [0.25, 0.0, 0.1], 12, opt=pc.pc_options_default(precision=prec))
            ev1, _, _ = pc.pc_eigs(g, [0.25, 0.0, 0.1], 12, opt=pc.pc_options_default(precision=prec, autotune=1))
            assert np.allclose(ev0, ev1, rtol=1e-10, atol=0)
    finally:
        pc.pc_grid_destroy(g)


def test_autotune_errors(pc):
    cell = two_phase_sphere(8, 0.35, 1)
    g = pc.pc_grid_create(8, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    try:
        with pytest.raises(pc.PcError):
            pc.pc_autotune(g, pc.PC_C64, 0, 4)  # no Bloch vector yet
        pc.pc_set_k(g, [0.1, 0.0, 0.0])
        for args in ((3, 0, 4), (pc.PC_C64, 3, 4), (pc.PC_C64, 0, 0), (pc.PC_C64, 0, 65)):
            with pytest.raises(pc.PcError):
                pc.pc_autotune(g, *args)
    finally:
        pc.pc_grid_destroy(g)


def test_apply_timing_through_graph_replays(pc):
    """With event timing on, the stencil applies replayed inside the PCG's CUDA graphs are timed
    and counted like eager ones, and the eigenvalues do not change."""
    N = 24
    cell = two_phase_sphere(N, 0.35, 4)
    g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    try:
        opt = pc.pc_options_default()
        ev0, _, _ = pc.pc_eigs(g, [0.1, 0.3, 0.0], 8, opt=opt)
        pc.pc_stats_reset()
        pc.pc_stats_timing(1)
        try:
            ev1, _, info = pc.pc_eigs(g, [0.1, 0.3, 0.0], 8, opt=opt)
        finally:
            pc.pc_stats_timing(0)
        st = pc.pc_stats_get()
        assert np.allclose(ev0, ev1, rtol=1e-12, atol=0)
        assert st["apply_launches"] > 20
        # one timing per batched apply call; a call of more items than one launch holds may launch twice
        assert 0.5 * st["apply_launches"] <= st["apply_timed"][1] <= st["apply_launches"]
        assert st["apply_ms"][1] > 0
    finally:
        pc.pc_grid_destroy(g)


@pytest.mark.parametrize("side_stream", [False, True])
def test_timed_apply_nodes_count_only_items_that_ran(pc, side_stream):
    """PCG runs its iterations in chunks of four (replayed as a CUDA graph on a side stream); once
    the system has converged, or reached maxit, the rest of the chunk's applies skip it on the
    device.  The timed node count holds only the applies that ran: one block per iteration."""
    import torch
    N = 16
    cell = two_phase_sphere(N, 0.35, 4)
    g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    try:
        pc.pc_set_k(g, [0.3, 0.1, 0.2])
        nb = N ** 3 // 4
        rhs = torch.from_numpy(complex_gaussian(3 * nb, 21)).cuda()
        x = torch.empty_like(rhs)
        stream = torch.cuda.Stream() if side_stream else None
        sigma = pc.pc_default_sigma(g)
        for tol, maxit in ((1e-10, 400), (1e-12, 1), (1e-12, 6)):
            pc.pc_shift_invert_pcg(g, 1, sigma, rhs, x, tol=tol, maxit=maxit, stream=stream,
                                   raise_on_fail=False)  # warm-up: workspace and graph
            torch.cuda.synchronize()
            pc.pc_stats_reset()
            pc.pc_stats_timing(1)
            try:
                r = pc.pc_shift_invert_pcg(g, 1, sigma, rhs, x, tol=tol, maxit=maxit, stream=stream,
                                           raise_on_fail=False)
            finally:
                pc.pc_stats_timing(0)
            st = pc.pc_stats_get()
            launched = st["apply_timed"][1]
            assert launched >= r["iters"] and launched % 4 == 0, (launched, r)
            assert st["apply_nodes"][1] == r["iters"] * nb, (st["apply_nodes"], r, launched)
            assert st["apply_nodes_launched"][1] == launched * nb
            if maxit < 400:
                assert r["iters"] == maxit and launched > maxit
    finally:
        pc.pc_grid_destroy(g)
