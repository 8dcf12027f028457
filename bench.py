#!/usr/bin/env python
"""Benchmark of the GB300 parity-blocked band solver.

One step = one chunk of --kbatch (default 16) consecutive Bloch vectors of the
plain FP64 workload: a seeded two-phase simple-cubic cell (N = 48, sphere
R = 0.35, seed 2), the Gamma-X-M-Gamma-R-X path of 31 k-points (6 intervals per
segment), the lowest 20 non-zero bands at true relative residual 1e-8, solved on
the four parity blocks with the shift-invert Krylov-Schur eigensolver and merged.
The Bloch vectors of a chunk are solved in lockstep (pc_eigs_multi: one batched
inner PCG, Gram and residual launch over all (Bloch vector, block) spaces).  A
step runs every step of the hot path: Bloch phases and Fourier symbol tables,
fused block applies, preconditioned inner CG, Gamma deflation,
orthogonalisation and Rayleigh-Ritz, FP64 true residuals and the block merge.

Printed JSON (one line, rank 0):
  value     = seconds per k-point for the whole job (max over ranks of the
              timed device time / k-points processed by all ranks)
  apply     = complex64 and complex128 four-block apply throughput at N = 160
              (GDoF/s, algorithmic HBM fraction)
  roofline  = the dominant kernel of the step (the FP64 stencil apply), its
              device time measured with CUDA events on its launch stream
  e2e       = the same metric through the C ABI from host material buffers
  cpu_baseline = the FP64 CPU oracle on the host cores (bounded sample)

``--impl reference`` times the CPU oracle as the reference arm instead.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "block B C B^H apply GDoF/s & HBM frac; sec per k-point for 20 bands @1e-8 resid"
# block applies per k-point of the FP64 band workload, as the GPU arm measures them on GB300
# (solver.block_applies_per_kpoint: the PCG iterations and true-residual checks of one k-point, items
# of converged systems not counted); the reference arm scales its per-apply time by it
APPLIES_PER_KPOINT_MEASURED = 5136
WORKLOAD = ("two-phase SC cell N=48 (R=0.35, seed 2), 31-point Gamma-X-M-Gamma-R-X path, 20 bands, resid 1e-8, "
            "FP64; Bloch vectors solved in lockstep chunks of --kbatch")
NEV = 20
TOL = 1e-8
# algorithmic cost of one stencil apply per node (cubic lattice, binary material):
#   bytes: read x (3 complex) + write y (3 complex) + 1 material byte
#   flops: 294 real flops (differences, reconstruction, 6x6 stiffness, fluxes, gather, shift)
BYTES_PER_NODE = {"c64": 3 * 8 * 2 + 1, "c128": 3 * 16 * 2 + 1}
FLOPS_PER_NODE = 294
# DRAM bytes per node of the two-pass complex128 apply (the four kernels together) at the bench's
# launches (64 block vectors per launch, the two-pass launcher's batch: a step of 16 Bloch vectors x
# 4 blocks x Krylov block 2 runs two such launches per apply; N = 48), from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, cold cache: ncu --metrics
# dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none
# --profile-from-start off -k regex:split_ -c 8 python bench.py --profile kpoint).
SPLIT_F64_DRAM_BYTES_PER_NODE = (36050432 + 900096 + 164037632 + 397710592 + 155104256 + 46386688 +
                                 549513216 + 71348992) / (64 * 27648)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 peak of GB300: measured in the run by the library's FP64 FMA throughput kernel
# (pc_fp64_peak); this nominal figure is used only when that measurement fails.
FP64_NOMINAL_TFLOPS = 1.25
PRECISION_FP64 = ("FP64 operator, inner PCG iterates and inner products, Krylov recurrences and true "
                  "residuals; complex64 Fourier preconditioner inside the FP64 PCG")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if sm:
            sm.sort()
            out["sm_mhz"] = sm[len(sm) // 2]
        out["sm_max_mhz"] = smax
        out["reasons"] = sorted(reasons)
        out["samples"] = len(sm)
        return out


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v, device="cuda"):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, v, device="cuda"):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def kpoint_chunk(step, world, rank, nk, kb=1):
    """Path indices of the Bloch vectors of a timed or warm-up step on one rank: chunk
    `step * world + rank` of kb consecutive points of the nk-point path (cyclic).  Chunks are dealt
    round-robin over the ranks (independent problems, no data exchange; weak scaling)."""
    c = step * world + rank
    return [(c * kb + j) % nk for j in range(kb)]


def cpu_oracle_sample(apply_count_per_kpoint, seconds=15.0):
    """Time the FP64 CPU oracle apply (OpenMP) on block applies of the N = 48 workload,
    and scale by the number of block applies one k-point solve performs."""
    import numpy as np
    from oracle import oracle as O
    from workloads import complex_gaussian, config_cell

    cell = config_cell("fp64")
    pb = O.problem_from_cell(cell, C0=1e9, rho0=1e3)
    threads = os.cpu_count() or 1
    kappa = [0.25, 0.0, 0.0]
    x = complex_gaussian((3, cell.N ** 3 // 4), 7)
    O.apply_block(pb, kappa, 0, x, 0.1, nthreads=threads)  # warm-up (builds and loads the oracle)
    n, t0 = 0, time.perf_counter()
    while True:
        O.apply_block(pb, kappa, n % 4, x, 0.1, nthreads=threads)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds or n >= 2000:
            break
    per_apply = el / n
    return {"value": per_apply * apply_count_per_kpoint, "unit": "s/k-point", "cores": threads, "kind": "oracle",
            "sample": ("%d FP64 oracle block applies (N=48, OpenMP %d threads, %.2f ms each) scaled by the %d "
                       "block applies one k-point solve performs; the oracle's exact eigen-solve (ARPACK + "
                       "SuperLU) takes ~35 min per block on one core and is not sampled" % (n, threads, per_apply * 1e3,
                                                                                 apply_count_per_kpoint)),
            "per_apply_ms": per_apply * 1e3}


def run_reference(args):
    """Reference arm: the CPU oracle, as it stands, on the same config, metric and unit."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import numpy as np
    from oracle import oracle as O
    from workloads import complex_gaussian, config_cell
    cell = config_cell("fp64")
    pb = O.problem_from_cell(cell, C0=1e9, rho0=1e3)
    threads = os.cpu_count() or 1
    x = complex_gaussian((3, cell.N ** 3 // 4), 7)
    # block applies one k-point solve of the GPU arm performs, as that arm measures it on GB300
    # (178 inner solves x ~27 PCG iterations, plus the residual checks); the GPU arm's own
    # cpu_baseline scales by the count it measures itself
    applies = int(os.environ.get("PC_APPLIES_PER_KPOINT", str(APPLIES_PER_KPOINT_MEASURED)))
    reps = 16
    for _ in range(args.warmup):
        O.apply_block(pb, [0.25, 0, 0], 0, x, 0.1, nthreads=threads)
    times, step_s = [], []
    for s in range(args.steps):
        t0 = time.perf_counter()
        for r in range(reps):
            O.apply_block(pb, [0.25, 0, 0], r % 4, x, 0.1, nthreads=threads)
        dt = time.perf_counter() - t0
        step_s.append(dt)
        times.append(dt / reps * applies)
    v = float(np.mean(times))
    # ms_per_step is the measured time of a step (its sample of applies); value is that sample's
    # time per apply times the applies of one k-point solve (see "extrapolation")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s/k-point", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(step_s)) * 1e3,
            "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": 48},
            "cpu_baseline": {"value": v, "unit": "s/k-point", "cores": threads, "kind": "oracle",
                             "sample": "%d FP64 oracle block applies per step at N=48, scaled by %d block applies "
                                       "per k-point solve" % (reps, applies)},
            "extrapolation": {"measured": "time of one FP64 oracle block apply at N=48 (OpenMP, all host cores)",
                              "applies_per_kpoint": applies,
                              "source": "the GPU arm's measured block-apply count per k-point "
                                        "(solver.block_applies_per_kpoint: PCG iterations and residual checks); "
                                        "the oracle's own exact eigen-solve "
                                        "(ARPACK + sparse LU) takes ~35 min per block on one core and is not run"},
            "e2e": {"value": v, "unit": "s/k-point", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def apply_throughput(pc, torch, reps=20):
    """Block apply at N = 160 (R = 0.3, seed 3), complex64 and complex128, one launch per rep:
    all four blocks in one launch with the shift term (the headline figures), the same without
    the shift term, and block 0 alone."""
    from workloads import config_cell
    cell = config_cell("precision")
    N = cell.N
    g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    hbm, src = peaks()
    out = {"workload": "N=160 two-phase cell (R=0.3, seed 3), all four parity blocks in one launch, "
                       "kappa=(0.3,0.1,0.2), shift on", "hbm_peak_gbs": hbm, "peak_source": src}
    try:
        pc.pc_set_k(g, [0.3, 0.1, 0.2])
        nb = N ** 3 // 4
        flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")

        def timed(name, nodes, launch):
            for _ in range(3):
                launch()
            torch.cuda.synchronize()
            ts = []
            for r in range(reps):
                flush.fill_(float(r))  # L2 flush between repetitions (512 MB > 129 MB L2)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                launch()
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) / 1e3)
            t = sorted(ts)[len(ts) // 2]
            gbs = nodes * BYTES_PER_NODE[name] / t / 1e9
            return {"ms": t * 1e3, "gdof_s": 3 * nodes / t / 1e9, "alg_gbs": gbs, "hbm_frac": gbs / hbm,
                    "fp_tflops": nodes * FLOPS_PER_NODE / t / 1e12}

        for name, dt in (("c64", torch.complex64), ("c128", torch.complex128)):
            xs = [torch.randn(3 * nb, dtype=dt, device="cuda") for _ in range(4)]
            ys = [torch.empty_like(x) for x in xs]
            res = timed(name, 4 * nb, lambda: pc.pc_apply_batch(g, [0, 1, 2, 3], xs, ys, [0.5] * 4))
            res["no_shift"] = timed(name, 4 * nb, lambda: pc.pc_apply_batch(g, [0, 1, 2, 3], xs, ys, [0.0] * 4))
            res["block0_alone"] = timed(name, nb, lambda: pc.pc_block_apply(g, 0, xs[0], ys[0], shift=0.5))
            out[name] = res
            del xs, ys
    finally:
        pc.pc_grid_destroy(g)
    return out


def cpu_oracle_apply_rate():
    """The FP64 CPU oracle's full-grid apply on the same N = 160 grid (the DoF of all four blocks),
    with every host thread (best of 3 after a warm-up) and with one thread (one run)."""
    from oracle import oracle as O
    from workloads import complex_gaussian, config_cell
    cell = config_cell("precision")
    pb = O.problem_from_cell(cell, C0=1e9, rho0=1e3)
    x = complex_gaussian((3, cell.N ** 3), 7)
    kappa = [0.3, 0.1, 0.2]
    dof = 3 * cell.N ** 3
    threads = os.cpu_count() or 1
    out = {"workload": "N=160 two-phase cell (R=0.3, seed 3), full-grid FP64 oracle apply, kappa=(0.3,0.1,0.2), "
                       "shift on"}
    O.apply_full(pb, kappa, x, 0.5, nthreads=threads)
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        O.apply_full(pb, kappa, x, 0.5, nthreads=threads)
        ts.append(time.perf_counter() - t0)
    out["threads_%d" % threads] = {"ms": min(ts) * 1e3, "gdof_s": dof / min(ts) / 1e9}
    t0 = time.perf_counter()
    O.apply_full(pb, kappa, x, 0.5, nthreads=1)
    t1 = time.perf_counter() - t0
    out["threads_1"] = {"ms": t1 * 1e3, "gdof_s": dof / t1 / 1e9}
    return out


def profile_run(what):
    import torch
    import paper_2606_03599_gb300 as pc
    from workloads import config_cell
    if what.startswith("kpoint"):
        # one timed step (a lockstep chunk of 16 path points) with the step's options; tuning and
        # one warm-up chunk stay outside the profiled range (ncu --profile-from-start off captures
        # only what runs between profiler start and stop)
        from workloads import sc_path
        cell = config_cell("fp64")
        g = pc.pc_grid_create(cell.N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
        prec = pc.PC_PREC_MIXED if what == "kpoint-mixed" else pc.PC_PREC_FP64
        opt = pc.pc_options_default(tol=TOL, inner_tol=1e-10, precision=prec, autotune=1)
        kpts = sc_path(6)
        pc.pc_eigs_multi(g, kpts[0:16], NEV, opt=opt)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        pc.pc_eigs_multi(g, kpts[15:31], NEV, opt=opt)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    elif what == "precision-mixed":
        cell = config_cell("precision")
        g = pc.pc_grid_create(cell.N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
        opt = pc.pc_options_default(tol=TOL, precision=pc.PC_PREC_MIXED, autotune=1)
        pc.pc_eigs(g, [0.25, 0.0, 0.0], NEV, opt=opt)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        pc.pc_eigs(g, [0.3, 0.1, 0.2], NEV, opt=opt)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    else:
        cell = config_cell("precision")
        N = cell.N
        g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
        pc.pc_set_k(g, [0.3, 0.1, 0.2])
        dt = torch.complex64 if what == "apply-c64" else torch.complex128
        xs = [torch.randn(3 * N ** 3 // 4, dtype=dt, device="cuda") for _ in range(4)]
        ys = [torch.empty_like(x) for x in xs]
        for _ in range(3):
            pc.pc_apply_batch(g, [0, 1, 2, 3], xs, ys, [0.5] * 4)
    torch.cuda.synchronize()
    pc.pc_grid_destroy(g)


def batching_run(args, emit=True, full_space_sample=2):
    """Ragged batch: N in {32, 48, 64, 96, 128} (own seeds, R ~ U[0.2, 0.4]), `--batch-k` Bloch vectors
    each along the SC path, four parity blocks, 16 bands at 1e-8, complex64 apply and inner PCG with
    the FP64 outer loop, autotuned launches, CUDA-graph PCG chunks, pc_eigs_batch worker pool.
    Reported against plain FP64 full-space solves of the same grids on the same GPU (sampled)."""
    import numpy as np
    import torch
    import paper_2606_03599_gb300 as pc
    from workloads import config_cell
    from workloads.kpath import sc_uniform_path
    sizes = [32, 48, 64, 96, 128]
    nk = max(1, args.batch_k)
    ks = sc_uniform_path(nk)
    cells = [config_cell("batch", N=N) for N in sizes]
    grids = [pc.pc_grid_create(c.N, c.C, c.rho, phase=c.phase, a_lat=c.a_lat) for c in cells]
    nev = 16
    opt = pc.pc_options_default(tol=TOL, precision=pc.PC_PREC_MIXED, autotune=1)
    # warm-up: tunes every grid size and builds the solver state once
    pc.pc_eigs_batch(grids, [ks[:1]] * len(grids), nev, opt=opt, workers=args.workers)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    evs, _, status, info = pc.pc_eigs_batch(grids, [ks] * len(grids), nev, opt=opt, workers=args.workers,
                                            raise_on_noconv=False)
    unconverged = [[sizes[gi], int(i)] for gi, s in enumerate(status) for i in np.nonzero(s)[0]]
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    total_k = nk * len(sizes)
    # plain FP64 full space, one Bloch vector at a time, on a sample of the same Bloch vectors
    fopt = pc.pc_options_default(tol=TOL, precision=pc.PC_PREC_FP64, full_space=1)
    sample = [ks[len(ks) // 3], ks[(2 * len(ks)) // 3]][:max(1, full_space_sample)]
    per_grid_full, max_diff = [], 0.0
    for g, ev in zip(grids, evs):
        pc.pc_eigs(g, sample[0], nev, opt=fopt)  # warm-up of the full-space state
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for kk in sample:
            ef, _, _ = pc.pc_eigs(g, kk, nev, opt=fopt)
            i = int(np.argmin(np.abs(ks - kk).sum(axis=1)))
            max_diff = max(max_diff, float(np.max(np.abs(ef - ev[i]) / np.abs(ef))))
        torch.cuda.synchronize()
        per_grid_full.append((time.perf_counter() - t1) / len(sample))
    full_est = nk * sum(per_grid_full)
    for g in grids:
        pc.pc_grid_destroy(g)
    line = {"metric": METRIC, "mode": "batching", "unit": "s/k-point", "dtype": "mixed c64/f64",
            "config": {"workload": "ragged two-phase SC cells N in %s (seeds 10..14, R ~ U[0.2,0.4]), %d Bloch "
                                   "vectors each on the SC path, 4 parity blocks, 16 bands, resid 1e-8" % (sizes, nk),
                       "block_solves": 4 * total_k, "workers": info["workers"], "autotune": True,
                       "cuda_graphs": True},
            "total_s": t_batch, "s_per_kpoint": t_batch / total_k,
            "full_space_fp64_s_per_kpoint_by_N": dict(zip(map(str, sizes), per_grid_full)),
            "full_space_fp64_estimated_total_s": full_est, "speedup_vs_fp64_full_space": full_est / t_batch,
            "max_rel_diff_vs_fp64_full_space_sampled": max_diff,
            "max_true_rel_resid": info["max_rel_resid"], "failed": info["failed"],
            "unconverged_N_and_path_index": unconverged, "pcg_iters": info["pcg_iters"]}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def precision_run(args, emit=True, nk_max=8):
    """N = 160 two-phase cell (R = 0.3, seed 3), Gamma/X/M/R and four midpoints, 20 bands at 1e-8:
    mixed precision s/k-point, and per-band relative error against the FP64 path on the first k-point."""
    import numpy as np
    import torch
    import paper_2606_03599_gb300 as pc
    from workloads import config_cell, sc_eight_points
    cell = config_cell("precision")
    kpts = sc_eight_points()
    g = pc.pc_grid_create(cell.N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    stream = torch.cuda.Stream()
    om = pc.pc_options_default(tol=TOL, precision=pc.PC_PREC_MIXED, autotune=1)
    om.stream = stream.cuda_stream
    pc.pc_set_k(g, kpts[0])  # launch shapes tuned before the timed solves
    for dt in (pc.PC_C64, pc.PC_C128):
        pc.pc_autotune(g, dt, 0, 4 * om.block_size, stream.cuda_stream)
    nk = max(1, min(args.steps, len(kpts), nk_max))
    res = []
    for i in range(nk):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ev, bl, info = pc.pc_eigs(g, kpts[i], NEV, opt=om)
        e1.record(stream)
        e1.synchronize()
        res.append((e0.elapsed_time(e1) / 1e3, ev, info))
    o64 = pc.pc_options_default(tol=TOL, precision=pc.PC_PREC_FP64, autotune=1)
    o64.stream = stream.cuda_stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ev64, _, info64 = pc.pc_eigs(g, kpts[0], NEV, opt=o64)
    e1.record(stream)
    e1.synchronize()
    t64 = e0.elapsed_time(e1) / 1e3
    per_band = (np.abs(res[0][1] - ev64) / ev64).tolist()
    pc.pc_grid_destroy(g)
    line = {"metric": METRIC, "mode": "precision", "unit": "s/k-point", "dtype": "mixed c64/f64",
            "config": {"workload": "two-phase SC cell N=160 (R=0.3, seed 3), 20 bands, resid 1e-8",
                       "k_points": nk},
            "mixed_s_per_kpoint": float(np.mean([r[0] for r in res])),
            "fp64_s_per_kpoint_first_k": t64,
            "per_band_rel_err_vs_fp64_first_k": per_band,
            "max_true_rel_resid_mixed": max(r[2]["max_rel_resid"] for r in res),
            "pcg_iters_per_kpoint_mixed": float(np.mean([r[2]["pcg_iters"] for r in res])),
            "pcg_iters_fp64_first_k": info64["pcg_iters"]}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def paper_run(args):
    """The paper's own FCC workload (Sec. 7.1): low-quartz matrix, silicon sphere of radius
    a0/4, sub-pixel inclusion fractions, FCC primitive cell, N^3 grid (--paper-n, 60 in the
    paper), 40 bands, Bloch vectors spread over the 91-point path Gamma-X-W-K-Gamma-L-U-W-L-K
    (--paper-k of them), in plain FP64 and in mixed precision.  Seconds per Bloch vector next
    to the wall times the paper prints for the same grid (context: other hardware, MATLAB,
    eigs/PCG tolerance 1e-12 against the true-residual bound here)."""
    import numpy as np
    import torch
    import paper_2606_03599_gb300 as pc
    from workloads import fcc_kappa, fcc_lattice, fcc_path, fcc_quartz_silicon_cell
    from workloads.materials import FCC_A0
    N, nev = args.paper_n, 40
    cell = fcc_quartz_silicon_cell(N)
    A = fcc_lattice()
    path = [fcc_kappa(k, A, FCC_A0) for k in fcc_path(10)]
    nk = max(1, min(args.paper_k, len(path)))
    sel = np.unique(np.linspace(0, len(path) - 1, nk).round().astype(int))
    g = pc.pc_grid_create(N, cell.C, cell.rho, theta=cell.theta, a_lat=cell.a_lat)
    stream = torch.cuda.Stream()
    modes = {}
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    try:
        kb = max(1, min(getattr(args, "kbatch", 8), 32, pc.pc_eigs_multi_max(g)))
        for name, prec in (("fp64", pc.PC_PREC_FP64), ("mixed", pc.PC_PREC_MIXED)):
            opt = pc.pc_options_default(tol=TOL, precision=prec, autotune=1)
            opt.stream = stream.cuda_stream
            pc.pc_eigs(g, path[sel[0]], nev, opt=opt)  # untimed: tunes this mode's launches
            ts, resid, iters = [], 0.0, 0
            for i in sel:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ev, _, info = pc.pc_eigs(g, path[i], nev, opt=opt)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1) / 1e3)
                resid = max(resid, info["max_rel_resid"])
                iters += info["pcg_iters"]
            one = {"s_per_kpoint": float(np.mean(ts)), "max_true_rel_resid": resid,
                   "pcg_iters_per_kpoint": iters / len(sel)}
            # the same Bloch vectors in lockstep chunks of kb (pc_eigs_multi)
            chunks = [sel[c:c + kb] for c in range(0, len(sel), kb)]
            if kb > 1:
                pc.pc_eigs_multi(g, np.array([path[i] for i in chunks[0]]), nev, opt=opt)  # untimed
            tl, resid_l = 0.0, 0.0
            for ch in chunks:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _, _, infs = pc.pc_eigs_multi(g, np.array([path[i] for i in ch]), nev, opt=opt)
                e1.record(stream)
                e1.synchronize()
                tl += e0.elapsed_time(e1) / 1e3
                resid_l = max(resid_l, max(x["max_rel_resid"] for x in infs))
            modes[name] = {"s_per_kpoint": tl / len(sel), "max_true_rel_resid": resid_l,
                           "lockstep_k_points_per_chunk": kb, "one_at_a_time": one}
    finally:
        clk = clocks.stop()
        pc.pc_grid_destroy(g)
    line = {"metric": "seconds per k-point, the paper's FCC quartz/silicon workload", "mode": "paper",
            "value": modes["fp64"]["s_per_kpoint"], "unit": "s/k-point", "n_gpus": 1, "higher_is_better": False,
            "dtype": "f64", "data": "synthetic from the paper's constants and geometry",
            "config": {"workload": "FCC quartz/silicon cell, sphere R=a0/4, sub-pixel theta (8^3 samples), "
                                   "N=%d, 40 non-zero bands, %d of the 91 path points" % (N, len(sel)),
                       "N": N, "bands": nev, "tol": TOL, "blocks": 4},
            "modes": modes,
            "clocks": clk,
            "paper_context": {"grid": 60, "bands": 40, "k_points": 91, "tol": "eigs 1e-12, PCG 1e-12",
                              "cpu_128_cores_full_space_s_per_kpoint": 613.7,
                              "v100_full_space_s_per_kpoint": 43.0,
                              "v100x4_blocks_s_per_kpoint": 18.8}}
    print(json.dumps(line), flush=True)


def differentiation_run(args, emit=True, nk=10):
    """N = 64 two-phase cell (R = 0.35, seed 4) entered as a nodewise material (the (N^3, 21)
    stiffness and (N^3,) density tensors): gradients of the lowest 12 eigenvalues at `nk` Bloch
    vectors of the SC path and of the width of the gap between bands 6 and 7 over them, through the
    torch.autograd functions whose inputs are those tensors (forward: the GPU solve of the nodewise
    grid, all Bloch vectors in lockstep; backward: the adjoint kernel).  Reported: seconds per Bloch
    vector for solve + eigenvectors + adjoint (lockstep, and one Bloch vector at a time, with the
    difference of the two summed gradients), the gap gradient's time, and central differences with a relative step of
    1e-6 along `--fd-dirs` seeded random directions in (C, rho) against the autograd gradient of
    sum(lambda) at one Bloch vector."""
    import numpy as np
    import torch
    from paper_2606_03599_gb300 import autodiff as ad
    from workloads import config_cell
    from workloads.kpath import sc_uniform_path
    import paper_2606_03599_gb300 as pc
    cell = config_cell("diff")
    N = cell.N
    nev = 12
    ks = sc_uniform_path(nk)
    C21, rho = ad.two_phase_nodewise(cell)
    opt = pc.pc_options_default(tol=TOL, autotune=1)
    Ct = torch.tensor(C21, dtype=torch.float64, requires_grad=True)
    rt = torch.tensor(rho, dtype=torch.float64, requires_grad=True)
    ad.band_eigenvalues_nodewise(Ct, rt, N, ks[0], nev, opt=opt).sum().backward()  # untimed: tuning
    Ct.grad = None
    rt.grad = None
    torch.cuda.synchronize()
    kfd = min(3, len(ks) - 1)
    t0 = time.perf_counter()
    grad_fd_k = None
    sum_gc, sum_gr = 0.0, 0.0
    for i, k in enumerate(ks):
        lam = ad.band_eigenvalues_nodewise(Ct, rt, N, k, nev, opt=opt)
        lam.sum().backward()
        if i == kfd:
            grad_fd_k = (Ct.grad.numpy().copy(), rt.grad.numpy().copy(), lam.detach().numpy())
        sum_gc = sum_gc + Ct.grad.numpy()
        sum_gr = sum_gr + rt.grad.numpy()
        Ct.grad = None
        rt.grad = None
    torch.cuda.synchronize()
    t_grad_one = (time.perf_counter() - t0) / len(ks)
    # the same gradients with every Bloch vector solved in lockstep (one forward, summed adjoints)
    Cl = torch.tensor(C21, dtype=torch.float64, requires_grad=True)
    rl = torch.tensor(rho, dtype=torch.float64, requires_grad=True)
    ad.band_structure_nodewise(Cl, rl, N, ks[:2], nev, opt=opt).sum().backward()  # untimed: state
    Cl.grad = None
    rl.grad = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ad.band_structure_nodewise(Cl, rl, N, ks, nev, opt=opt).sum().backward()
    torch.cuda.synchronize()
    t_grad = (time.perf_counter() - t0) / len(ks)
    lock_diff = max(float(np.abs(Cl.grad.numpy() - sum_gc).max() / np.abs(sum_gc).max()),
                    float(np.abs(rl.grad.numpy() - sum_gr).max() / np.abs(sum_gr).max()))
    Cg = torch.tensor(C21, dtype=torch.float64, requires_grad=True)
    rg = torch.tensor(rho, dtype=torch.float64, requires_grad=True)
    t0 = time.perf_counter()
    gap = ad.band_gap_nodewise(Cg, rg, N, ks, 5, opt=opt)
    gap.backward()
    torch.cuda.synchronize()
    t_gap = time.perf_counter() - t0
    gc, gr, lam0 = grad_fd_k
    h = 1e-6
    sC, sr = float(np.abs(C21[:, [0, 6, 11]]).mean()), float(rho.mean())
    rng = np.random.default_rng(2024)
    errs = []
    for _ in range(max(1, args.fd_dirs)):
        dCd = sC * rng.standard_normal(C21.shape)
        drd = sr * rng.standard_normal(rho.shape)
        vals = []
        for sgn in (1.0, -1.0):
            ev, _ = ad._solve_nodewise(C21 + sgn * h * dCd, rho + sgn * h * drd, N, ks[kfd], nev, None, opt)
            vals.append(float(np.sum(ev)))
        fd = (vals[0] - vals[1]) / (2 * h)
        an = float(np.sum(gc * dCd) + np.sum(gr * drd))
        errs.append(abs(fd - an) / abs(fd))
    line = {"metric": METRIC, "mode": "differentiation", "unit": "s/k-point", "dtype": "f64",
            "config": {"workload": "two-phase SC cell N=64 (R=0.35, seed 4) as a nodewise material "
                                   "((N^3, 21) stiffness, (N^3,) density), %d Bloch vectors on the SC path, "
                                   "12 bands, gap between bands 6 and 7, resid 1e-8" % len(ks),
                       "k_points": len(ks), "fd_directions": max(1, args.fd_dirs), "fd_relative_step": h,
                       "fd_direction_scale": {"C": sC, "rho": sr}},
            "grad_s_per_kpoint": t_grad, "grad_s_per_kpoint_one_at_a_time": t_grad_one,
            "lockstep_grad_rel_diff_vs_one_at_a_time": lock_diff,
            "gap_hz": float(gap.detach()), "gap_grad_s": t_gap,
            "gap_grad_norm": float(np.sqrt(float((Cg.grad ** 2).sum()) + float((rg.grad ** 2).sum()))),
            "fd_rel_err_sum_lambda": errs, "fd_rel_err_max": max(errs)}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--kbatch", type=int, default=16,
                    help="Bloch vectors per step, solved together in lockstep (1 = one pc_eigs per step)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the reduced precision / batching / differentiation sub-results of the default line")
    ap.add_argument("--precision", action="store_true",
                    help="run the N=160 precision workload (8 k-points, 20 bands, mixed precision) instead")
    ap.add_argument("--batching", action="store_true",
                    help="run the ragged batching workload (N in {32..128}, --batch-k Bloch vectors each) instead")
    ap.add_argument("--batch-k", type=int, default=64, help="Bloch vectors per grid of --batching")
    ap.add_argument("--differentiation", action="store_true",
                    help="run the N=64 gradient workload (10 Bloch vectors, 12 bands, gap 6-7) instead")
    ap.add_argument("--fd-dirs", type=int, default=50, help="finite-difference directions of --differentiation")
    ap.add_argument("--workers", type=int, default=4, help="host worker threads of --batching")
    ap.add_argument("--paper", action="store_true",
                    help="run the paper's own FCC quartz/silicon workload (40 bands) instead")
    ap.add_argument("--paper-n", type=int, default=60, help="grid size of --paper (the paper's: 60)")
    ap.add_argument("--paper-k", type=int, default=16, help="Bloch vectors of the 91-point path timed by --paper")
    ap.add_argument("--profile", default=None,
                    choices=["kpoint", "kpoint-mixed", "precision-mixed", "apply-c64", "apply-c128"],
                    help="profiling aid for ncu: run only one lockstep chunk of 16 Bloch vectors of the "
                         "workload (after an untimed one), one mixed-precision solve of the N=160 precision "
                         "cell (after an untimed one), or one N=160 four-block apply (after two untimed "
                         "ones), and print nothing else")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile:
        profile_run(args.profile)
        return
    if args.precision:
        precision_run(args)
        return
    if args.batching:
        batching_run(args)
        return
    if args.differentiation:
        differentiation_run(args)
        return
    if args.paper:
        paper_run(args)
        return
    args.warmup = max(3, args.warmup)

    import numpy as np
    import torch
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2606_03599_gb300 as pc
    from workloads import config_cell, sc_path

    cell = config_cell("fp64")
    kpts = sc_path(6)
    KB = max(1, min(args.kbatch, 32))
    stream = torch.cuda.Stream()
    opt = pc.pc_options_default(tol=TOL, inner_tol=1e-10, precision=pc.PC_PREC_FP64, autotune=1)
    opt.stream = stream.cuda_stream
    g = pc.pc_grid_create(cell.N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")

    def kchunk(step):
        return np.array([kpts[i] for i in kpoint_chunk(step, world, rank, len(kpts), KB)])

    def solve(gr, ks, o):
        if KB == 1:
            ev, _, inf = pc.pc_eigs(gr, ks[0], NEV, opt=o)
            return ev[None, :], [inf]
        ev, _, infs = pc.pc_eigs_multi(gr, ks, NEV, opt=o)
        return ev, infs

    # warm-up (untimed)
    for w in range(args.warmup):
        solve(g, kchunk(w), opt)
    torch.cuda.synchronize()

    # timed region
    clocks = ClockSampler(local)
    clocks.start()
    pc.pc_stats_reset()
    pc.pc_stats_timing(1)
    barrier(world)
    torch.cuda.synchronize()
    step_ms, infos, residuals, evals, kdone = [], [], [], [], []
    for s in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(s))  # L2 flush between timed steps (not timed)
        ks = kchunk(args.warmup + s)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ev, infs = solve(g, ks, opt)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        infos.append(infs[0])
        residuals.append(max(i["max_rel_resid"] for i in infs))
        evals.append(ev)
        kdone.append(ks)
    torch.cuda.synchronize()
    barrier(world)
    st = pc.pc_stats_get()
    pc.pc_stats_timing(0)
    clk = clocks.stop()
    local_time = sum(step_ms) / 1e3
    t_max = max_over_ranks(world, local_time)
    kpts_total = sum_over_ranks(world, float(args.steps * KB))
    value = t_max / kpts_total

    # dominant kernel: FP64 stencil apply, device time from events on its launch stream; its
    # roofline denominator is the FP64 FMA rate measured here (outside the timed region)
    try:
        fp64_peak, fma_rate = pc.pc_fp64_peak(0.5)
        peak_src = "measured: pc_fp64_peak FP64 FMA throughput kernel on this GPU (2 flops per FMA)"
    except Exception:
        fp64_peak, fma_rate = FP64_NOMINAL_TFLOPS, None
        peak_src = "nominal FP64 dense rate of GB300 (measurement failed)"
    n_app = st["apply_timed"][1]
    app_ms = st["apply_ms"][1] / max(1, n_app)
    # nodes of the items that ran (a launch's items of converged systems return at once)
    nodes_per_launch = st["apply_nodes"][1] / max(1, n_app)
    skipped_frac = 1.0 - st["apply_nodes"][1] / max(1.0, st["apply_nodes_launched"][1])
    achieved_tflops = nodes_per_launch * FLOPS_PER_NODE / (app_ms / 1e3) / 1e12
    kind = pc.pc_tuned_config(g, pc.PC_C128, 0, 4 * opt.block_size * KB)[0]
    kname = {0: "apply_kernel<double>", 1: "apply_tma_kernel<double>", 2: "apply_row_kernel",
             3: "split_fill_x + split_flux + split_fill_f + split_gather (two-pass FP64)"}[kind]
    traffic = SPLIT_F64_DRAM_BYTES_PER_NODE * nodes_per_launch if (kind == 3 and KB >= 8) else None
    roofline = {"kernel": kname + " (block stencil, FP64, autotuned launch)", "bound": "alu",
                "achieved": achieved_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved_tflops / fp64_peak, "traffic": traffic,
                "traffic_note": "DRAM bytes per timed apply (two 64-vector launches of the four kernels), ncu "
                                "cold-cache capture per node scaled by the nodes per timed apply"
                if traffic is not None else None,
                "launches": n_app, "avg_launch_us": app_ms * 1e3, "nodes_per_launch": nodes_per_launch,
                "skipped_item_frac": skipped_frac,
                "flops_per_node": FLOPS_PER_NODE, "peak_source": peak_src,
                "fp64_fma_per_s": fma_rate, "peak_nominal_tflops": FP64_NOMINAL_TFLOPS}

    # end-to-end through the C ABI from host buffers: material upload, solve, eigenvalues back
    e2e = None
    if rank == 0 or world > 1:
        phase_pinned = torch.from_numpy(cell.phase).pin_memory()
        e2e_ms = []
        for s in range(min(args.steps, 2)):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g2 = pc.pc_grid_create(cell.N, cell.C, cell.rho, phase=phase_pinned.numpy(), a_lat=cell.a_lat)
            solve(g2, kchunk(s), opt)
            pc.pc_grid_destroy(g2)
            e1.record(stream)
            e1.synchronize()
            e2e_ms.append(e0.elapsed_time(e1))
        n = cell.N ** 3
        e2e = {"value": float(np.mean(e2e_ms)) / 1e3 / KB, "unit": "s/k-point", "h2d_bytes_per_step": 2 * n,
               "d2h_bytes_per_step": KB * NEV * 8, "steps": len(e2e_ms), "k_points_per_step": KB}

    # comparisons on this GPU over the Bloch vectors of the first timed steps: mixed precision
    # (complex64 inner PCG + FP64 refinement) and the FP64-preconditioner variant, both in lockstep
    # chunks as the main leg; the blocked FP64 solve and the plain FP64 full-space solve one Bloch
    # vector at a time (pc_eigs)
    compare = None
    if rank == 0:
        compare = {}
        nc = max(1, min(args.steps, 24 // KB))  # about 24 Bloch vectors
        cks = [kchunk(args.warmup + s) for s in range(nc)]
        legs = (("mixed", pc.pc_options_default(tol=TOL, precision=pc.PC_PREC_MIXED, autotune=1), True),
                ("fp64_preconditioner", pc.pc_options_default(tol=TOL, precond_fp32=0, autotune=1), True),
                # Krylov block width 1 (not the default: a one-vector Krylov space can miss a copy of
                # an exactly degenerate eigenvalue; reported with its difference to the main leg)
                ("fp64_block_width_1", pc.pc_options_default(tol=TOL, block_size=1, autotune=1), True),
                ("mixed_block_width_1", pc.pc_options_default(tol=TOL, precision=pc.PC_PREC_MIXED, block_size=1,
                                                              autotune=1), True),
                ("one_at_a_time_fp64", pc.pc_options_default(tol=TOL, autotune=1), False),
                ("full_space_fp64", pc.pc_options_default(tol=TOL, full_space=1, autotune=1), False))
        for name, o2, lockstep in legs:
            o2.stream = stream.cuda_stream
            pc.pc_eigs(g, cks[0][0], NEV, opt=o2)  # untimed: tunes this leg's launches, builds its state
            if lockstep and KB > 1:
                pc.pc_eigs_multi(g, cks[0], NEV, opt=o2)
            ms, err, nk = [], 0.0, 0
            for s in range(nc):
                for j in (range(1) if lockstep else range(KB)):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    if lockstep:
                        ev2, _ = solve(g, cks[s], o2)
                    else:
                        e_, _, _ = pc.pc_eigs(g, cks[s][j], NEV, opt=o2)
                        ev2 = e_[None, :]
                    e1.record(stream)
                    e1.synchronize()
                    ms.append(e0.elapsed_time(e1))
                    ref = evals[s] if lockstep else evals[s][j:j + 1]
                    err = max(err, float(np.max(np.abs(ev2 - ref) / ref)))
                    nk += ev2.shape[0]
            compare[name] = {"s_per_kpoint": float(np.sum(ms)) / 1e3 / nk, "k_points": nk,
                             "lockstep": bool(lockstep and KB > 1), "same_k_points_as_main_leg": True,
                             "max_rel_diff_vs_main_leg": err}
        compare["main_leg_s_per_kpoint"] = value
        compare["lockstep_speedup_vs_one_at_a_time"] = compare["one_at_a_time_fp64"]["s_per_kpoint"] / value
        compare["blocked_speedup_vs_full_space"] = compare["full_space_fp64"]["s_per_kpoint"] / value
        compare["mixed_vs_fp64"] = compare["mixed"]["s_per_kpoint"] / value
        compare["mixed_speedup_vs_fp64_full_space"] = (compare["full_space_fp64"]["s_per_kpoint"] /
                                                        compare["mixed"]["s_per_kpoint"])

    apply = apply_throughput(pc, torch) if rank == 0 else None
    pc.pc_grid_destroy(g)

    # reduced runs of the precision, batching and differentiation workloads (counts in each config)
    forms = None
    if rank == 0 and not args.no_forms:
        import copy
        forms = {}
        try:
            forms["precision"] = precision_run(args, emit=False, nk_max=2)
        except Exception as e:  # reported, never fatal for the headline
            forms["precision"] = {"error": str(e)}
        try:
            a2 = copy.copy(args)
            a2.batch_k = 4
            forms["batching"] = batching_run(a2, emit=False, full_space_sample=1)
        except Exception as e:
            forms["batching"] = {"error": str(e)}
        try:
            a3 = copy.copy(args)
            a3.fd_dirs = 4
            forms["differentiation"] = differentiation_run(a3, emit=False, nk=2)
        except Exception as e:
            forms["differentiation"] = {"error": str(e)}

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    # block applies per k-point of the timed steps: nodes of the FP64 apply items that ran, in units
    # of one parity block (items of systems that had converged are skipped inside a launch and not
    # counted); the PCG iterations plus the true-residual checks
    pcg_total = sum(i["pcg_iters"] for i in infos)
    applies_per_k = int(round(st["apply_nodes"][1] / (cell.N ** 3 / 4) / (args.steps * KB)))
    cpu = None if args.no_cpu else cpu_oracle_sample(applies_per_k)
    if cpu is not None:
        cpu["apply_n160"] = cpu_oracle_apply_rate()
    line = {
        "metric": METRIC, "value": value, "unit": "s/k-point", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": cell.N, "bands": NEV, "tol": TOL, "blocks": 4,
                   "k_points_per_step": KB, "k_points_per_rank": args.steps * KB, "precision": PRECISION_FP64,
                   "l2": "512 MB buffer written between timed steps (L2 = 129 MB)"},
        "roofline": roofline,
        "apply": apply,
        "compare_same_gpu": compare,
        "forms": forms,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": st["launches"],
        "clocks": clk,
        "solver": {"pcg_iters_per_kpoint": pcg_total / (args.steps * KB),
                   "max_pcg_iters": max(i["max_pcg_iters"] for i in infos),
                   "inner_solves_per_kpoint": sum(i["inner_solves"] for i in infos) / (args.steps * KB),
                   "block_applies_per_kpoint": applies_per_k,
                   "max_true_rel_resid": max(residuals),
                   "step_ms": step_ms},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
