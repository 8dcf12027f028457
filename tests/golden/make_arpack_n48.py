"""Write the lowest non-zero eigenvalues of the N = 48 two-phase band cell, per parity block,
computed by the oracle alone (ARPACK shift-invert with an exact sparse LU, the eigen oracle
that the CPU tests pin to dense LAPACK).

Cell: simple cubic a = 1 m, N = 48, inclusion sphere R = 0.35, seed 2 (the FP64 band
workload).  Bloch vectors (reduced): Gamma (0,0,0), X (1/2,0,0) and the generic
(0.3,0.1,0.2).  Per block the lowest ``--per-block`` non-zero eigenvalues (Gamma's
zero-derivative modes projected out exactly, Sec. 6.2); values are lambda = omega^2 in SI.

The four blocks of one Bloch vector are independent problems (Theorem 4.1), so each
(Bloch vector, block) pair is one job; ``--jobs`` runs them in parallel processes.  Each job
writes its own part file, and the merge step collects them into ``arpack_n48.json``.

    python tests/golden/make_arpack_n48.py --jobs 6        # all 12 parts, then the merge
    python tests/golden/make_arpack_n48.py --part 2 1      # Bloch vector 2, block 1 only
    python tests/golden/make_arpack_n48.py --merge         # collect finished parts

Units inside the oracle: C / 1 GPa, rho / (1000 kg/m^3), lengths / 1 m; the eigenvalues
scale back to SI by 1e9 / 1e3.  The shift is sigma = -0.3 max|C| / max rho in those
units (any shift below the spectrum gives the same eigenvalues).
"""

from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

KAPPAS = [("Gamma", [0.0, 0.0, 0.0]), ("X", [0.5, 0.0, 0.0]), ("generic", [0.3, 0.1, 0.2])]
OUT = os.path.join(HERE, "arpack_n48.json")
PART_DIR = os.path.join(HERE, "arpack_n48_parts")
C0, RHO0, L = 1e9, 1e3, 1.0


def _problem():
    from oracle import oracle as O
    from workloads import config_cell
    cell = config_cell("fp64")
    return cell, O.problem_from_cell(cell, C0=C0, rho0=RHO0, L=L)


def _sigma(pb):
    return -0.3 * float(np.abs(pb.C).max()) / float(pb.rho.max())


def run_part(ki: int, b: int, per_block: int) -> str:
    from oracle import oracle as O
    cell, pb = _problem()
    name, kappa = KAPPAS[ki]
    t0 = time.time()
    lam = O.eigs_oracle(pb, kappa, per_block, sigma=_sigma(pb), b=b, tol=1e-13)
    lam = np.sort(lam) * (C0 / (RHO0 * L * L))
    os.makedirs(PART_DIR, exist_ok=True)
    path = os.path.join(PART_DIR, "k%d_b%d.json" % (ki, b))
    with open(path, "w") as f:
        json.dump({"kappa_name": name, "kappa": kappa, "block": b, "per_block": per_block,
                   "eigenvalues_si": [float(v) for v in lam], "seconds": time.time() - t0}, f)
    return path


def _run_part_star(a):
    return run_part(*a)


def merge(nev: int) -> None:
    _cell, pb = _problem()
    out = {
        "what": "lowest non-zero eigenvalues lambda = omega^2 (rad^2/s^2) of the N = 48 two-phase "
                "cell (R = 0.35, seed 2, simple cubic a = 1 m), per parity block and merged",
        "computed_by": "oracle.eigs_oracle (scipy ARPACK shift-invert, exact sparse LU, tol 1e-13)",
        "command": "python tests/golden/make_arpack_n48.py --jobs 6",
        "citation": "Theorem 4.1 and Cor. 4.2 (block spectra, merged); Sec. 6.2 (Gamma zero modes "
                    "projected out)",
        "sigma_oracle_units": _sigma(pb),
        "nev_merged": nev,
        "points": [],
    }
    for ki, (name, kappa) in enumerate(KAPPAS):
        blocks = []
        for b in range(4):
            with open(os.path.join(PART_DIR, "k%d_b%d.json" % (ki, b))) as f:
                blocks.append(json.load(f))
        parts = [np.array(p["eigenvalues_si"]) for p in blocks]
        union = np.sort(np.concatenate(parts))[:nev]
        complete = all(p.max() >= union[-1] for p in parts)
        out["points"].append({"name": name, "kappa": kappa,
                              "blocks": [p["eigenvalues_si"] for p in blocks],
                              "merged": [float(v) for v in union],
                              "complete": bool(complete),
                              "seconds": [p["seconds"] for p in blocks]})
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--part", nargs=2, type=int, metavar=("KAPPA_INDEX", "BLOCK"))
    ap.add_argument("--merge", action="store_true")
    ap.add_argument("--jobs", type=int, default=4)
    ap.add_argument("--per-block", type=int, default=12)
    ap.add_argument("--nev", type=int, default=20)
    a = ap.parse_args()
    if a.part:
        print(run_part(a.part[0], a.part[1], a.per_block))
        return
    if not a.merge:
        todo = [(ki, b, a.per_block) for ki in range(len(KAPPAS)) for b in range(4)
                if not os.path.exists(os.path.join(PART_DIR, "k%d_b%d.json" % (ki, b)))]
        with mp.get_context("spawn").Pool(a.jobs) as pool:
            for p in pool.imap_unordered(_run_part_star, todo):
                print("done", p, flush=True)
    merge(a.nev)


if __name__ == "__main__":
    main()
