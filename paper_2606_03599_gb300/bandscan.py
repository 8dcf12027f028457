"""Band-structure scan over a list of Bloch vectors with a resumable JSON-lines record.

A band scan solves the pencil at every Bloch vector of a path (the paper's Sec. 7 scans 91
points of the FCC path; the synthetic workloads use the 31-point simple-cubic path).  With a
record file, the scan writes one JSON line per finished Bloch vector, behind a header line
that fingerprints the scan (grid size, band count, the Bloch vectors, the shift, the solver
options).  Running the same scan again with the same file skips every Bloch vector already
recorded, so an interrupted scan resumes where it stopped; a final line cut short by the
interruption is discarded and its Bloch vector solved again.  A file written by a different
scan is refused rather than mixed in.

Record line: {"k": index, "kappa": [3], "lambda": [nev] (rad^2/s^2), "f_hz": [nev]
(f = sqrt(lambda) / (2 pi)), "block": [nev] (source parity block, -1 for the full space),
"info": {...solver statistics...}}.
"""

from __future__ import annotations

import hashlib
import json
import math
import os

import numpy as np

FORMAT = "pcband-scan-1"


def _fingerprint(N, kappas, nev, sigma, opt_fields):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(kappas, dtype=np.float64).tobytes())
    return {"format": FORMAT, "N": int(N), "nk": int(len(kappas)), "nev": int(nev),
            "sigma": None if sigma is None or math.isnan(sigma) else float(sigma),
            "kappas_sha256": h.hexdigest(), "options": opt_fields}


def _options_fields(opt):
    if opt is None:
        return None
    out = {}
    for name, _ in getattr(opt, "_fields_", []):
        if name == "stream":
            continue
        v = getattr(opt, name)
        out[name] = v if isinstance(v, (int, float)) else str(v)
    return out


def _read_records(path, header):
    """Records already in `path` for the scan `header`; drops a final line cut short."""
    with open(path, "rb") as f:
        raw = f.read()
    lines = raw.split(b"\n")
    complete = lines[:-1]  # text after the last newline is an unfinished write
    keep_bytes = len(raw) - len(lines[-1])
    if not complete:
        if raw and not raw.startswith(b'{"scan"'):
            raise ValueError("%s is not a scan record" % path)
        return {}, 0  # empty, or only an unfinished header: start over
    try:
        head = json.loads(complete[0])
    except json.JSONDecodeError as e:
        raise ValueError("%s: unreadable header line" % path) from e
    if head.get("scan") != header:
        raise ValueError("%s was written by a different scan (grid, Bloch vectors, bands, shift or options)"
                         % path)
    records = {}
    for i, line in enumerate(complete[1:], start=2):
        try:
            rec = json.loads(line)
        except json.JSONDecodeError as e:
            raise ValueError("%s: line %d is not valid JSON" % (path, i)) from e
        records[int(rec["k"])] = rec
    return records, keep_bytes


def scan(grid, N, kappas, nev, path=None, opt=None, sigma=float("nan"), solve=None):
    """Solve every Bloch vector of `kappas` ([nk][3], reduced coordinates) on `grid` (a handle of
    an N^3 grid) for its `nev` lowest non-zero eigenvalues.

    path:  optional JSON-lines record (created, or resumed when it holds this scan).
    opt:   pc_options for every solve (None: library defaults); sigma: shift (NaN: default).
    solve: the eigen-solve, pc_eigs by default (same signature; a stand-in can be passed).
    Returns (lambda [nk][nev] rad^2/s^2, f_hz [nk][nev], block [nk][nev], infos [nk]).
    """
    if solve is None:
        from ._lib import pc_eigs as solve
    kappas = np.asarray(kappas, dtype=np.float64).reshape(-1, 3)
    nk = kappas.shape[0]
    header = _fingerprint(N, kappas, nev, sigma, _options_fields(opt))
    records = {}
    out = None
    if path is not None:
        if os.path.exists(path) and os.path.getsize(path) > 0:
            records, keep = _read_records(path, header)
            if keep == 0:
                out = open(path, "w")
                out.write(json.dumps({"scan": header}) + "\n")
            else:
                out = open(path, "r+")
                out.truncate(keep)
                out.seek(keep)
        else:
            out = open(path, "w")
            out.write(json.dumps({"scan": header}) + "\n")
        out.flush()
        os.fsync(out.fileno())
    lam = np.zeros((nk, nev))
    blk = np.zeros((nk, nev), dtype=np.int64)
    infos = [None] * nk
    try:
        for k in range(nk):
            rec = records.get(k)
            if rec is None:
                ev, bo, info = solve(grid, kappas[k], nev, sigma=sigma, opt=opt)
                rec = {"k": k, "kappa": [float(v) for v in kappas[k]],
                       "lambda": [float(v) for v in ev],
                       "f_hz": [math.sqrt(max(float(v), 0.0)) / (2.0 * math.pi) for v in ev],
                       "block": [int(b) for b in bo],
                       "info": {key: (val if isinstance(val, (int, float)) else str(val))
                                for key, val in dict(info).items()}}
                if out is not None:
                    out.write(json.dumps(rec) + "\n")
                    out.flush()
                    os.fsync(out.fileno())
            lam[k] = rec["lambda"]
            blk[k] = rec["block"]
            infos[k] = rec["info"]
    finally:
        if out is not None:
            out.close()
    return lam, np.sqrt(np.maximum(lam, 0.0)) / (2.0 * np.pi), blk, infos
