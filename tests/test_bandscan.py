"""Band scan with a resumable record (host logic; the eigen-solve is a stand-in here, so
these tests need no GPU).  Checks that an interrupted scan resumes with only the missing
Bloch vectors solved and the same results as an uninterrupted one, that a final line cut
short is recomputed, and that a record of a different scan is refused untouched."""

import json
import math

import numpy as np
import pytest

from paper_2606_03599_gb300 import bandscan
from workloads.kpath import sc_path


class StandIn:
    """Deterministic stand-in for pc_eigs: eigenvalues depend on kappa only."""

    def __init__(self, fail_at=None):
        self.calls = []
        self.fail_at = fail_at

    def __call__(self, grid, kappa, nev, sigma=float("nan"), opt=None):
        self.calls.append([float(v) for v in kappa])
        if self.fail_at is not None and len(self.calls) == self.fail_at:
            raise RuntimeError("interrupted")
        base = 1.0 + float(np.sum(np.asarray(kappa) ** 2))
        return (base * 1e8 * np.arange(1, nev + 1, dtype=np.float64), np.arange(nev) % 4,
                {"pcg_iters": 10, "max_rel_resid": 1e-9})


def _lines(path):
    with open(path) as f:
        return [json.loads(line) for line in f]


def test_scan_without_record():
    ks = sc_path(2)
    lam, f, blk, infos = bandscan.scan(None, 8, ks, 5, solve=StandIn())
    assert lam.shape == (len(ks), 5) and blk.shape == (len(ks), 5)
    assert np.allclose(f, np.sqrt(lam) / (2 * math.pi), rtol=1e-15)
    assert infos[0]["pcg_iters"] == 10


def test_interrupted_scan_resumes_with_the_missing_points_only(tmp_path):
    ks = sc_path(2)
    path = str(tmp_path / "scan.jsonl")
    ref = bandscan.scan(None, 8, ks, 5, solve=StandIn())
    with pytest.raises(RuntimeError):
        bandscan.scan(None, 8, ks, 5, path=path, solve=StandIn(fail_at=4))
    lines = _lines(path)
    assert "scan" in lines[0] and [r["k"] for r in lines[1:]] == [0, 1, 2]
    s = StandIn()
    got = bandscan.scan(None, 8, ks, 5, path=path, solve=s)
    assert len(s.calls) == len(ks) - 3
    assert np.allclose(s.calls[0], ks[3])
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[2], ref[2])
    assert [r["k"] for r in _lines(path)[1:]] == list(range(len(ks)))
    # a finished scan solves nothing on a rerun
    s2 = StandIn()
    again = bandscan.scan(None, 8, ks, 5, path=path, solve=s2)
    assert s2.calls == [] and np.array_equal(again[0], ref[0])


def test_final_line_cut_short_is_recomputed(tmp_path):
    ks = sc_path(1)
    path = str(tmp_path / "scan.jsonl")
    ref = bandscan.scan(None, 8, ks, 4, path=path, solve=StandIn())
    raw = open(path, "rb").read()
    last_start = raw.rstrip(b"\n").rfind(b"\n") + 1
    with open(path, "wb") as f:
        f.write(raw[:last_start + (len(raw) - last_start) // 2])  # half of the last record
    s = StandIn()
    got = bandscan.scan(None, 8, ks, 4, path=path, solve=s)
    assert len(s.calls) == 1 and np.allclose(s.calls[0], ks[-1])
    assert np.array_equal(got[0], ref[0])
    assert [r["k"] for r in _lines(path)[1:]] == list(range(len(ks)))


def test_record_of_another_scan_is_refused_untouched(tmp_path):
    ks = sc_path(1)
    path = str(tmp_path / "scan.jsonl")
    bandscan.scan(None, 8, ks, 4, path=path, solve=StandIn())
    before = open(path, "rb").read()
    for kwargs in ({"N": 8, "kappas": ks, "nev": 6}, {"N": 10, "kappas": ks, "nev": 4},
                   {"N": 8, "kappas": ks[:-1], "nev": 4}, {"N": 8, "kappas": ks, "nev": 4, "sigma": -3.0}):
        with pytest.raises(ValueError):
            bandscan.scan(None, path=path, solve=StandIn(), **kwargs)
    assert open(path, "rb").read() == before


def test_corrupt_inner_line_is_an_error(tmp_path):
    ks = sc_path(1)
    path = str(tmp_path / "scan.jsonl")
    bandscan.scan(None, 8, ks, 4, path=path, solve=StandIn())
    lines = open(path).read().split("\n")
    lines[2] = lines[2][:10]
    open(path, "w").write("\n".join(lines))
    with pytest.raises(ValueError):
        bandscan.scan(None, 8, ks, 4, path=path, solve=StandIn())
    other = str(tmp_path / "other.txt")
    open(other, "w").write("not a scan")
    with pytest.raises(ValueError):
        bandscan.scan(None, 8, ks, 4, path=other, solve=StandIn())
