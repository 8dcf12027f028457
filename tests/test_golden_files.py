"""Consistency of the stored oracle eigenvalues of the N = 48 cell (no GPU): every Bloch vector's
merged list is the lowest 20 of the union of its four block spectra (Cor. 4.2), each block list is
ascending and positive (Gamma's zero modes were projected out, Sec. 6.2), and every block holds
enough values for the merge to be complete."""

import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "arpack_n48.json")


def test_arpack_n48_golden_is_a_complete_merge():
    with open(GOLDEN) as f:
        g = json.load(f)
    assert g["nev_merged"] == 20 and "make_arpack_n48.py" in g["command"]
    assert [p["name"] for p in g["points"]] == ["Gamma", "X", "generic"]
    for p in g["points"]:
        blocks = [np.array(b) for b in p["blocks"]]
        assert len(blocks) == 4
        for b in blocks:
            assert (np.diff(b) >= 0).all() and (b > 0).all()
        union = np.sort(np.concatenate(blocks))[:20]
        assert np.array_equal(union, np.array(p["merged"]))
        assert p["complete"] and all(b.max() >= union[-1] for b in blocks)
