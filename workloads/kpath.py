"""Bloch-vector samples in reduced reciprocal coordinates kappa (phase 2*pi*kappa_l).

Simple-cubic high-symmetry points: Gamma=(0,0,0), X=(1/2,0,0), M=(1/2,1/2,0),
R=(1/2,1/2,1/2).
"""

from __future__ import annotations

import numpy as np

SC_POINTS = {
    "G": np.array([0.0, 0.0, 0.0]),
    "X": np.array([0.5, 0.0, 0.0]),
    "M": np.array([0.5, 0.5, 0.0]),
    "R": np.array([0.5, 0.5, 0.5]),
}
SC_ROUTE = ["G", "X", "M", "G", "R", "X"]


def sc_path(intervals_per_segment: int = 6) -> np.ndarray:
    """Gamma-X-M-Gamma-R-X with equal intervals per segment, all vertices included.

    With 6 intervals per segment this gives 5*6+1 = 31 points.
    """
    pts = [SC_POINTS["G"]]
    for a, b in zip(SC_ROUTE[:-1], SC_ROUTE[1:]):
        pa, pb = SC_POINTS[a], SC_POINTS[b]
        for s in range(1, intervals_per_segment + 1):
            pts.append(pa + (pb - pa) * (s / intervals_per_segment))
    return np.array(pts)


def sc_eight_points() -> np.ndarray:
    """Gamma, X, M, R and the midpoints of Gamma-X, X-M, M-Gamma, Gamma-R."""
    G, X, M, R = (SC_POINTS[c] for c in "GXMR")
    return np.array([G, X, M, R, (G + X) / 2, (X + M) / 2, (M + G) / 2, (G + R) / 2])


def sc_uniform_path(count: int) -> np.ndarray:
    """``count`` points equally spaced in arc length along Gamma-X-M-Gamma-R-X (ends included)."""
    verts = np.array([SC_POINTS[c] for c in SC_ROUTE])
    seg = np.linalg.norm(np.diff(verts, axis=0), axis=1)
    cum = np.concatenate([[0.0], np.cumsum(seg)])
    s = np.linspace(0.0, cum[-1], count)
    out = []
    for t in s:
        i = min(np.searchsorted(cum, t, side="right") - 1, len(seg) - 1)
        f = (t - cum[i]) / seg[i]
        out.append(verts[i] + f * (verts[i + 1] - verts[i]))
    return np.array(out)


# FCC high-symmetry points in reduced reciprocal coordinates (q . a_l = 2 pi kappa_l) of the
# paper's FCC example (Sec. 7, Eq. fcc_high_symmetry_points).
FCC_POINTS = {
    "G": np.array([0.0, 0.0, 0.0]),
    "X": np.array([0.0, 0.5, 0.5]),
    "W": np.array([0.25, 0.5, 0.75]),
    "K": np.array([0.375, 0.375, 0.75]),
    "L": np.array([0.5, 0.5, 0.5]),
    "U": np.array([0.25, 0.625, 0.625]),
}
FCC_ROUTE = ["G", "X", "W", "K", "G", "L", "U", "W", "L", "K"]


def fcc_path(intervals_per_segment: int = 10) -> np.ndarray:
    """The paper's FCC path Gamma-X-W-K-Gamma-L-U-W-L-K (Sec. 7) with equal intervals per
    segment, vertices included: 9 * 10 + 1 = 91 points, in the coordinates of ``FCC_POINTS``."""
    pts = [FCC_POINTS["G"]]
    for a, b in zip(FCC_ROUTE[:-1], FCC_ROUTE[1:]):
        pa, pb = FCC_POINTS[a], FCC_POINTS[b]
        for s in range(1, intervals_per_segment + 1):
            pts.append(pa + (pb - pa) * (s / intervals_per_segment))
    return np.array(pts)


def fcc_kappa(k_cartesian, a_lat, a0) -> np.ndarray:
    """Reduced Bloch vector kappa_l = a_l . k / a0 of a wave vector k given in Cartesian units of
    2 pi / a0 (the reading under which the paper's listed FCC points reproduce its printed
    results), so that q . a_l = 2 pi kappa_l with q = 2 pi k / a0."""
    return np.asarray(a_lat, dtype=np.float64).T @ np.asarray(k_cartesian, dtype=np.float64) / a0
