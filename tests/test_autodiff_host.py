"""Host logic of the differentiation wrappers, without a GPU: degenerate clusters, the
subspace weights that make cluster gradients basis independent, and the band-gap
gradient's choice of active Bloch vectors and weights (the eigen-solve and the adjoint
kernel are replaced by stand-ins with known outputs)."""

import math

import numpy as np
import pytest

from paper_2606_03599_gb300 import autodiff


def test_clusters_group_relative_ties_only():
    ev = np.array([1.0, 1.0 + 1e-12, 2.0, 3.0, 3.0 * (1 + 5e-10), 3.0 * (1 + 2e-9), 4.0])
    assert autodiff.clusters(ev) == [[0, 1], [2], [3, 4], [5], [6]]
    assert autodiff.clusters(ev, cluster_tol=1e-8) == [[0, 1], [2], [3, 4, 5], [6]]
    assert autodiff.clusters(np.array([5.0])) == [[0]]


def test_subspace_weights_share_the_cluster_mean():
    ev = np.array([1.0, 1.0, 1.0, 2.0, 3.0, 3.0])
    g = np.array([3.0, 0.0, 0.0, 7.0, -1.0, 1.0])
    w = autodiff.subspace_weights(ev, g)
    assert np.array_equal(w, [1.0, 1.0, 1.0, 7.0, 0.0, 0.0])
    # the total weight of every cluster (the gradient of the cluster's sum) is unchanged
    for grp in autodiff.clusters(ev):
        assert math.isclose(w[grp].sum(), g[grp].sum(), abs_tol=1e-15)
    assert np.array_equal(g, [3.0, 0.0, 0.0, 7.0, -1.0, 1.0])  # input not modified


def test_band_gap_uses_the_two_active_bloch_vectors(monkeypatch):
    kappas = [(0.0, 0.0, 0.0), (0.25, 0.0, 0.0), (0.5, 0.0, 0.0), (0.5, 0.5, 0.0)]
    # eigenvalues per Bloch vector (SI); band lo = 1, band hi = 2
    table = {kappas[0]: [1.0e8, 4.0e8, 9.0e8], kappas[1]: [1.5e8, 5.0e8, 8.5e8],
             kappas[2]: [2.0e8, 4.5e8, 8.0e8], kappas[3]: [2.5e8, 3.9e8, 9.5e8]}
    N = 4
    n = N ** 3

    def fake_eigs(g, k, nev, opt=None, **kw):
        return np.array(table[tuple(k)][:nev]), np.zeros(nev, dtype=int), {}

    calls = []

    def fake_grads(g, N_, k, nev, weights=None, opt=None, **kw):
        calls.append((tuple(k), np.array(weights)))
        idx = kappas.index(tuple(k)) + 1
        return np.array(table[tuple(k)][:nev]), np.full((n, 21), float(idx)), np.full(n, 10.0 * idx)

    monkeypatch.setattr(autodiff.pc, "pc_eigs", fake_eigs)
    monkeypatch.setattr(autodiff, "nodewise_gradients", fake_grads)
    width, dC, drho = autodiff.band_gap(None, N, kappas, 1)

    f = {k: np.sqrt(np.array(v)) / (2 * np.pi) for k, v in table.items()}
    top_k = min(kappas, key=lambda k: f[k][2])  # lowest band 2
    bot_k = max(kappas, key=lambda k: f[k][1])  # highest band 1
    assert top_k == kappas[2] and bot_k == kappas[1]
    assert math.isclose(width, f[top_k][2] - f[bot_k][1], rel_tol=1e-15)
    # weights: +df/dlambda on band 2 at the top point, -df/dlambda on band 1 at the bottom point
    (k1, w1), (k2, w2) = calls
    assert k1 == top_k and k2 == bot_k
    assert np.allclose(w1, [0.0, 0.0, 1.0 / (8 * np.pi ** 2 * f[top_k][2])], rtol=1e-15, atol=0)
    assert np.allclose(w2, [0.0, -1.0 / (8 * np.pi ** 2 * f[bot_k][1]), 0.0], rtol=1e-15, atol=0)
    # df/dlambda = 1 / (8 pi^2 f) is the derivative of f = sqrt(lambda) / (2 pi)
    lam = table[top_k][2]
    h = lam * 1e-7
    fd = (np.sqrt(lam + h) - np.sqrt(lam - h)) / (2 * np.pi) / (2 * h)
    assert math.isclose(fd, 1.0 / (8 * np.pi ** 2 * f[top_k][2]), rel_tol=1e-8)
    # the gradients of the two active points add up
    assert np.all(dC == 3.0 + 2.0) and np.all(drho == 30.0 + 20.0)


def test_band_gap_width_is_negative_when_bands_overlap(monkeypatch):
    """A negative width (bands overlap across the k-set) is returned as is, not clipped."""
    kappas = [(0.0, 0.0, 0.0), (0.5, 0.0, 0.0)]
    table = {kappas[0]: [1.0e8, 5.0e8, 6.0e8], kappas[1]: [1.0e8, 7.0e8, 8.0e8]}

    monkeypatch.setattr(autodiff.pc, "pc_eigs",
                        lambda g, k, nev, opt=None, **kw: (np.array(table[tuple(k)][:nev]), np.zeros(nev), {}))
    monkeypatch.setattr(autodiff, "nodewise_gradients",
                        lambda g, N, k, nev, weights=None, opt=None, **kw: (None, np.zeros((8, 21)), np.zeros(8)))
    width, _, _ = autodiff.band_gap(None, 2, kappas, 1)
    f_hi = np.sqrt(6.0e8) / (2 * np.pi)
    f_lo = np.sqrt(7.0e8) / (2 * np.pi)
    assert width < 0 and math.isclose(width, f_hi - f_lo, rel_tol=1e-15)


@pytest.mark.parametrize("tol", [1e-9, 1e-6])
def test_subspace_weights_identity_without_degeneracy(tol):
    ev = np.array([1.0, 2.0, 3.0, 4.0])
    g = np.array([0.5, -1.0, 2.0, 0.0])
    assert np.array_equal(autodiff.subspace_weights(ev, g, tol), g)
