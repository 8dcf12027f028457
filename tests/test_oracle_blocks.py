"""Pins of the oracle's parity blocks, zero modes, Fourier basis and eigen oracles (CPU only)."""

import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from oracle import sparse_ops as so
from workloads import complex_gaussian, two_phase_sphere


def _cell(N=8, seed=1, R=0.35):
    return O.problem_from_cell(two_phase_sphere(N, R, seed), C0=1e9, rho0=1e3)


@pytest.mark.parametrize("N", [4, 6, 8])
def test_index_map_brute_force(N):
    """Blocks partition the nodes; block b holds exactly the nodes with
    ((i+j) mod 2, (i+k) mod 2) = (p12, p13), in ascending order (Eqs. V_sigma_main, Proj_sigma)."""
    dims = (N, N, N)
    seen = np.zeros(N ** 3, dtype=int)
    for b in range(4):
        idx = O.block_index(dims, b)
        assert idx.size == N ** 3 // 4
        assert np.all(np.diff(idx) > 0)
        seen[idx] += 1
        i, j, k = idx % N, (idx // N) % N, idx // (N * N)
        assert np.all((i + j) % 2 == (b >> 1)) and np.all((i + k) % 2 == (b & 1))
    assert np.all(seen == 1)


def test_projectors_orthogonal_and_complete():
    dims = (6, 6, 6)
    P = [so.projector_diag(dims, b) for b in range(4)]
    assert np.array_equal(sum(P), np.ones(216))
    for a in range(4):
        assert np.array_equal(P[a] * P[a], P[a])
        for b in range(a + 1, 4):
            assert not np.any(P[a] * P[b])


@pytest.mark.parametrize("kappa", [np.array([0.3, 0.1, 0.2]), np.zeros(3)])
def test_off_block_couplings_vanish(kappa):
    pb = _cell(N=6, seed=5)
    A, M = O.sparse_pencil(pb, kappa)
    lab = np.tile(O.block_of_node(pb.dims), 3)
    Acoo = A.tocoo()
    off = lab[Acoo.row] != lab[Acoo.col]
    assert np.all(Acoo.data[off] == 0)


@pytest.mark.parametrize("N", [4, 6, 8])
def test_plane_by_plane_closed_form_equals_per_mode_loop(N):
    """The array form used at large N equals the per-mode closed form (skew lattice, two kappas)."""
    rng = np.random.default_rng(9)
    G = rng.standard_normal((6, 6))
    C = G @ G.T + 3 * np.eye(6)
    ainv = np.linalg.inv(np.array([[1.0, 0.2, 0.0], [0.1, 1.1, 0.3], [0.0, -0.2, 0.9]]))
    for kappa in ([0.3, -0.1, 0.2], [0.0, 0.0, 0.0]):
        ref = O.homogeneous_spectrum((N,) * 3, kappa, ainv, C, 1.7)
        got = O.homogeneous_spectrum_planes((N,) * 3, kappa, ainv, C, 1.7)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("N", [4, 8])
@pytest.mark.parametrize("kappa", [np.array([0.3, 0.1, 0.2]), np.zeros(3), np.array([0.5, 0.5, 0.5])])
def test_merged_block_spectra_equal_full(N, kappa):
    """Cor. 4.2: the full spectrum is the union of the four block spectra."""
    pb = _cell(N=N, seed=6)
    ev_full = O.dense_eigvals(pb, kappa)
    ev_b = np.sort(np.concatenate([O.dense_eigvals(pb, kappa, b) for b in range(4)]))
    assert np.abs(ev_full - ev_b).max() <= 1e-12 * np.abs(ev_full).max()


def test_zero_mode_counts(golden_dir):
    with open(os.path.join(golden_dir, "paper_counts.json")) as f:
        counts = json.load(f)
    pb = _cell(N=8, seed=1)
    assert O.zero_mode_count(O.dense_eigvals(pb, np.zeros(3))) == counts["gamma_zero_modes_full"]
    for b in range(4):
        assert (O.zero_mode_count(O.dense_eigvals(pb, np.zeros(3), b))
                == counts["gamma_zero_modes_per_block"])
    assert O.zero_mode_count(O.dense_eigvals(pb, np.array([0.3, 0.1, 0.2]))) == 0
    assert O.zero_mode_count(O.dense_eigvals(pb, np.array([1.0, -2.0, 0.0]))) == 12


def test_gamma_null_vectors_in_kernel():
    """B_h(Gamma)^H chi_mu e_alpha = 0 for the four scalar modes (App. C)."""
    pb = _cell(N=6, seed=2)
    Z = O.gamma_null_basis(pb)
    assert Z.shape[1] == 12
    for c in range(12):
        e = O.strain_full(pb, np.zeros(3), Z[:, c].reshape(3, -1))
        assert np.abs(e).max() <= 1e-12
    assert np.linalg.matrix_rank(Z) == 12


def test_velocity_dof_counts(golden_dir):
    with open(os.path.join(golden_dir, "paper_counts.json")) as f:
        counts = json.load(f)
    for N, dof in counts["velocity_dofs"].items():
        assert 3 * int(N) ** 3 == dof
        assert sum(O.block_index((4, 4, 4), b).size for b in range(4)) == 64


def test_homogeneous_closed_form_and_fourfold():
    """Homogeneous spectrum = union of eig(B_hat C B_hat^H)/rho; each block holds it with multiplicity / 4."""
    rng = np.random.default_rng(7)
    G = rng.standard_normal((6, 6))
    C = G @ G.T + 3 * np.eye(6)
    hp = O.homogeneous_problem(4, C, 1.7)
    kappa = np.array([0.3, 0.1, 0.2])
    cf = O.homogeneous_spectrum(hp.dims, kappa, hp.ainv, C, 1.7)
    ev = O.dense_eigvals(hp, kappa)
    assert np.abs(ev - cf).max() <= 1e-12 * np.abs(cf).max()
    quarter = cf.reshape(-1, 4)
    assert np.abs(quarter - quarter[:, :1]).max() <= 1e-11 * np.abs(cf).max()
    for b in range(4):
        evb = O.dense_eigvals(hp, kappa, b)
        assert np.abs(evb - quarter[:, 0]).max() <= 1e-11 * np.abs(cf).max()


@pytest.mark.parametrize("N", [4, 8])
def test_block_fourier_separable_equals_dense(N):
    """T_sigma^H w by separable quarter-grid Bloch DFTs = dense T F_sigma (Eqs. f_sigma_unified, Tsigma_unified)."""
    dims = (N, N, N)
    kappa = np.array([0.3, -0.1, 0.45])
    for b in range(4):
        T = O.T_sigma_dense(dims, kappa, b)
        assert np.abs(T.conj().T @ T - np.eye(T.shape[0])).max() <= 1e-13
        w = complex_gaussian(T.shape[0], 10 + b)
        d = T.conj().T @ w
        s = O.block_fourier_separable(w.reshape(N, N // 2, N // 2), dims, kappa, b).reshape(-1)
        assert np.abs(d - s).max() <= 1e-12 * np.abs(d).max()


def test_block_symbol_diagonalises_homogeneous_block():
    """T_sigma^H A_sigma T_sigma = blockdiag_m B_hat(m) C B_hat(m)^H / for a homogeneous medium (Eq. Bhat_xi_def)."""
    N = 4
    rng = np.random.default_rng(8)
    G = rng.standard_normal((6, 6))
    C = G @ G.T + 3 * np.eye(6)
    hp = O.homogeneous_problem(N, C, 1.0)
    kappa = np.array([0.21, 0.37, -0.12])
    for b in (0, 3):
        A, _ = O.sparse_pencil(hp, kappa, b)
        T = O.T_sigma_dense(hp.dims, kappa, b)
        nb = T.shape[0]
        I3T = np.kron(np.eye(3), T)
        Ahat = I3T.conj().T @ A.toarray() @ I3T
        for c, (p, q, r) in enumerate(O.representatives(hp.dims)):
            Bh = O.symbol_block(hp.dims, kappa, hp.ainv, p, q, r)
            blk = Ahat[np.ix_([c, nb + c, 2 * nb + c], [c, nb + c, 2 * nb + c])]
            assert np.abs(blk - Bh @ C @ Bh.conj().T).max() <= 1e-11 * np.abs(Ahat).max()


@pytest.mark.parametrize("kappa", [np.array([0.3, 0.1, 0.2]), np.zeros(3)])
def test_shift_invert_oracle_matches_dense(kappa):
    pb = _cell(N=8, seed=1)
    dense = O.lowest_nonzero(O.dense_eigvals(pb, kappa), 12)
    lam = O.eigs_oracle(pb, kappa, 12, sigma=-5.0)
    assert np.abs(lam - dense).max() <= 1e-11 * dense.max()
    for b in range(4):
        dense_b = O.lowest_nonzero(O.dense_eigvals(pb, kappa, b), 4)
        lam_b = O.eigs_oracle(pb, kappa, 4, sigma=-5.0, b=b)
        assert np.abs(lam_b - dense_b).max() <= 1e-11 * dense_b.max()


def test_merge_rule():
    vals = [np.array([1.0, 3.0]), np.array([2.0, 2.5]), np.array([4.0]), np.array([0.5, 5.0])]
    merged, ok, ext = O.merge_complete(vals, [True] * 4, 4)
    assert np.array_equal(merged, [0.5, 1.0, 2.0, 2.5]) and ok
    merged, ok, ext = O.merge_complete(vals, [True] * 4, 6)
    # cut = 4.0: block 0 tops out at 3.0 and block 1 at 2.5 -> not known complete below 4.0
    assert not ok and ext == [0, 1]
