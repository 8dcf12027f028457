"""Pins of the oracle's reference-medium preconditioner (Sec. 5.4) and of the inverse block
Fourier transform it uses (Sec. 5.2).

The decisive pin is exactness on a homogeneous medium: there the reference material is the
material itself, and z = P r must solve (A_sigma - sigma M_sigma) z = r with the operator
evaluated by the matrix-free C apply, which shares nothing with the symbols, the weighted
SVD or the separable transforms.  A wrong transform sign or normalisation, a transposed
symbol block, a wrong shift sign or a wrong mode set each break it.
"""

import numpy as np
import pytest

from oracle import oracle as O
from workloads import complex_gaussian, two_phase_sphere

SKEW = np.array([[1.0, 0.2, 0.0], [0.1, 1.1, 0.3], [0.0, -0.2, 0.9]])


def _spd6(seed):
    G = np.random.default_rng(seed).standard_normal((6, 6))
    return G @ G.T + 6 * np.eye(6)


def _hdot(a, b):
    return np.vdot(np.ravel(a), np.ravel(b))


@pytest.mark.parametrize("N", [4, 6, 8])
def test_separable_inverse_equals_dense_basis(N):
    dims = (N, N, N)
    kappa = np.array([0.3, -0.1, 0.45])
    for b in range(4):
        T = O.T_sigma_dense(dims, kappa, b)
        what = complex_gaussian(N ** 3 // 4, 40 + b)
        ref = T @ what
        got = O.block_fourier_separable_inverse(what.reshape(N, N // 2, N // 2), dims, kappa, b).reshape(-1)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
        back = O.block_fourier_separable(got.reshape(N, N // 2, N // 2), dims, kappa, b).reshape(-1)
        assert np.abs(back - what).max() <= 1e-12 * np.abs(what).max()


def test_weighted_svd_local_factorisation():
    """B_hat = P Sigma Q^{H,Psi}, Q^{H,Psi} Q = I (Eq. weighted_svd_local_unified) for a general Psi."""
    rng = np.random.default_rng(8)
    G = rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6))
    Psi = G @ G.conj().T + 2 * np.eye(6)
    dims = (8, 8, 8)
    for mode in [(1, 2, 3), (0, 0, 0), (3, 1, 7)]:
        Bh = O.symbol_block(dims, [0.23, -0.41, 0.17], SKEW, *mode)
        P, sig, Q, QH = O.weighted_svd(Bh, Psi)
        assert np.allclose(P.conj().T @ P, np.eye(3), atol=1e-13)
        assert np.abs((P * sig) @ QH - Bh).max() <= 1e-12 * max(np.abs(Bh).max(), 1.0)
        assert np.abs(QH @ Q - np.eye(3)).max() <= 1e-12
        # Psi = I reduces to the ordinary SVD
        _, sig_i, _, _ = O.weighted_svd(Bh, np.eye(6))
        assert np.allclose(sig_i, np.linalg.svd(Bh, compute_uv=False), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("N", [4, 6, 8])
@pytest.mark.parametrize("kappa", [[0.23, -0.41, 0.17], [0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
@pytest.mark.parametrize("a_lat", ["cubic", "skew"])
def test_precond_is_exact_inverse_for_homogeneous_medium(N, kappa, a_lat):
    C = _spd6(5)
    rho = 2.5
    hp = O.homogeneous_problem(N, C, rho, a_lat=None if a_lat == "cubic" else SKEW)
    sigma = -0.3 * np.abs(C).max() / rho
    for b in range(4):
        r = complex_gaussian((3, N ** 3 // 4), 60 + b)
        z = O.precond_block(hp, kappa, b, sigma, r)
        back = O.apply_block(hp, kappa, b, z, shift=sigma)
        assert np.abs(back - r).max() <= 1e-11 * np.abs(r).max()


def test_full_space_precond_is_exact_inverse_for_homogeneous_medium():
    N = 6
    C = _spd6(6)
    hp = O.homogeneous_problem(N, C, 1.7, a_lat=SKEW)
    sigma = -0.25 * np.abs(C).max() / 1.7
    kappa = [0.1, 0.35, -0.2]
    r = complex_gaussian((3, N ** 3), 70)
    z = O.precond_full(hp, kappa, sigma, r)
    back = O.apply_full(hp, kappa, z, shift=sigma)
    assert np.abs(back - r).max() <= 1e-11 * np.abs(r).max()


def test_precond_hermitian_positive_definite_and_label_invariant():
    cell = two_phase_sphere(8, 0.35, 1)
    pb = O.problem_from_cell(cell, C0=1e9, rho0=1e3)
    sigma = -0.3 * np.abs(pb.C).max() / pb.rho.max()
    kappa = np.array([0.3, 0.1, 0.2])
    for b in (0, 3):
        x = complex_gaussian((3, 128), 80 + b)
        y = complex_gaussian((3, 128), 90 + b)
        Px = O.precond_block(pb, kappa, b, sigma, x)
        Py = O.precond_block(pb, kappa, b, sigma, y)
        assert abs(_hdot(x, Py) - np.conj(_hdot(y, Px))) <= 1e-13 * abs(_hdot(x, Px))
        xPx = _hdot(x, Px)
        assert xPx.real > 0 and abs(xPx.imag) <= 1e-13 * xPx.real
        # the operator depends on exp(i phi) only: integer shifts of kappa relabel the modes
        Px2 = O.precond_block(pb, kappa + np.array([1.0, -1.0, 2.0]), b, sigma, x)
        assert np.abs(Px2 - Px).max() <= 1e-12 * np.abs(Px).max()


def test_single_mode_input_maps_to_scaled_mode():
    """T_sigma column m times u maps to the same column times F(m) u (the diagonal form of Sec. 5.4)."""
    cell = two_phase_sphere(8, 0.35, 1)
    pb = O.problem_from_cell(cell, C0=1e9, rho0=1e3)
    C_ref, rho_ref = O.reference_medium(pb)
    sigma = -0.3 * np.abs(pb.C).max() / pb.rho.max()
    kappa = [0.3, 0.1, 0.2]
    u = np.array([0.4 - 0.2j, 1.1, -0.3j])
    for b, m in ((0, (1, 0, 0)), (2, (3, 2, 7)), (3, (0, 0, 0))):
        col = O.block_mode_vector(pb.dims, kappa, b, *m)
        T = O.T_sigma_dense(pb.dims, kappa, b)
        X = pb.dims[0] // 2
        assert np.abs(col - T[:, m[0] + X * (m[1] + X * m[2])]).max() <= 1e-14
        z = O.precond_block(pb, kappa, b, sigma, np.outer(u, col))
        F = O.precond_mode_factor(pb, kappa, sigma, *m, C_ref, rho_ref)
        ref = np.outer(F @ u, col)
        assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max()


def test_reference_medium_is_the_nodal_average():
    cell = two_phase_sphere(8, 0.35, 1)
    pb = O.problem_from_cell(cell, C0=1e9, rho0=1e3)
    C_ref, rho_ref = O.reference_medium(pb)
    assert np.allclose(C_ref, pb.node_C().mean(axis=0), rtol=1e-14, atol=0)
    assert np.isclose(rho_ref, pb.node_rho().mean(), rtol=1e-14)


def test_planted_transposed_mode_factor_fails_the_exactness_pin(monkeypatch):
    """Planted mistake: each mode's 3x3 factor transposed (P -> conj P) must break the pin."""
    real = O.weighted_svd

    def wrong(Bh, Psi):
        P, sig, Q, QH = real(Bh, Psi)
        return P.conj(), sig, Q, QH

    monkeypatch.setattr(O, "weighted_svd", wrong)
    N = 4
    C = _spd6(5)
    hp = O.homogeneous_problem(N, C, 2.5)
    sigma = -0.3 * np.abs(C).max() / 2.5
    kappa = [0.23, -0.41, 0.17]
    r = complex_gaussian((3, N ** 3 // 4), 61)
    z = O.precond_block(hp, kappa, 1, sigma, r)
    back = O.apply_block(hp, kappa, 1, z, shift=sigma)
    assert np.abs(back - r).max() > 1e-3 * np.abs(r).max()


@pytest.mark.parametrize("mistake", ["shift_sign", "conjugate_forward"])
def test_planted_shift_sign_or_conjugated_transform_fails_the_exactness_pin(monkeypatch, mistake):
    """Planted mistakes: the shift term added with the wrong sign, or the forward transform
    taken with the conjugate phase (the inverse left as is); each must break the pin."""
    N = 4
    C = _spd6(5)
    hp = O.homogeneous_problem(N, C, 2.5)
    sigma = -0.3 * np.abs(C).max() / 2.5
    kappa = [0.23, -0.41, 0.17]
    if mistake == "shift_sign":
        real = O.precond_mode_factor

        def wrong(pb, kap, sig, p, q, r, C_ref, rho_ref):
            return real(pb, kap, -sig, p, q, r, C_ref, rho_ref)

        monkeypatch.setattr(O, "precond_mode_factor", wrong)
    else:
        real = O.block_fourier_separable

        def wrong(w, dims, kap, b):
            return np.conj(real(np.conj(w), dims, kap, b))

        monkeypatch.setattr(O, "block_fourier_separable", wrong)
    r = complex_gaussian((3, N ** 3 // 4), 62)
    z = O.precond_block(hp, kappa, 2, sigma, r)
    back = O.apply_block(hp, kappa, 2, z, shift=sigma)
    assert np.abs(back - r).max() > 1e-3 * np.abs(r).max()
