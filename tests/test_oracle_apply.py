"""Pins of the oracle apply A_h = B_h C_h B_h^H against closed forms and invariants (CPU only)."""

import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from oracle import sparse_ops as so
from workloads import complex_gaussian, isotropic_voigt, two_phase_sphere

KAPPAS = [np.array([0.3, 0.1, 0.2]), np.zeros(3), np.array([0.5, 0.5, 0.5]),
          np.array([1.3, 0.1, -0.8])]


def _cell(N=8, seed=1, R=0.35):
    return O.problem_from_cell(two_phase_sphere(N, R, seed), C0=1e9, rho0=1e3)


def _voigt_from_dict(d):
    C = np.zeros((6, 6))
    for key, v in d.items():
        p, q = int(key[0]) - 1, int(key[1]) - 1
        C[p, q] = C[q, p] = v
    return C


@pytest.mark.parametrize("kappa", KAPPAS[:3])
def test_c_apply_equals_sparse_transcription(kappa):
    pb = _cell()
    x = complex_gaussian((3, pb.n), 11)
    A, M = O.sparse_pencil(pb, kappa)
    y_ref = (A @ x.reshape(-1) - 0.37 * (M @ x.reshape(-1))).reshape(3, -1)
    y = O.apply_full(pb, kappa, x, shift=0.37)
    assert np.linalg.norm(y - y_ref) <= 1e-14 * np.linalg.norm(y_ref)


@pytest.mark.parametrize("N", [4, 6, 8])
@pytest.mark.parametrize("mode", [(0, 0, 0), (1, 2, 3), (3, 1, 5), (2, 3, 1)])
def test_plane_wave_identity(N, mode):
    """A (psi_m u) = psi_m B_hat(m) C B_hat(m)^H u for a homogeneous medium (Sec. 5.3, App. B).

    A sign error in a shift direction, a transposed Voigt index or a dropped
    derivative term changes B_hat and fails this identity.
    """
    rng = np.random.default_rng(5)
    G = rng.standard_normal((6, 6))
    C = G @ G.T + 6 * np.eye(6)
    a_lat = np.array([[1.0, 0.2, 0.0], [0.1, 1.1, 0.3], [0.0, -0.2, 0.9]])
    hp = O.homogeneous_problem(N, C, 2.5, a_lat=a_lat)
    kappa = np.array([0.23, -0.41, 0.17])
    p, q, r = (m % N for m in mode)
    psi = O.plane_wave(hp.dims, kappa, p, q, r)
    u = np.array([0.3, -1.2 + 0.5j, 0.7j])
    x = np.stack([psi * u[a] for a in range(3)])
    Bh = O.symbol_block(hp.dims, kappa, hp.ainv, p, q, r)
    # strain and divergence separately, then the composite
    e = O.strain_full(hp, kappa, x)
    e_ref = np.stack([psi * v for v in Bh.conj().T @ u])
    assert np.abs(e - e_ref).max() <= 1e-12 * np.abs(e_ref).max() + 1e-14
    y = O.apply_full(hp, kappa, x)
    pred = Bh @ C @ Bh.conj().T @ u
    y_ref = np.stack([psi * pred[a] for a in range(3)])
    assert np.abs(y - y_ref).max() <= 1e-12 * max(np.abs(y_ref).max(), 1e-300) + 1e-14


def test_symbol_low_frequency_consistency():
    """delta_s(theta) = i xi_s + O(h |xi|^2) (Remark symbol_consistency)."""
    for N in (16, 32, 64):
        dims = (N, N, N)
        kappa = np.array([0.05, -0.03, 0.02])  # p = q = r = 0
        Bh = O.symbol_block(dims, kappa, np.eye(3), 0, 0, 0)
        eta = np.array([Bh[0, 0], Bh[1, 1], Bh[2, 2]])
        xi = 2 * np.pi * kappa  # reduced derivative of exp(i xi . r)
        # eta = -i delta ~ -i (i xi) = xi
        err = np.abs(eta - xi).max()
        assert err <= 2.0 * (1.0 / N) * np.sum(xi ** 2) + 1e-12


def test_christoffel_long_wave_silicon(golden_dir):
    """Long-wave limit: lowest eigenvalues -> rho v^2 |q|^2 with textbook cubic velocities.

    Along [100]: C11 (longitudinal), C44 (two transverse).  Along [110]:
    (C11+C12+2C44)/2, C44, (C11-C12)/2.  Pins the Voigt order and the
    engineering-shear convention (Sec. 2, Eqs. tau_voigt_main, eps_voigt_main).
    """
    with open(os.path.join(golden_dir, "paper_materials.json")) as f:
        mat = json.load(f)
    C = _voigt_from_dict(mat["silicon"]["C"])  # GPa
    rho = mat["silicon"]["rho"] / 1e3
    N = 8
    hp = O.homogeneous_problem(N, C, rho)
    eps = 0.004
    for direction, expect in (((1, 0, 0), [C[3, 3], C[3, 3], C[0, 0]]),
                              ((1, 1, 0), [(C[0, 0] - C[0, 1]) / 2, C[3, 3],
                                           (C[0, 0] + C[0, 1] + 2 * C[3, 3]) / 2])):
        kappa = eps * np.array(direction, dtype=float)
        q2 = np.sum((2 * np.pi * kappa) ** 2)
        # each parity block carries one copy of the acoustic branches (fourfold for a
        # homogeneous medium), so read the branches from one block's spectrum
        ev = O.dense_eigvals(hp, kappa, 0)[:3]
        pred = np.sort(np.array(expect)) * q2 / rho
        assert np.allclose(np.sort(ev), pred, rtol=1e-3)


def test_isotropic_sound_speeds():
    lam, mu, rho = 40.0, 30.0, 1.2
    hp = O.homogeneous_problem(8, isotropic_voigt(lam, mu), rho)
    kappa = np.array([0.003, 0.002, -0.001])
    q2 = np.sum((2 * np.pi * kappa) ** 2)
    ev = O.dense_eigvals(hp, kappa, 2)[:3]
    assert np.allclose(ev, np.array([mu, mu, lam + 2 * mu]) * q2 / rho, rtol=1e-3)
    full = O.dense_eigvals(hp, kappa)[:12]
    assert np.allclose(full.reshape(3, 4), np.repeat(ev[:, None], 4, axis=1), rtol=1e-9)


@pytest.mark.parametrize("kappa", KAPPAS)
def test_hermitian_and_psd(kappa):
    pb = _cell()
    x = complex_gaussian((3, pb.n), 1)
    z = complex_gaussian((3, pb.n), 2)
    Ax = O.apply_full(pb, kappa, x)
    Az = O.apply_full(pb, kappa, z)
    lhs = np.vdot(z, Ax)
    rhs = np.conj(np.vdot(x, Az))
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(Ax) * np.linalg.norm(z)
    # x^H A x = || C^1/2 B^H x ||^2 >= 0, real
    q = np.vdot(x, Ax)
    assert abs(q.imag) <= 1e-13 * abs(q.real)
    e = O.strain_full(pb, kappa, x)
    Cn = pb.node_C()
    energy = np.real(np.einsum("vn,nvw,wn->", np.conj(e), Cn, e))
    assert q.real > 0
    assert abs(q.real - energy) <= 1e-12 * energy


@pytest.mark.parametrize("kappa", KAPPAS)
def test_strain_divergence_adjoint(kappa):
    """<B^H x, t> = <x, B t> with strain and divergence evaluated by separate code paths."""
    pb = _cell(N=6, seed=3)
    x = complex_gaussian((3, pb.n), 3)
    t = complex_gaussian((6, pb.n), 4)
    lhs = np.vdot(O.strain_full(pb, kappa, x), t)
    rhs = np.vdot(x, O.divergence_full(pb, kappa, t))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


@pytest.mark.parametrize("kappa", KAPPAS[:2])
def test_theorem_4_1_commutation(kappa):
    """A_h Gamma_a = Gamma_a A_h and M_h Gamma_a = Gamma_a M_h (Theorem 4.1)."""
    pb = _cell(N=8, seed=9)
    g12, g13 = so.parity_signs(pb.dims)
    x = complex_gaussian((3, pb.n), 8)
    for g in (g12, g13):
        lhs = O.apply_full(pb, kappa, g[None, :] * x)
        rhs = g[None, :] * O.apply_full(pb, kappa, x)
        assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(rhs).max()


def test_bloch_symmetries_of_spectrum():
    """Spectra at kappa, -kappa and kappa + e_l coincide (Bloch periodicity of the phases)."""
    pb = _cell(N=4, seed=2)
    k = np.array([0.3, 0.1, 0.2])
    e0 = O.dense_eigvals(pb, k)
    for kk in (-k, k + np.array([1.0, 0, 0]), k + np.array([0, -1.0, 0]), k + np.array([0, 0, 2.0])):
        e1 = O.dense_eigvals(pb, kk)
        assert np.abs(e1 - e0).max() <= 1e-11 * np.abs(e0).max()


def test_sampled_apply_matches_full():
    pb = _cell(N=8, seed=4)
    kappa = KAPPAS[3]
    x = complex_gaussian((3, pb.n), 5)
    nodes = np.array([0, 1, 7, 8, 63, 64, 200, 511])
    y = O.apply_full(pb, kappa, x, shift=1.5)
    ys = O.apply_at_nodes(pb, kappa, x, nodes, shift=1.5)
    assert np.abs(ys - y[:, nodes].T).max() <= 1e-14 * np.abs(y).max()


def test_golden_materials_match_workloads(golden_dir):
    from workloads import quartz_silicon_constants
    with open(os.path.join(golden_dir, "paper_materials.json")) as f:
        mat = json.load(f)
    Cq, rq, Cs, rs = quartz_silicon_constants()
    assert np.array_equal(Cq / 1e9, _voigt_from_dict(mat["quartz"]["C"]))
    assert np.array_equal(Cs / 1e9, _voigt_from_dict(mat["silicon"]["C"]))
    assert rq == mat["quartz"]["rho"] and rs == mat["silicon"]["rho"]


def test_fcc_workload_geometry():
    """The paper's FCC cell generator: primitive cell volume a0^3 / 4, the sphere inside the
    cell, sub-pixel fractions in [0, 1] summing to the sphere's volume fraction."""
    import math
    from workloads import fcc_lattice, fcc_quartz_silicon_cell
    from workloads.materials import FCC_A0
    A = fcc_lattice()
    assert abs(abs(np.linalg.det(A)) - FCC_A0 ** 3 / 4) <= 1e-15
    cell = fcc_quartz_silicon_cell(32)
    th = cell.theta.astype(np.float64)
    assert th.min() >= 0.0 and th.max() <= 1.0
    exact = (4.0 / 3.0) * math.pi * (0.25 * FCC_A0) ** 3 / (FCC_A0 ** 3 / 4)
    assert abs(th.mean() - exact) <= 2e-4
    assert 0 < np.count_nonzero((th > 0) & (th < 1)) < th.size // 4


def test_fcc_path_and_bloch_vector_conversion():
    """The paper's 91-point FCC path (9 segments of 10 intervals, vertices in route order), and
    the conversion of its Cartesian points (units 2 pi / a0) to reduced kappa with
    q . a_l = 2 pi kappa_l; kappa is defined modulo integers, so Gamma maps to 0 and L, which
    both readings share, to (1/2, 1/2, 1/2)."""
    from workloads import FCC_POINTS, fcc_kappa, fcc_lattice, fcc_path
    from workloads.kpath import FCC_ROUTE
    from workloads.materials import FCC_A0
    path = fcc_path(10)
    assert path.shape == (91, 3)
    for s, name in enumerate(FCC_ROUTE):
        assert np.array_equal(path[10 * s], FCC_POINTS[name])
    A = fcc_lattice()
    for name, k in FCC_POINTS.items():
        kap = fcc_kappa(k, A, FCC_A0)
        q = 2 * np.pi * np.asarray(k) / FCC_A0
        assert np.allclose([q @ A[:, l] for l in range(3)], 2 * np.pi * kap, rtol=0, atol=1e-12)
    assert np.allclose(fcc_kappa(FCC_POINTS["G"], A, FCC_A0), 0.0)
    assert np.allclose(fcc_kappa(FCC_POINTS["L"], A, FCC_A0), 0.5)
