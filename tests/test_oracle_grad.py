"""Pins of the oracle's eigenvalue gradients (Hellmann-Feynman for the pencil of
Eq. discrete_GEP_main) against things other than the formula itself:

* central finite differences of dense LAPACK eigenvalues along seeded random
  nodewise directions of stiffness and density;
* Euler homogeneity: lambda is homogeneous of degree 1 in the stiffness and of
  degree -1 in the density, so sum_l <dlambda/dC_l, C_l> = lambda and
  sum_l rho_l dlambda/drho_l = -lambda;
* block support: a block eigenvalue does not depend on material off its block
  (Theorem 4.1), so its gradient vanishes there.
"""

import numpy as np
import pytest

from oracle import oracle as O
from workloads import two_phase_sphere

KAPPA = (0.13, 0.27, 0.41)


def _problem(N=4):
    cell = two_phase_sphere(N, 0.35, 1)
    pb = O.problem_from_cell(cell, C0=1e9, rho0=1e3, L=1.0)
    pb.C_nodes = pb.node_C().copy()
    pb.rho_nodes = pb.node_rho().copy()
    return pb


def _perturbed(pb, dC, drho, h):
    q = O.Problem(dims=pb.dims, ainv=pb.ainv, C=pb.C, rho=pb.rho, theta=pb.theta,
                  C_nodes=pb.C_nodes + h * dC, rho_nodes=pb.rho_nodes + h * drho)
    return q


def _direction(pb, rng):
    n = pb.n
    a = rng.standard_normal((n, 6, 6))
    dC = 0.5 * (a + np.transpose(a, (0, 2, 1))) * np.abs(pb.C_nodes).max()
    drho = rng.standard_normal(n) * pb.rho_nodes.max()
    return dC, drho


def _directional(gC, grho, dC, drho):
    iu = np.triu_indices(6)
    return float(np.sum(gC[:, iu[0], iu[1]] * dC[:, iu[0], iu[1]]) + np.sum(grho * drho))


@pytest.mark.parametrize("b", [0, 1, 2, 3])
def test_gradient_matches_central_differences(b):
    pb = _problem()
    w, X = O.dense_eigpairs(pb, KAPPA, b)
    rng = np.random.default_rng(100 + b)
    for j in range(3):
        assert min(w[j + 1] - w[j], w[j] - (w[j - 1] if j else -np.inf)) > 1e-3 * w[j]
        gC, grho = O.eigpair_gradients(pb, KAPPA, X[j], w[j])
        for _ in range(3):
            dC, drho = _direction(pb, rng)
            h = 1e-5
            lp = O.dense_eigvals(_perturbed(pb, dC, drho, h), KAPPA, b)[j]
            lm = O.dense_eigvals(_perturbed(pb, dC, drho, -h), KAPPA, b)[j]
            fd = (lp - lm) / (2 * h)
            an = _directional(gC, grho, dC, drho)
            assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * w[j]), (fd, an)


@pytest.mark.parametrize("b", [0, 3])
def test_gradient_euler_identities_and_block_support(b):
    pb = _problem()
    w, X = O.dense_eigpairs(pb, KAPPA, b)
    idx = O.block_index(pb.dims, b)
    off = np.setdiff1d(np.arange(pb.n), idx)
    iu = np.triu_indices(6)
    for j in range(4):
        gC, grho = O.eigpair_gradients(pb, KAPPA, X[j], w[j])
        assert np.isclose(np.sum(gC[:, iu[0], iu[1]] * pb.C_nodes[:, iu[0], iu[1]]), w[j], rtol=1e-10)
        assert np.isclose(np.sum(grho * pb.rho_nodes), -w[j], rtol=1e-10)
        assert np.abs(gC[off]).max() == 0.0 and np.abs(grho[off]).max() == 0.0


def test_planted_mistake_in_gradient_is_caught():
    """A dropped factor 2 on the off-diagonal entries fails the finite-difference pin."""
    pb = _problem()
    w, X = O.dense_eigpairs(pb, KAPPA, 0)
    gC, grho = O.eigpair_gradients(pb, KAPPA, X[0], w[0])
    off = ~np.eye(6, dtype=bool)
    bad = gC.copy()
    bad[:, off] *= 0.5
    dC, drho = _direction(pb, np.random.default_rng(7))
    h = 1e-5
    fd = (O.dense_eigvals(_perturbed(pb, dC, drho, h), KAPPA, 0)[0]
          - O.dense_eigvals(_perturbed(pb, dC, drho, -h), KAPPA, 0)[0]) / (2 * h)
    assert abs(fd - _directional(gC, grho, dC, drho)) <= 1e-6 * abs(fd)
    assert abs(fd - _directional(bad, grho, dC, drho)) > 1e-3 * abs(fd)
