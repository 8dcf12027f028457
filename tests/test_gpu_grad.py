"""GPU parity of the adjoint (Hellmann-Feynman) gradient kernel and of the
autograd wrapper, through the C ABI, against the oracle.

* the kernel's per-node strain products equal the oracle's on random vectors in
  every layout (full space and the four parity blocks), FP64, 1e-12 relative;
* gradients of solver eigenvalues equal the oracle's dense-eigenvector gradients
  at N=8 (1e-7 relative), including degenerate clusters as subspaces;
* directional derivatives equal central finite differences of dense LAPACK
  eigenvalues on 50 seeded nodewise directions (stiffness and density);
* Euler homogeneity (degree 1 in C, degree -1 in rho) per band;
* d lambda / d theta through torch.autograd and the band-gap gradient equal
  central differences of the GPU's own eigenvalues.
"""

import numpy as np
import pytest

from oracle import oracle as O
from workloads import complex_gaussian, isotropic_voigt, two_phase_sphere

pytestmark = pytest.mark.gpu

KAPPA = (0.13, 0.27, 0.41)
IU = np.triu_indices(6)


@pytest.fixture(scope="module")
def pc():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_03599_gb300 as pc
    return pc


@pytest.fixture(scope="module")
def ad(pc):
    from paper_2606_03599_gb300 import autodiff
    return autodiff


class Grid:
    def __init__(self, pc, cell):
        self.pc, self.cell = pc, cell
        self.h = pc.pc_grid_create(cell.N, cell.C, cell.rho, phase=cell.phase, theta=cell.theta,
                                   a_lat=cell.a_lat)
        self.C0, self.rho0, self.L = pc.pc_grid_units(self.h)
        self.pb = O.problem_from_cell(cell, C0=self.C0, rho0=self.rho0, L=self.L)
        self.to_si = self.C0 / (self.rho0 * self.L ** 2)

    def close(self):
        self.pc.pc_grid_destroy(self.h)


def _oracle_weighted(g, kappa, X, lam_si, w):
    """sum_v w_v (dC [n,21] per Pa, drho [n] per kg/m^3) from the oracle, SI units."""
    n = g.pb.n
    dC, drho = np.zeros((n, 21)), np.zeros(n)
    for v in range(len(w)):
        gC, grho = O.eigpair_gradients(g.pb, kappa, X[v], lam_si[v])
        dC += w[v] * gC[:, IU[0], IU[1]] / (g.rho0 * g.L ** 2)
        drho += w[v] * grho / g.rho0
    return dC, drho


@pytest.mark.parametrize("block", [-1, 0, 1, 2, 3])
@pytest.mark.parametrize("N", [4, 8, 12])
def test_grad_kernel_matches_oracle_on_random_vectors(pc, N, block):
    import torch
    g = Grid(pc, two_phase_sphere(N, 0.35, 3))
    try:
        pc.pc_set_k(g.h, KAPPA)
        m = N ** 3 if block < 0 else N ** 3 // 4
        nvec = 3
        xs = complex_gaussian((nvec, 3, m), 40 + N + block)
        lam = np.array([1.5e7, 3.0e7, 7.0e7])
        w = np.array([0.7, -1.3, 2.1])
        dC = torch.zeros(21 * N ** 3, dtype=torch.float64, device="cuda")
        drho = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
        dC += 0.25  # the call accumulates
        pc.pc_eig_grad(g.h, block, torch.from_numpy(xs.reshape(-1)).cuda(), lam, w, dC, drho)
        torch.cuda.synchronize()
        full = xs if block < 0 else np.stack([O.inject(g.pb, block, xs[v]) for v in range(nvec)])
        refC, refr = _oracle_weighted(g, KAPPA, full, lam, w)
        gotC = dC.view(21, -1).T.cpu().numpy() - 0.25
        gotr = drho.cpu().numpy()
        assert np.abs(gotC - refC).max() <= 1e-12 * np.abs(refC).max()
        assert np.abs(gotr - refr).max() <= 1e-12 * np.abs(refr).max()
        if block >= 0:
            off = np.setdiff1d(np.arange(N ** 3), O.block_index(g.pb.dims, block))
            assert np.abs(gotC[off]).max() == 0.0 and np.abs(gotr[off]).max() == 0.0
    finally:
        g.close()


def test_grad_errors(pc):
    import torch
    g = Grid(pc, two_phase_sphere(8, 0.35, 3))
    try:
        x = torch.zeros(3 * 512, dtype=torch.complex128, device="cuda")
        d = torch.zeros(21 * 512, dtype=torch.float64, device="cuda")
        r = torch.zeros(512, dtype=torch.float64, device="cuda")
        with pytest.raises(pc.PcError):  # no Bloch vector set yet
            pc.pc_eig_grad(g.h, -1, x, [1.0], [1.0], d, r)
        pc.pc_set_k(g.h, KAPPA)
        with pytest.raises(pc.PcError):
            pc.pc_eig_grad(g.h, 4, x, [1.0], [1.0], d, r)
        with pytest.raises(pc.PcError):
            pc.pc_eig_grad(g.h, -1, x, [np.nan], [1.0], d, r)
        pc.pc_eig_grad(g.h, -1, x, [], [], d, r)  # nothing to do
    finally:
        g.close()


def _solver_gradients(pc, ad, g, kappa, nev, weights):
    opt = pc.pc_options_default(tol=1e-10, inner_tol=1e-12)
    return ad.nodewise_gradients(g.h, g.cell.N, kappa, nev, weights=weights, opt=opt)


def _oracle_merged(g, kappa, nev):
    """Dense eigenpairs of the four blocks merged: lowest nev eigenvalues (SI), full-space
    vectors, and for each its block and its rank inside the block."""
    vals, vecs, blk, rank = [], [], [], []
    for b in range(4):
        w, X = O.dense_eigpairs(g.pb, kappa, b)
        vals.append(w[:nev])
        vecs.append(X[:nev])
        blk += [b] * min(nev, w.size)
        rank += list(range(min(nev, w.size)))
    vals = np.concatenate(vals)
    order = np.argsort(vals, kind="stable")[:nev]
    return (vals[order] * g.to_si, np.concatenate(vecs)[order], np.asarray(blk)[order],
            np.asarray(rank)[order])


def test_solver_gradient_matches_dense_oracle_n8(pc, ad):
    g = Grid(pc, two_phase_sphere(8, 0.35, 1))
    try:
        nev = 8
        lam_ref, X, _, _ = _oracle_merged(g, KAPPA, nev)
        gaps = np.diff(lam_ref) / lam_ref[1:]
        assert gaps.min() > 1e-6  # generic Bloch vector: simple eigenvalues
        w = np.random.default_rng(5).standard_normal(nev)
        ev, dC, drho = _solver_gradients(pc, ad, g, KAPPA, nev, w)
        assert np.allclose(ev, lam_ref, rtol=1e-10, atol=0)
        refC, refr = _oracle_weighted(g, KAPPA, X, lam_ref, w)
        assert np.abs(dC - refC).max() <= 1e-7 * np.abs(refC).max()
        assert np.abs(drho - refr).max() <= 1e-7 * np.abs(refr).max()
    finally:
        g.close()


def test_euler_identities_per_band(pc, ad):
    g = Grid(pc, two_phase_sphere(8, 0.35, 2))
    try:
        nev = 6
        Cn = g.cell.node_C()[:, IU[0], IU[1]]
        rn = g.cell.node_rho()
        for v in range(nev):
            w = np.zeros(nev)
            w[v] = 1.0
            ev, dC, drho = _solver_gradients(pc, ad, g, KAPPA, nev, w)
            assert np.isclose(np.sum(dC * Cn), ev[v], rtol=1e-9)
            assert np.isclose(np.sum(drho * rn), -ev[v], rtol=1e-9)
    finally:
        g.close()


def test_degenerate_cluster_is_a_subspace(pc, ad):
    """Homogeneous isotropic medium along [100]: the transverse level is eightfold (two
    branches in each of the four blocks) and the longitudinal one fourfold.  With weights
    constant on each cluster the gradient does not depend on the basis the solver returned."""
    from workloads.materials import TwoPhaseCell
    N = 8
    C = isotropic_voigt(40e9, 30e9)
    cell = TwoPhaseCell(N=N, C=np.stack([C, C]), rho=np.array([2000.0, 2000.0]),
                        phase=np.zeros(N ** 3, np.uint8), theta=None, a_lat=np.eye(3))
    g = Grid(pc, cell)
    try:
        kappa = (0.125, 0.0, 0.0)
        nev = 12
        lam, X, _, _ = _oracle_merged(g, kappa, nev)
        assert np.allclose(lam[:8], lam[0], rtol=1e-9) and np.allclose(lam[8:], lam[8], rtol=1e-9)
        assert lam[8] > 2 * lam[0]
        w = np.array([1.0] * 8 + [-2.0] * 4)
        ev, dC, drho = _solver_gradients(pc, ad, g, kappa, nev, w)
        assert np.allclose(ev, lam, rtol=1e-10, atol=0)
        refC, refr = _oracle_weighted(g, kappa, X, lam, w)
        assert np.abs(dC - refC).max() <= 1e-7 * np.abs(refC).max()
        assert np.abs(drho - refr).max() <= 1e-7 * np.abs(refr).max()
        # unequal weights inside a cluster are replaced by the cluster mean
        w2 = np.array([2.0, 0.0] * 4 + [-2.0] * 4)
        _, dC2, drho2 = _solver_gradients(pc, ad, g, kappa, nev, w2)
        assert np.abs(dC2 - refC).max() <= 1e-7 * np.abs(refC).max()
    finally:
        g.close()


def test_fifty_directions_central_differences_n8(pc, ad):
    g = Grid(pc, two_phase_sphere(8, 0.35, 1))
    try:
        nev = 4
        w = np.random.default_rng(11).standard_normal(nev)
        ev, dC, drho = _solver_gradients(pc, ad, g, KAPPA, nev, w)
        lam, _, blocks, ranks = _oracle_merged(g, KAPPA, nev)
        assert np.allclose(ev, lam, rtol=1e-10, atol=0)
        Cn = g.cell.node_C() / g.C0
        rn = g.cell.node_rho() / g.rho0
        pb = g.pb
        rng = np.random.default_rng(2024)
        h = 1e-5
        worst = 0.0
        for _ in range(50):
            a = rng.standard_normal((pb.n, 6, 6))
            dCd = 0.5 * (a + np.transpose(a, (0, 2, 1))) * np.abs(Cn).max()
            drd = rng.standard_normal(pb.n) * rn.max()
            fd = 0.0
            for b in sorted(set(blocks.tolist())):
                sel = np.flatnonzero(blocks == b)
                lp = O.dense_eigvals(O.Problem(pb.dims, pb.ainv, pb.C, pb.rho, pb.theta,
                                               Cn + h * dCd, rn + h * drd), KAPPA, b)
                lm = O.dense_eigvals(O.Problem(pb.dims, pb.ainv, pb.C, pb.rho, pb.theta,
                                               Cn - h * dCd, rn - h * drd), KAPPA, b)
                for v in sel:
                    fd += w[v] * (lp[ranks[v]] - lm[ranks[v]]) / (2 * h) * g.to_si
            # analytic directional derivative in SI: (per Pa) x Pa and (per kg/m^3) x kg/m^3
            an = np.sum(dC * dCd[:, IU[0], IU[1]] * g.C0) + np.sum(drho * drd * g.rho0)
            worst = max(worst, abs(fd - an) / np.sum(np.abs(w) * ev))
        assert worst <= 1e-6, worst
    finally:
        g.close()


def _dyadic_theta(N, seed):
    """A smoothly graded inclusion fraction on multiples of 1/256 inside [1/16, 15/16]
    (exact in float32, so theta +- 2^-10 steps are exact on the device)."""
    cell = two_phase_sphere(N, 0.35, seed)
    t = cell.theta_f64()
    rng = np.random.default_rng(seed)
    t = 0.0625 + 0.875 * (0.8 * t + 0.2 * rng.random(t.size))
    return cell, np.round(t * 256) / 256


def test_theta_autograd_matches_gpu_differences(pc, ad):
    import torch
    N, nev = 8, 5
    cell, th = _dyadic_theta(N, 4)
    opt = pc.pc_options_default(tol=1e-10, inner_tol=1e-12)
    theta = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    lam = ad.band_eigenvalues(theta, N, cell.C, cell.rho, KAPPA, nev, a_lat=cell.a_lat, opt=opt)
    w = torch.tensor(np.random.default_rng(8).standard_normal(nev), dtype=torch.float64)
    (lam * w).sum().backward()
    grad = theta.grad.numpy()
    assert np.all(np.diff(lam.detach().numpy()) > 1e-6 * lam.detach().numpy()[1:])
    rng = np.random.default_rng(9)
    for _ in range(3):
        d = rng.integers(-4, 5, size=th.size) / 1024.0
        with torch.no_grad():
            lp = ad.band_eigenvalues(torch.tensor(th + d), N, cell.C, cell.rho, KAPPA, nev, cell.a_lat, opt)
            lm = ad.band_eigenvalues(torch.tensor(th - d), N, cell.C, cell.rho, KAPPA, nev, cell.a_lat, opt)
        fd = float(((lp - lm) * w).sum()) / 2.0
        an = float(np.dot(grad, d))
        assert abs(fd - an) <= 1e-4 * abs(an) + 1e-9 * float((lam.detach().abs() * w.abs()).sum()), (fd, an)


def test_band_gap_gradient_matches_gpu_differences(pc, ad):
    N = 8
    cell, th = _dyadic_theta(N, 6)
    kappas = [(0.0, 0.0, 0.25), (0.25, 0.25, 0.0), (0.5, 0.0, 0.0), (0.5, 0.5, 0.5)]
    opt = pc.pc_options_default(tol=1e-10, inner_tol=1e-12)
    lo = 2

    def gap_at(t):
        g = pc.pc_grid_create(N, cell.C, cell.rho, theta=t.astype(np.float32), a_lat=cell.a_lat)
        try:
            return ad.band_gap(g, N, kappas, lo, opt=opt)
        finally:
            pc.pc_grid_destroy(g)

    gap, dC, drho = gap_at(th)
    dCdt = (cell.C[1] - cell.C[0])[IU]
    gtheta = dC @ dCdt + drho * (cell.rho[1] - cell.rho[0])
    d = np.random.default_rng(12).integers(-4, 5, size=th.size) / 1024.0
    fd = (gap_at(th + d)[0] - gap_at(th - d)[0]) / 2.0
    an = float(np.dot(gtheta, d))
    assert abs(fd - an) <= 1e-3 * abs(an) + 1e-9 * gap, (fd, an)
