"""Differentiable band eigenvalues (torch.autograd) on top of the C ABI.

The forward pass solves the band problem on the GPU (``pc_eigs``); the
backward pass runs the library's adjoint kernel (``pc_eig_grad``), which
returns Hellmann-Feynman gradients of weighted eigenvalues with respect to
the nodewise stiffness (21 independent Voigt entries per node) and density.
Degenerate clusters are treated as subspaces: eigenvalues closer than a
relative ``cluster_tol`` share the mean of their incoming gradients, which is
the gradient of any symmetric function of the cluster (basis independent).

``NodewiseBandEigenvalues``, ``NodewiseBandStructure`` (several Bloch vectors, solved in
lockstep) and ``NodewiseBandGap`` take the nodewise material itself as their inputs: a (N^3, 21) tensor of the independent Voigt stiffness entries of every node
and a (N^3,) density tensor (the general pencil of Eq. discrete_GEP_main, solved on a grid
made by ``pc_grid_create_nodewise``); their gradients are the (N^3, 21) and (N^3,)
Hellmann-Feynman gradients.  ``BandEigenvalues`` differentiates with respect to the
sub-pixel inclusion fraction theta of every node (C_i = (1-theta_i) C0 + theta_i C1, rho
likewise), by the chain rule through the nodewise gradients.
"""

from __future__ import annotations

import numpy as np
import torch

from . import _lib as pc

IU = np.triu_indices(6)


def clusters(evals, cluster_tol=1e-9):
    """Groups of indices of numerically degenerate eigenvalues (ascending input)."""
    groups, cur = [], [0]
    for i in range(1, len(evals)):
        if abs(evals[i] - evals[i - 1]) <= cluster_tol * max(abs(evals[i]), 1e-300):
            cur.append(i)
        else:
            groups.append(cur)
            cur = [i]
    groups.append(cur)
    return groups


def subspace_weights(evals, grad_out, cluster_tol=1e-9):
    """Per-eigenvalue weights with each degenerate cluster sharing the mean of its gradients."""
    w = np.array(grad_out, dtype=np.float64).copy()
    for grp in clusters(evals, cluster_tol):
        if len(grp) > 1:
            w[grp] = w[grp].mean()
    return w


def nodewise_gradients(g, N, kappa, nev, weights=None, opt=None, sigma=float("nan"), cluster_tol=1e-9):
    """Eigenvalues at kappa and sum_v w_v d lambda_v / d(C_l, rho_l) on the grid g of size N.

    Returns (evals [nev] SI, dC [N^3, 21] per Pa, drho [N^3] per kg/m^3) as numpy
    arrays, full-grid node order, stiffness entries in ``IU`` order; ``weights``
    defaults to all ones (gradient of the sum).
    """
    n = N ** 3
    evecs = torch.empty(nev * 3 * n, dtype=torch.complex128, device="cuda")
    ev, _, _ = pc.pc_eigs(g, kappa, nev, sigma=sigma, opt=opt, evecs=evecs)
    w = np.ones(nev) if weights is None else subspace_weights(ev, weights, cluster_tol)
    dC = torch.zeros(21 * n, dtype=torch.float64, device="cuda")
    drho = torch.zeros(n, dtype=torch.float64, device="cuda")
    pc.pc_set_k(g, kappa)
    pc.pc_eig_grad(g, -1, evecs, ev, w, dC, drho)
    torch.cuda.synchronize()
    return ev, dC.view(21, n).T.cpu().numpy(), drho.cpu().numpy()


class BandEigenvalues(torch.autograd.Function):
    """lambda(theta): lowest ``nev`` non-zero eigenvalues (SI) at ``kappa`` as a function of the
    nodewise inclusion fraction theta (float64 tensor of N^3 entries in [0, 1], full-grid order;
    the grid stores it in float32)."""

    @staticmethod
    def forward(ctx, theta, N, C, rho, kappa, nev, a_lat=None, opt=None, cluster_tol=1e-9):
        th = theta.detach().to("cpu", torch.float32).numpy()
        g = pc.pc_grid_create(N, C, rho, theta=th, a_lat=a_lat)
        try:
            evecs = torch.empty(nev * 3 * N ** 3, dtype=torch.complex128, device="cuda")
            ev, _, _ = pc.pc_eigs(g, kappa, nev, opt=opt, evecs=evecs)
        except Exception:
            pc.pc_grid_destroy(g)
            raise
        ctx.g, ctx.N, ctx.evecs, ctx.ev, ctx.kappa = g, N, evecs, ev, kappa
        ctx.C, ctx.rho = np.asarray(C, dtype=np.float64), np.asarray(rho, dtype=np.float64)
        ctx.cluster_tol = cluster_tol
        return torch.as_tensor(ev, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        g, n = ctx.g, ctx.N ** 3
        try:
            w = subspace_weights(ctx.ev, grad_out.detach().cpu().numpy(), ctx.cluster_tol)
            dC = torch.zeros(21 * n, dtype=torch.float64, device="cuda")
            drho = torch.zeros(n, dtype=torch.float64, device="cuda")
            pc.pc_set_k(g, ctx.kappa)
            pc.pc_eig_grad(g, -1, ctx.evecs, ctx.ev, w, dC, drho)
            dCdt = torch.as_tensor((ctx.C[1] - ctx.C[0])[IU], dtype=torch.float64, device="cuda")
            grad_theta = dC.view(21, n).T @ dCdt + drho * float(ctx.rho[1] - ctx.rho[0])
        finally:
            pc.pc_grid_destroy(g)
            ctx.evecs = None
        return (grad_theta.to(grad_out.device),) + (None,) * 8


def band_eigenvalues(theta, N, C, rho, kappa, nev, a_lat=None, opt=None):
    """Differentiable lowest ``nev`` eigenvalues (SI) at ``kappa`` as a function of theta."""
    return BandEigenvalues.apply(theta, N, C, rho, kappa, nev, a_lat, opt)


def _solve_nodewise(C21, rho, N, kappa, nev, a_lat, opt):
    """Eigenvalues (numpy, SI) and M-normalised full-space eigenvectors (device complex128) of the
    nodewise material at kappa; the grid lives only for the solve."""
    g = pc.pc_grid_create_nodewise(N, C21, rho, a_lat=a_lat)
    try:
        evecs = torch.empty(nev * 3 * N ** 3, dtype=torch.complex128, device="cuda")
        ev, _, _ = pc.pc_eigs(g, kappa, nev, opt=opt, evecs=evecs)
    finally:
        pc.pc_grid_destroy(g)
    return ev, evecs


def _solve_nodewise_multi(C21, rho, N, kappas, nev, a_lat, opt):
    """Eigenvalues ([nk][nev] numpy, SI) and M-normalised full-space eigenvectors (a list of nk device
    complex128 tensors of nev * 3 N^3) of the nodewise material at several Bloch vectors, solved in
    lockstep chunks (pc_eigs_multi; one at a time where the grid's size needs the library FFT)."""
    ks = np.ascontiguousarray(np.asarray(kappas, dtype=np.float64).reshape(-1, 3))
    g = pc.pc_grid_create_nodewise(N, C21, rho, a_lat=a_lat)
    try:
        kb = pc.pc_eigs_multi_max(g)
        vn = nev * 3 * N ** 3
        evs, vecs = [], []
        for c in range(0, len(ks), kb):
            ch = ks[c:c + kb]
            buf = torch.empty(len(ch) * vn, dtype=torch.complex128, device="cuda")
            ev, _, _ = pc.pc_eigs_multi(g, ch, nev, opt=opt, evecs=buf)
            evs.append(ev)
            vecs += list(buf.view(len(ch), vn).unbind(0))
    finally:
        pc.pc_grid_destroy(g)
    return np.concatenate(evs, axis=0), vecs


def _adjoint(N, a_lat, kappa, evecs, ev, w):
    """sum_v w_v d lambda_v / d(C_l, rho_l) for full-space eigenvectors: (dC [N^3, 21], drho [N^3])
    device tensors.  The adjoint kernel reads the grid's geometry, units and Bloch vector only, so a
    grid of any material with the same N and lattice serves."""
    return _adjoint_many(N, a_lat, [(kappa, evecs, ev, w)])


def _adjoint_many(N, a_lat, terms):
    """The sum of _adjoint over terms (kappa, evecs, ev, w) on one scratch grid."""
    n = N ** 3
    C = np.stack([np.eye(6), np.eye(6)]) * 1e9
    g = pc.pc_grid_create(N, C, np.array([1e3, 1e3]), a_lat=a_lat)
    try:
        dC = torch.zeros(21 * n, dtype=torch.float64, device="cuda")
        drho = torch.zeros(n, dtype=torch.float64, device="cuda")
        for kappa, evecs, ev, w in terms:
            if not np.any(w):
                continue
            pc.pc_set_k(g, kappa)
            pc.pc_eig_grad(g, -1, evecs, ev, w, dC, drho)
    finally:
        pc.pc_grid_destroy(g)
    return dC.view(21, n).T, drho


class NodewiseBandEigenvalues(torch.autograd.Function):
    """lambda(C, rho): lowest ``nev`` non-zero eigenvalues (SI, ascending) at ``kappa`` as a function
    of the nodewise stiffness C21 (float64 (N^3, 21): entries C_l[p][r], p <= r, row order, Pa) and
    density rho (float64 (N^3,), kg/m^3), full-grid node order.  Backward: d lambda / d C21 (an
    off-diagonal entry stands for both C[p][r] and C[r][p]) and d lambda / d rho, with numerically
    degenerate eigenvalues treated as subspaces."""

    @staticmethod
    def forward(ctx, C21, rho, N, kappa, nev, a_lat=None, opt=None, cluster_tol=1e-9):
        ev, evecs = _solve_nodewise(C21.detach().cpu().numpy(), rho.detach().cpu().numpy(), N, kappa, nev, a_lat,
                                    opt)
        ctx.N, ctx.a_lat, ctx.kappa, ctx.ev, ctx.evecs, ctx.cluster_tol = N, a_lat, kappa, ev, evecs, cluster_tol
        return torch.as_tensor(ev, dtype=torch.float64, device=C21.device)

    @staticmethod
    def backward(ctx, grad_out):
        w = subspace_weights(ctx.ev, grad_out.detach().cpu().numpy(), ctx.cluster_tol)
        dC, drho = _adjoint(ctx.N, ctx.a_lat, ctx.kappa, ctx.evecs, ctx.ev, w)
        ctx.evecs = None
        dev = grad_out.device
        return (dC.to(dev), drho.to(dev)) + (None,) * 6


def band_eigenvalues_nodewise(C21, rho, N, kappa, nev, a_lat=None, opt=None):
    """Differentiable lowest ``nev`` eigenvalues (SI) at ``kappa`` of the nodewise material (C21, rho)."""
    return NodewiseBandEigenvalues.apply(C21, rho, N, kappa, nev, a_lat, opt)


class NodewiseBandGap(torch.autograd.Function):
    """Width (Hz) of the gap above band ``lo`` (0-based) over a set of Bloch vectors,
    min_k f_{lo+1}(k) - max_k f_lo(k) with f = sqrt(lambda) / (2 pi), as a function of the nodewise
    material (C21, rho) (as ``NodewiseBandEigenvalues``).  Backward: through the two active Bloch
    vectors (the minimiser and the maximiser) with d f / d lambda = 1 / (8 pi^2 f); a band that is
    degenerate there is treated as a subspace (one more band is solved to see its cluster)."""

    @staticmethod
    def forward(ctx, C21, rho, N, kappas, lo, a_lat=None, opt=None, cluster_tol=1e-9):
        hi, nev = lo + 1, lo + 3
        Cn, rn = C21.detach().cpu().numpy(), rho.detach().cpu().numpy()
        evs, vecs = _solve_nodewise_multi(Cn, rn, N, kappas, nev, a_lat, opt)  # all Bloch vectors in lockstep
        f = np.sqrt(evs) / (2 * np.pi)
        it, ib = int(np.argmin(f[:, hi])), int(np.argmax(f[:, lo]))
        # keep only the two active Bloch vectors' eigenvectors (copies: the rest can be freed)
        top = (f[it, hi], kappas[it], evs[it], vecs[it].clone())
        bot = (f[ib, lo], kappas[ib], evs[ib], vecs[ib].clone() if ib != it else top[3])
        del vecs
        ctx.N, ctx.a_lat, ctx.lo, ctx.top, ctx.bot, ctx.cluster_tol = N, a_lat, lo, top, bot, cluster_tol
        return torch.as_tensor(top[0] - bot[0], dtype=torch.float64, device=C21.device)

    @staticmethod
    def backward(ctx, grad_out):
        g = float(grad_out.detach().cpu())
        n = ctx.N ** 3
        dC = torch.zeros((n, 21), dtype=torch.float64, device="cuda")
        drho = torch.zeros(n, dtype=torch.float64, device="cuda")
        for sign, band, (fval, k, ev, evecs) in ((1.0, ctx.lo + 1, ctx.top), (-1.0, ctx.lo, ctx.bot)):
            w = np.zeros(len(ev))
            w[band] = g * sign / (8 * np.pi ** 2 * fval)
            w = subspace_weights(ev, w, ctx.cluster_tol)
            dc, dr = _adjoint(ctx.N, ctx.a_lat, k, evecs, ev, w)
            dC += dc
            drho += dr
        ctx.top = ctx.bot = None
        dev = grad_out.device
        return (dC.to(dev), drho.to(dev)) + (None,) * 6


class NodewiseBandStructure(torch.autograd.Function):
    """lambda(C, rho) at several Bloch vectors: the lowest ``nev`` non-zero eigenvalues (SI) at each
    of ``kappas`` ([nk, nev]), as a function of the nodewise material (as
    ``NodewiseBandEigenvalues``); the forward solves all Bloch vectors in lockstep
    (pc_eigs_multi), the backward sums the adjoint over them, with numerically degenerate
    eigenvalues treated as subspaces at each Bloch vector."""

    @staticmethod
    def forward(ctx, C21, rho, N, kappas, nev, a_lat=None, opt=None, cluster_tol=1e-9):
        evs, vecs = _solve_nodewise_multi(C21.detach().cpu().numpy(), rho.detach().cpu().numpy(), N, kappas, nev,
                                          a_lat, opt)
        ctx.N, ctx.a_lat, ctx.kappas, ctx.evs, ctx.vecs, ctx.cluster_tol = N, a_lat, kappas, evs, vecs, cluster_tol
        return torch.as_tensor(evs, dtype=torch.float64, device=C21.device)

    @staticmethod
    def backward(ctx, grad_out):
        go = grad_out.detach().cpu().numpy()
        terms = [(k, ctx.vecs[i], ctx.evs[i], subspace_weights(ctx.evs[i], go[i], ctx.cluster_tol))
                 for i, k in enumerate(ctx.kappas)]
        dC, drho = _adjoint_many(ctx.N, ctx.a_lat, terms)
        ctx.vecs = None
        dev = grad_out.device
        return (dC.to(dev), drho.to(dev)) + (None,) * 6


def band_structure_nodewise(C21, rho, N, kappas, nev, a_lat=None, opt=None):
    """Differentiable lowest ``nev`` eigenvalues (SI) at every Bloch vector of ``kappas`` ([nk, nev])
    of the nodewise material (C21, rho), the Bloch vectors solved in lockstep."""
    return NodewiseBandStructure.apply(C21, rho, N, kappas, nev, a_lat, opt)


def band_gap_nodewise(C21, rho, N, kappas, lo, a_lat=None, opt=None):
    """Differentiable width (Hz) of the gap above band ``lo`` over ``kappas`` of the nodewise material."""
    return NodewiseBandGap.apply(C21, rho, N, kappas, lo, a_lat, opt)


def two_phase_nodewise(cell):
    """(C21 (N^3, 21), rho (N^3,)) numpy arrays of a two-phase cell's nodewise material (phase ids or
    inclusion fractions, Eq. subpixel_material_average)."""
    th = cell.theta_f64()
    C = np.asarray(cell.C, dtype=np.float64)
    C21 = (1.0 - th)[:, None] * C[0][IU][None, :] + th[:, None] * C[1][IU][None, :]
    rho = (1.0 - th) * float(cell.rho[0]) + th * float(cell.rho[1])
    return C21, rho


def band_gap(g, N, kappas, lo, opt=None):
    """Width (Hz) of the gap above band ``lo`` (0-based) over a set of Bloch vectors,
    min_k f_{lo+1} - max_k f_lo with f = sqrt(lambda) / (2 pi), and its nodewise gradient
    (dC [N^3, 21], drho [N^3]) taken through the two active k-points."""
    hi, nev = lo + 1, lo + 2
    top, bot = None, None
    for k in kappas:
        ev, _, _ = pc.pc_eigs(g, k, nev, opt=opt)
        f = np.sqrt(ev) / (2 * np.pi)
        if top is None or f[hi] < top[0]:
            top = (f[hi], k)
        if bot is None or f[lo] > bot[0]:
            bot = (f[lo], k)
    n = N ** 3
    dC, drho = np.zeros((n, 21)), np.zeros(n)
    for sign, band, (fval, k) in ((1.0, hi, top), (-1.0, lo, bot)):
        w = np.zeros(nev)
        w[band] = sign / (8 * np.pi ** 2 * fval)  # d f / d lambda = 1 / (8 pi^2 f)
        _, dc, dr = nodewise_gradients(g, N, k, nev, weights=w, opt=opt)
        dC += dc
        drho += dr
    return top[0] - bot[0], dC, drho
