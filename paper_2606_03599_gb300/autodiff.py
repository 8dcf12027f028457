"""Differentiable band eigenvalues (torch.autograd) on top of the C ABI.

The forward pass solves the band problem on the GPU (``pc_eigs``); the
backward pass runs the library's adjoint kernel (``pc_eig_grad``), which
returns Hellmann-Feynman gradients of weighted eigenvalues with respect to
the nodewise stiffness (21 independent Voigt entries per node) and density.
Degenerate clusters are treated as subspaces: eigenvalues closer than a
relative ``cluster_tol`` share the mean of their incoming gradients, which is
the gradient of any symmetric function of the cluster (basis independent).

``BandEigenvalues`` differentiates with respect to the sub-pixel inclusion
fraction theta of every node (C_i = (1-theta_i) C0 + theta_i C1, rho likewise),
by the chain rule through the nodewise gradients.
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
