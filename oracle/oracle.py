"""FP64 CPU oracle: the plain definitions the GPU path must reproduce.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Units are whatever the
caller passes: the oracle evaluates the definitions for the given stiffness,
density and lattice basis.

Pins (tests under ``tests/test_oracle_*.py``, marker ``not gpu``):

* apply (C matrix-free and sparse): plane-wave identity against the Fourier
  symbol of Sec. 5.3 (Eqs. Sd_phase_maintext, delta1-3_xi_unified,
  Bhat_xi_m_def), long-wave Christoffel velocities (textbook elastodynamics),
  Hermiticity, positivity, adjointness of strain/divergence, Theorem 4.1
  commutation, Bloch symmetries, Gamma zero-mode count (App. C);
* index maps: brute force against the projector of Eq. Proj_sigma;
* block reduction: merged dense block spectra equal the dense full spectrum
  (Cor. 4.2), off-block couplings exactly zero;
* block Fourier basis: dense T_sigma = T F_sigma (Eqs. f_sigma_unified,
  Tsigma_unified) against the separable forms (both directions), unitarity;
* reference-medium preconditioner: for a homogeneous medium it is the exact
  inverse of the shifted block operator evaluated by the C apply (independent of
  the symbols and transforms); the weighted SVD satisfies
  Eq. weighted_svd_local_unified for any Hermitian positive definite Psi;
* eigen oracles: dense LAPACK, homogeneous closed form, ARPACK shift-invert.
"""

from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import tempfile

import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import sparse_ops as so

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_oracle_c.so")
_SRC = os.path.join(_HERE, "oracle_apply.c")
_lib = None

STEPS = np.array([[1, 1, 1], [1, 1, -1], [1, -1, 1], [1, -1, -1]])
BPAT = np.array([[0, -1, -1, -1, 2, 1], [-1, 1, -1, 2, -1, 0], [-1, -1, 2, 1, 0, -1]])


# --------------------------------------------------------------------------- build / load
def build_c(force: bool = False) -> str:
    """Compile ``oracle_apply.c`` with gcc into ``_oracle_c.so`` (portable flags, OpenMP)."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build_c()
        lib = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        ci = ctypes.c_int
        lib.oracle_strain.argtypes = [ci, ci, ci, dp, dp, dp, dp, ci]
        lib.oracle_divergence.argtypes = [ci, ci, ci, dp, dp, dp, dp, ci]
        lib.oracle_apply_full.argtypes = [ci, ci, ci, dp, dp, dp, dp, dp, dp, dp,
                                          ctypes.c_double, ci]
        lib.oracle_apply_nodes.argtypes = [ci, ci, ci, dp, dp, dp, dp, dp, dp, i64p,
                                           ctypes.c_int64, dp, ctypes.c_double, ci]
        for f in (lib.oracle_strain, lib.oracle_divergence, lib.oracle_apply_full,
                  lib.oracle_apply_nodes):
            f.restype = ci
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# --------------------------------------------------------------------------- problem data
@dataclasses.dataclass
class Problem:
    """Discrete two-phase problem: dims (n1,n2,n3), A_lat^-1, phase tables, per-node theta."""

    dims: tuple
    ainv: np.ndarray  # (3,3): ainv[s, m] = (A_lat^-1)_{s m}
    C: np.ndarray  # (2,6,6)
    rho: np.ndarray  # (2,)
    theta: np.ndarray  # (n,) float64 in [0,1]
    C_nodes: np.ndarray | None = None  # optional (n,6,6) nodewise stiffness replacing the two-phase rule
    rho_nodes: np.ndarray | None = None  # optional (n,) nodewise density

    @property
    def n(self):
        return int(np.prod(self.dims))

    def node_C(self):
        if self.C_nodes is not None:
            return self.C_nodes
        t = self.theta[:, None, None]
        return (1.0 - t) * self.C[0][None] + t * self.C[1][None]

    def node_rho(self):
        if self.rho_nodes is not None:
            return self.rho_nodes
        return (1.0 - self.theta) * self.rho[0] + self.theta * self.rho[1]


def problem_from_cell(cell, C0: float = 1.0, rho0: float = 1.0, L: float = 1.0) -> Problem:
    """Problem in units C/C0, rho/rho0, lengths/L from a ``workloads.TwoPhaseCell``."""
    theta = cell.theta_f64()
    a_lat = np.asarray(cell.a_lat, dtype=np.float64) / L
    return Problem(dims=(cell.N,) * 3, ainv=np.linalg.inv(a_lat), C=np.asarray(cell.C) / C0,
                   rho=np.asarray(cell.rho, dtype=np.float64) / rho0, theta=theta)


def homogeneous_problem(N, C, rho, a_lat=None) -> Problem:
    a_lat = np.eye(3) if a_lat is None else np.asarray(a_lat, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    return Problem(dims=(N,) * 3, ainv=np.linalg.inv(a_lat), C=np.stack([C, C]),
                   rho=np.array([rho, rho], dtype=np.float64), theta=np.zeros(N ** 3))


def phases(kappa) -> np.ndarray:
    """phi_l = 2 pi kappa_l (Eq. phi_def)."""
    return 2.0 * np.pi * np.asarray(kappa, dtype=np.float64)


# --------------------------------------------------------------------------- matrix-free apply (C)
def _c_args(pb: Problem, kappa):
    ainv = np.ascontiguousarray(pb.ainv, dtype=np.float64)
    phi = np.ascontiguousarray(phases(kappa))
    Ctab = np.ascontiguousarray(pb.C.reshape(2, 36), dtype=np.float64)
    rho = np.ascontiguousarray(pb.rho, dtype=np.float64)
    theta = np.ascontiguousarray(pb.theta, dtype=np.float64)
    return ainv, phi, Ctab, rho, theta


def apply_full(pb: Problem, kappa, x, shift: float = 0.0, nthreads: int = 0) -> np.ndarray:
    """y = (A_h - shift M_h) x on the full grid; x, y are (3, n) complex128."""
    lib = _load()
    x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128).reshape(3, pb.n))
    y = np.empty_like(x)
    ainv, phi, Ctab, rho, theta = _c_args(pb, kappa)
    n1, n2, n3 = pb.dims
    rc = lib.oracle_apply_full(n1, n2, n3, _dp(ainv), _dp(phi), _dp(Ctab), _dp(rho), _dp(theta),
                               _dp(x), _dp(y), float(shift), int(nthreads))
    if rc != 0:
        raise MemoryError("oracle_apply_full failed (%d)" % rc)
    return y


def strain_full(pb: Problem, kappa, x, nthreads: int = 0) -> np.ndarray:
    """e = B_h^H x, (3, n) -> (6, n)."""
    lib = _load()
    x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128).reshape(3, pb.n))
    e = np.empty((6, pb.n), dtype=np.complex128)
    ainv, phi, *_ = _c_args(pb, kappa)
    n1, n2, n3 = pb.dims
    lib.oracle_strain(n1, n2, n3, _dp(ainv), _dp(phi), _dp(x), _dp(e), int(nthreads))
    return e


def divergence_full(pb: Problem, kappa, tau, nthreads: int = 0) -> np.ndarray:
    """y = B_h tau, (6, n) -> (3, n)."""
    lib = _load()
    tau = np.ascontiguousarray(np.asarray(tau, dtype=np.complex128).reshape(6, pb.n))
    y = np.empty((3, pb.n), dtype=np.complex128)
    ainv, phi, *_ = _c_args(pb, kappa)
    n1, n2, n3 = pb.dims
    lib.oracle_divergence(n1, n2, n3, _dp(ainv), _dp(phi), _dp(tau), _dp(y), int(nthreads))
    return y


def apply_at_nodes(pb: Problem, kappa, x, nodes, shift: float = 0.0, nthreads: int = 0):
    """((A_h - shift M_h) x) at the listed full-grid nodes only: returns (count, 3)."""
    lib = _load()
    x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128).reshape(3, pb.n))
    nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.int64))
    out = np.empty((nodes.size, 3), dtype=np.complex128)
    ainv, phi, Ctab, rho, theta = _c_args(pb, kappa)
    n1, n2, n3 = pb.dims
    lib.oracle_apply_nodes(n1, n2, n3, _dp(ainv), _dp(phi), _dp(Ctab), _dp(rho), _dp(theta),
                           _dp(x), nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                           nodes.size, _dp(out), float(shift), int(nthreads))
    return out


# --------------------------------------------------------------------------- parity blocks (Sec. 4)
def block_of_node(dims) -> np.ndarray:
    """Block label b = 2 p12 + p13 of every node, read off the projectors of Eq. Proj_sigma."""
    n = int(np.prod(dims))
    lab = np.full(n, -1, dtype=np.int64)
    for b in range(4):
        d = so.projector_diag(dims, b)
        lab[d > 0.5] = b
    return lab


def block_index(dims, b: int) -> np.ndarray:
    """Full node of block position t: the block's nodes in ascending full linear index."""
    return so.block_nodes(dims, b)


def inject(pb: Problem, b: int, xb) -> np.ndarray:
    """Q_sigma y: block vector (3, n_b) -> full (3, n), zero off the block."""
    idx = block_index(pb.dims, b)
    x = np.zeros((3, pb.n), dtype=np.complex128)
    x[:, idx] = np.asarray(xb).reshape(3, idx.size)
    return x


def extract(pb: Problem, b: int, x) -> np.ndarray:
    """Q_sigma^T x: full (3, n) -> block (3, n_b)."""
    idx = block_index(pb.dims, b)
    return np.asarray(x).reshape(3, pb.n)[:, idx]


def apply_block(pb: Problem, kappa, b: int, xb, shift: float = 0.0, nthreads: int = 0):
    """(A_sigma - shift M_sigma) y via inject -> full apply -> extract (Eq. Asigma_main)."""
    return extract(pb, b, apply_full(pb, kappa, inject(pb, b, xb), shift, nthreads))


def apply_block_at(pb: Problem, kappa, b: int, xb, ts, shift: float = 0.0, nthreads: int = 0):
    """Sampled block apply: rows t of (A_sigma - shift M_sigma) y, returns (len(ts), 3)."""
    idx = block_index(pb.dims, b)
    return apply_at_nodes(pb, kappa, inject(pb, b, xb), idx[np.asarray(ts)], shift, nthreads)


# --------------------------------------------------------------------------- sparse / dense pencils
def sparse_pencil(pb: Problem, kappa, b=None):
    """(A, M) as scipy.sparse matrices: full space, or block b via Q_sigma^* A Q_sigma (Eq. Asigma_main)."""
    A = so.A_matrix(pb.dims, phases(kappa), pb.ainv, pb.node_C())
    M = so.M_matrix(pb.node_rho())
    if b is None:
        return A, M
    Q = so.Q_matrix(pb.dims, b)
    return (Q.conj().T @ A @ Q).tocsr(), (Q.conj().T @ M @ Q).tocsr()


def dense_eigvals(pb: Problem, kappa, b=None) -> np.ndarray:
    """All generalized eigenvalues of (A, M), ascending (LAPACK zhegvd via scipy.linalg.eigh)."""
    A, M = sparse_pencil(pb, kappa, b)
    Ad = A.toarray()
    Ad = 0.5 * (Ad + Ad.conj().T)
    return scipy.linalg.eigh(Ad, M.toarray(), eigvals_only=True)


def dense_eigpairs(pb: Problem, kappa, b=None):
    """All eigenpairs of (A, M) (scipy.linalg.eigh): ascending values and M-normalised vectors as
    full-space (count, 3, n) arrays (block vectors injected with Q_sigma)."""
    A, M = sparse_pencil(pb, kappa, b)
    Ad = A.toarray()
    Ad = 0.5 * (Ad + Ad.conj().T)
    w, Z = scipy.linalg.eigh(Ad, M.toarray())
    if b is None:
        X = Z.T.reshape(-1, 3, pb.n)
    else:
        X = np.stack([inject(pb, b, Z[:, j]) for j in range(Z.shape[1])])
    return w, X


def zero_mode_count(evals, rel: float = 1e-9) -> int:
    """#{lambda : |lambda| < rel * max|lambda|} (the Gamma zero-derivative modes, App. C)."""
    ev = np.asarray(evals)
    return int(np.sum(np.abs(ev) < rel * np.max(np.abs(ev))))


def lowest_nonzero(evals, nev: int, rel: float = 1e-9) -> np.ndarray:
    """Lowest nev eigenvalues after removing the zero-derivative modes (Sec. 6.2 post-processing)."""
    ev = np.sort(np.asarray(evals))
    keep = ev[np.abs(ev) >= rel * np.max(np.abs(ev))]
    return keep[:nev]


# --------------------------------------------------------------------------- Fourier symbols (Sec. 5)
def bloch_freqs(dims, kappa):
    """alpha_p, beta_q, gamma_r = (phi_l + 2 pi p) / n_l (Sec. 4, Sec. 5.1)."""
    phi = phases(kappa)
    return [(phi[l] + 2.0 * np.pi * np.arange(dims[l])) / dims[l] for l in range(3)]


def shift_symbols(dims, kappa, p, q, r) -> np.ndarray:
    """Symbols of S_d1..S_d4 at mode (p,q,r): exp(i(alpha +- beta +- gamma)) (Eq. Sd_phase_maintext)."""
    al, be, ga = bloch_freqs(dims, kappa)
    a, bb, g = al[p], be[q], ga[r]
    return np.array([np.exp(1j * (a + bb + g)), np.exp(1j * (a + bb - g)),
                     np.exp(1j * (a - bb + g)), np.exp(1j * (a - bb - g))])


def symbol_block(dims, kappa, ainv, p, q, r) -> np.ndarray:
    """3x6 symbol B_hat(m) (Eqs. delta1-3_xi_unified, Bhat_xi_m_def).

    d_l = (s_l - 1)/h_d, delta_s = c_s * sum_l c_{s l} d_l, eta in Cartesian
    axes: eta_m = sum_s (A_lat^-1)_{s m} (-i delta_s) (equals the paper's
    eta_j = -i delta_j when A_lat = I).
    """
    h = np.array([1.0 / m for m in dims])
    hd = np.sqrt(np.sum(h ** 2))
    s = shift_symbols(dims, kappa, p, q, r)
    d = (s - 1.0) / hd
    delta = np.array([hd / (4.0 * h[t]) * np.dot(so.C_SIGNS[t], d) for t in range(3)])
    eta = np.array([np.sum(ainv[:, m] * (-1j * delta)) for m in range(3)])
    e1, e2, e3 = eta
    return np.array([[e1, 0, 0, 0, e3, e2],
                     [0, e2, 0, e3, 0, e1],
                     [0, 0, e3, e2, e1, 0]], dtype=np.complex128)


def plane_wave(dims, kappa, p, q, r) -> np.ndarray:
    """psi_pqr(i,j,k) = n^-1/2 exp(i(i alpha_p + j beta_q + k gamma_r)) (Eq. psi_pqr_unified), full order."""
    al, be, ga = bloch_freqs(dims, kappa)
    n1, n2, n3 = dims
    k, j, i = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    psi = np.exp(1j * (i * al[p] + j * be[q] + k * ga[r])) / np.sqrt(n1 * n2 * n3)
    return psi.reshape(-1)


def homogeneous_spectrum(dims, kappa, ainv, C, rho) -> np.ndarray:
    """Closed-form spectrum of a homogeneous medium: union over all modes of eig(B_hat C B_hat^H)/rho."""
    out = []
    for r in range(dims[2]):
        for q in range(dims[1]):
            for p in range(dims[0]):
                Bh = symbol_block(dims, kappa, ainv, p, q, r)
                S = Bh @ C @ Bh.conj().T
                out.append(np.linalg.eigvalsh(0.5 * (S + S.conj().T)) / rho)
    return np.sort(np.concatenate(out))


def homogeneous_spectrum_planes(dims, kappa, ainv, C, rho) -> np.ndarray:
    """``homogeneous_spectrum`` evaluated one r-plane of modes at a time with array operations,
    for grids where a loop over every mode is too slow.  The symbol is the one of
    ``symbol_block`` (Eqs. Sd_phase_maintext, delta1-3_xi_unified, Bhat_xi_m_def) on arrays:
    s_l = exp(i(alpha +- beta +- gamma)), d_l = (s_l - 1)/h_d,
    delta_s = h_d/(4 h_s) sum_l c_{s l} d_l, eta_m = sum_s (A_lat^-1)_{s m} (-i delta_s)."""
    n1, n2, n3 = dims
    h = np.array([1.0 / m for m in dims])
    hd = np.sqrt(np.sum(h ** 2))
    al, be, ga = bloch_freqs(dims, kappa)
    a, bb = al[None, :], be[:, None]  # (q, p) plane of modes
    C = np.asarray(C, dtype=np.float64)
    out = []
    for r in range(n3):
        g = ga[r]
        s = np.stack([np.exp(1j * (a + bb + g)), np.exp(1j * (a + bb - g)),
                      np.exp(1j * (a - bb + g)), np.exp(1j * (a - bb - g))])
        d = (s - 1.0) / hd
        delta = np.stack([hd / (4.0 * h[t]) * np.tensordot(so.C_SIGNS[t], d, axes=(0, 0)) for t in range(3)])
        eta = np.tensordot(np.asarray(ainv).T, -1j * delta, axes=(1, 0))  # eta[m] = sum_s ainv[s, m] (-i delta[s])
        e1, e2, e3 = eta
        Bh = np.zeros((n2, n1, 3, 6), dtype=np.complex128)
        Bh[..., 0, 0], Bh[..., 0, 4], Bh[..., 0, 5] = e1, e3, e2
        Bh[..., 1, 1], Bh[..., 1, 3], Bh[..., 1, 5] = e2, e3, e1
        Bh[..., 2, 2], Bh[..., 2, 3], Bh[..., 2, 4] = e3, e2, e1
        S = Bh @ C @ np.conj(np.swapaxes(Bh, -1, -2))
        out.append(np.linalg.eigvalsh(0.5 * (S + np.conj(np.swapaxes(S, -1, -2)))).reshape(-1) / rho)
    return np.sort(np.concatenate(out))


# --------------------------------------------------------------------------- block Fourier basis (Sec. 5.2)
def representatives(dims):
    """Representative set R = {p < n1/2, q < n2/2, all r} of the half-period orbits (Eq. orbit_unified)."""
    n1, n2, n3 = dims
    return [(p, q, r) for r in range(n3) for q in range(n2 // 2) for p in range(n1 // 2)]


def T_sigma_dense(dims, kappa, b: int) -> np.ndarray:
    """Block Fourier basis T_sigma = T F_sigma restricted to block rows, n_b x n_b (Eqs. f_sigma_unified, Tsigma_unified).

    Column order: representatives in the order of ``representatives`` (p fastest).
    """
    n1, n2, n3 = dims
    s12, s13 = so.block_signs(b)
    h12, h13 = (n1 // 2, n2 // 2, 0), (n1 // 2, 0, n3 // 2)
    h23 = (0, n2 // 2, n3 // 2)  # h12 + h13 modulo the grid
    rows = block_index(dims, b)
    cols = []
    for (p, q, r) in representatives(dims):
        f = plane_wave(dims, kappa, p, q, r)
        f = f + s12 * plane_wave(dims, kappa, (p + h12[0]) % n1, (q + h12[1]) % n2, (r + h12[2]) % n3)
        f = f + s13 * plane_wave(dims, kappa, (p + h13[0]) % n1, (q + h13[1]) % n2, (r + h13[2]) % n3)
        f = f + s12 * s13 * plane_wave(dims, kappa, (p + h23[0]) % n1, (q + h23[1]) % n2,
                                       (r + h23[2]) % n3)
        cols.append(0.5 * f[rows])
    return np.stack(cols, axis=1)


def block_fourier_separable(w_compact, dims, kappa, b: int) -> np.ndarray:
    """T_sigma^H w for a block field w in quarter-grid order, by separable Bloch DFTs.

    w_compact: (n3, n2/2, n1/2) array (k slowest, i' fastest) of the block's
    nodes; node (i', j'', k) sits at i = 2 i' + ((k + p13) mod 2),
    j = 2 j'' + ((k + p12 + p13) mod 2).  Output: (n3, n2/2, n1/2) indexed
    (r, q, p) with p < n1/2, q < n2/2 (the representative set).

    Derived from Eq. psi_pqr_unified and Eq. Tsigma_unified: T_sigma^H w equals
    2 (T^H w) on the representatives for w supported on the block.
    """
    n1, n2, n3 = dims
    X, Y = n1 // 2, n2 // 2
    p12, p13 = b >> 1, b & 1
    al, be, ga = bloch_freqs(dims, kappa)
    ip = np.arange(X)
    jp = np.arange(Y)
    out = np.zeros((n3, Y, X), dtype=np.complex128)
    for k in range(n3):
        i0 = (k + p13) % 2
        j0 = (k + p12 + p13) % 2
        # sum over i', j'' with exp(-i (i alpha_p + j beta_q)) for p < X, q < Y
        Ei = np.exp(-1j * np.outer(al[:X], 2 * ip + i0))  # (p, i')
        Ej = np.exp(-1j * np.outer(be[:Y], 2 * jp + j0))  # (q, j'')
        plane = Ej @ w_compact[k] @ Ei.T  # (q, p)
        out += np.exp(-1j * k * ga)[:, None, None] * plane[None, :, :]
    return out * (2.0 / np.sqrt(n1 * n2 * n3))


def block_fourier_separable_inverse(what, dims, kappa, b: int) -> np.ndarray:
    """T_sigma what for mode coefficients on the representatives, by separable Bloch sums.

    what: (n3, n2/2, n1/2) indexed (r, q, p); output (n3, n2/2, n1/2) in quarter-grid order
    (k, j'', i').  Column m of T_sigma on the block is 2 n^-1/2 exp(i(i alpha_p + j beta_q +
    k gamma_r)) (Eqs. psi_pqr_unified, Tsigma_unified), so
    w(i', j'', k) = 2 n^-1/2 sum_{p,q,r} what(r,q,p) exp(i(i alpha_p + j beta_q + k gamma_r)).
    """
    n1, n2, n3 = dims
    X, Y = n1 // 2, n2 // 2
    p12, p13 = b >> 1, b & 1
    al, be, ga = bloch_freqs(dims, kappa)
    what = np.asarray(what, dtype=np.complex128).reshape(n3, Y, X)
    ip = np.arange(X)
    jp = np.arange(Y)
    out = np.empty((n3, Y, X), dtype=np.complex128)
    for k in range(n3):
        i0 = (k + p13) % 2
        j0 = (k + p12 + p13) % 2
        S = np.tensordot(np.exp(1j * k * ga), what, axes=(0, 0))  # (q, p): sum over r
        Ei = np.exp(1j * np.outer(al[:X], 2 * ip + i0))  # (p, i')
        Ej = np.exp(1j * np.outer(be[:Y], 2 * jp + j0))  # (q, j'')
        out[k] = Ej.T @ S @ Ei
    return out * (2.0 / np.sqrt(n1 * n2 * n3))


# --------------------------------------------------------------------------- reference-medium preconditioner (Sec. 5.4)
def weighted_svd(Bh, Psi):
    """Psi-weighted local SVD of a 3x6 symbol block (Eq. weighted_svd_unified).

    SVD of B_hat Psi^-1/2 = P Sigma Q~^H; Q = Psi^-1/2 Q~ and Q^{H,Psi} = Q^H Psi, so that
    B_hat = P Sigma Q^{H,Psi} and Q^{H,Psi} Q = I (Eq. weighted_svd_local_unified).
    Returns (P (3x3), sigma (3,), Q (6x3), Q^{H,Psi} (3x6)).
    """
    Psi = np.asarray(Psi, dtype=np.complex128)
    w, V = np.linalg.eigh(0.5 * (Psi + Psi.conj().T))
    Psi_mhalf = (V * (1.0 / np.sqrt(w))) @ V.conj().T
    P, sig, Qt_h = np.linalg.svd(np.asarray(Bh) @ Psi_mhalf, full_matrices=False)
    Q = Psi_mhalf @ Qt_h.conj().T
    return P, sig, Q, Q.conj().T @ Psi


def reference_medium(pb: Problem):
    """Constant reference material: the volume averages of the nodal stiffness and density
    (for the two-phase rule C_i = (1 - theta_i) C0 + theta_i C1, the rule at the mean theta)."""
    if pb.C_nodes is None and pb.rho_nodes is None:
        t = float(np.mean(pb.theta))
        return (1.0 - t) * pb.C[0] + t * pb.C[1], float((1.0 - t) * pb.rho[0] + t * pb.rho[1])
    return pb.node_C().mean(axis=0), float(pb.node_rho().mean())


def precond_mode_factor(pb: Problem, kappa, sigma: float, p, q, r, C_ref, rho_ref) -> np.ndarray:
    """F(m) = (B_hat(m) C_ref B_hat(m)^H - sigma rho_ref I_3)^-1 at mode m = (p, q, r).

    Formed from the weighted SVD with Psi = C_ref^-1 (Eq. weighted_svd_unified):
    B_hat C_ref^(1/2) = P Sigma Q~^H gives B_hat C_ref B_hat^H = P Sigma^2 P^H, hence
    F(m) = P (Sigma^2 - sigma rho_ref)^-1 P^H.
    """
    Psi = np.linalg.inv(np.asarray(C_ref, dtype=np.float64))
    P, sig, _, _ = weighted_svd(symbol_block(pb.dims, kappa, pb.ainv, p, q, r), Psi)
    return (P * (1.0 / (sig ** 2 - sigma * rho_ref))) @ P.conj().T


def block_mode_vector(dims, kappa, b: int, p, q, r) -> np.ndarray:
    """Column m = (p, q, r) of T_sigma at every node of block b (quarter-grid order):
    2 n^-1/2 exp(i(i alpha_p + j beta_q + k gamma_r)) (Eqs. psi_pqr_unified, Tsigma_unified)."""
    n1, n2, n3 = dims
    al, be, ga = bloch_freqs(dims, kappa)
    l = block_index(dims, b)
    i, j, k = l % n1, (l // n1) % n2, l // (n1 * n2)
    return np.exp(1j * (i * al[p] + j * be[q] + k * ga[r])) * (2.0 / np.sqrt(n1 * n2 * n3))


def precond_block(pb: Problem, kappa, b: int, sigma: float, r, C_ref=None, rho_ref=None) -> np.ndarray:
    """z = T_sigma diag_m F(m) T_sigma^H r on block b (Sec. 5.4 with a constant reference material),
    F(m) of ``precond_mode_factor`` for every representative mode m.
    r: block vector (3, n_b) in quarter-grid order; C_ref, rho_ref default to the volume averages.
    """
    n1, n2, n3 = pb.dims
    X, Y = n1 // 2, n2 // 2
    if C_ref is None or rho_ref is None:
        C_ref, rho_ref = reference_medium(pb)
    r = np.asarray(r, dtype=np.complex128).reshape(3, n3, Y, X)
    what = np.stack([block_fourier_separable(r[a], pb.dims, kappa, b) for a in range(3)])  # (3, n3, Y, X)
    what = what.reshape(3, -1)
    zhat = np.empty_like(what)
    for idx, (p, q, rr) in enumerate(representatives(pb.dims)):
        zhat[:, idx] = precond_mode_factor(pb, kappa, sigma, p, q, rr, C_ref, rho_ref) @ what[:, idx]
    zhat = zhat.reshape(3, n3, Y, X)
    z = np.stack([block_fourier_separable_inverse(zhat[a], pb.dims, kappa, b) for a in range(3)])
    return z.reshape(3, -1)


def precond_full(pb: Problem, kappa, sigma: float, r) -> np.ndarray:
    """Full-space preconditioner: the four block preconditioners on the block parts of r."""
    r = np.asarray(r, dtype=np.complex128).reshape(3, pb.n)
    z = np.zeros_like(r)
    for b in range(4):
        z += inject(pb, b, precond_block(pb, kappa, b, sigma, extract(pb, b, r)))
    return z


# --------------------------------------------------------------------------- eigen oracles (Sec. 6)
def eigs_shift_invert(A, M, nev: int, sigma: float, tol: float = 1e-13, deflate=None):
    """Lowest eigenpairs of (A, M) by ARPACK shift-invert (scipy eigsh, the algorithm class of MATLAB eigs).

    The inner solve is a sparse LU of A - sigma M.  ``deflate``: optional
    (3n x r) basis of a null space to project out (M-orthogonal complement).
    Returns (evals ascending, evecs).
    """
    Ash = (A - sigma * M).tocsc()
    lu = spla.splu(Ash)
    n = A.shape[0]
    Md = M.diagonal().real
    if deflate is not None:
        Z = np.asarray(deflate)
        G = Z.conj().T @ (Md[:, None] * Z)
        L = np.linalg.cholesky(G)
        Z = np.linalg.solve(L, Z.conj().T).conj().T  # M-orthonormal
    else:
        Z = None

    def proj(v):
        if Z is None:
            return v
        return v - Z @ (Z.conj().T @ (Md * v))

    # ARPACK mode 3: OP = (A - sigma M)^-1 M in the M inner product; OPinv receives M x.
    def opinv(y):
        return proj(lu.solve(np.asarray(y).reshape(-1)))

    OPinv = spla.LinearOperator((n, n), matvec=opinv, dtype=np.complex128)
    rng = np.random.default_rng(12345)
    v0 = proj(rng.standard_normal(n) + 1j * rng.standard_normal(n))
    lam, V = spla.eigs(A, k=nev, M=M.tocsr(), sigma=sigma, OPinv=OPinv, which="LM", tol=tol,
                       v0=v0, ncv=min(n - 1, max(2 * nev + 1, 24)))
    lam = lam.real
    order = np.argsort(lam)
    return lam[order], V[:, order]


def gamma_null_basis(pb: Problem, b=None) -> np.ndarray:
    """Zero-derivative modes chi_mu e_alpha at Gamma (Eq. gamma_null_space_main, App. C).

    Full space: 12 columns; block b: the 3 restrictions of chi_0 e_alpha
    (chi_12, chi_13, chi_23 are +-1 constants on a block).
    """
    n1, n2, n3 = pb.dims
    k, j, i = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    chis = [np.ones_like(i), (-1) ** (i + j), (-1) ** (i + k), (-1) ** (j + k)]
    n = pb.n
    cols = []
    for chi in chis:
        c = chi.reshape(-1).astype(np.complex128)
        for a in range(3):
            v = np.zeros(3 * n, dtype=np.complex128)
            v[a * n:(a + 1) * n] = c
            cols.append(v)
    Z = np.stack(cols, axis=1)
    if b is None:
        return Z
    Q = so.Q_matrix(pb.dims, b)
    Zb = Q.conj().T @ Z
    return Zb[:, :3]


def eigs_oracle(pb: Problem, kappa, nev: int, sigma: float, b=None, tol: float = 1e-13):
    """Lowest nev non-zero eigenvalues of the (block) pencil by ARPACK shift-invert.

    At kappa == 0 (mod 1) the zero-derivative modes are projected out exactly.
    """
    A, M = sparse_pencil(pb, kappa, b)
    at_gamma = np.all(np.abs(np.asarray(kappa) - np.round(kappa)) < 1e-15)
    Z = gamma_null_basis(pb, b) if at_gamma else None
    lam, _ = eigs_shift_invert(A, M, nev, sigma, tol=tol, deflate=Z)
    return lam


def merge_complete(block_vals, block_complete_upto, nev: int):
    """Merge four block spectra (Sec. 6.1) with the completeness rule.

    block_vals[b]: ascending eigenvalues found in block b.
    block_complete_upto[b]: True iff block b's list holds *all* of its
    eigenvalues below its largest listed one (true for a converged
    lowest-first solve).
    Returns (merged lowest nev, ok, blocks_to_extend).  The union's lowest nev
    are final iff each block either lists a value >= the nev-th merged value or
    is known to have no further eigenvalues below it.
    """
    allv = np.sort(np.concatenate([np.asarray(v) for v in block_vals]))
    if allv.size < nev:
        return allv, False, list(range(len(block_vals)))
    cut = allv[nev - 1]
    extend = []
    for b, v in enumerate(block_vals):
        v = np.asarray(v)
        if not block_complete_upto[b]:
            extend.append(b)
        elif v.size == 0 or v[-1] < cut:
            extend.append(b)
    return allv[:nev], len(extend) == 0, extend


# --------------------------------------------------------------------------- Hellmann-Feynman gradients
def upper21(g66):
    """(n,6,6) -> (n,21): the independent upper-triangular entries (p <= r), row order."""
    iu = np.triu_indices(6)
    return g66[:, iu[0], iu[1]]


def eigpair_gradients(pb: Problem, kappa, x_full, lam):
    """d lambda / d C_i[p][q] and d lambda / d rho_i for an M-normalised eigenvector x.

    Hellmann-Feynman: d lambda = x^H (dA - lambda dM) x with dA = B dC B^H, so
    d lambda/d C_i[p][q] = Re(conj(e_p) e_q) (entries p,q and q,p tied: factor
    2 off the diagonal, per independent upper-triangular entry), e = (B^H x)(i);
    d lambda/d rho_i = -lambda sum_alpha |x_alpha(i)|^2.
    Returns (gC (n, 6, 6) symmetric-pair convention, grho (n,)).
    """
    e = strain_full(pb, kappa, x_full)  # (6, n)
    g = np.real(np.conj(e)[:, None, :] * e[None, :, :])  # (6,6,n)
    gC = np.transpose(g, (2, 0, 1)).copy()
    off = ~np.eye(6, dtype=bool)
    gC[:, off] *= 2.0
    x = np.asarray(x_full).reshape(3, pb.n)
    grho = -lam * np.sum(np.abs(x) ** 2, axis=0)
    return gC, grho
