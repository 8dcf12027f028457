"""Sparse-matrix transcription of the paper's discrete operators (FP64, CPU).

Test infrastructure only (tests, the smoke check and the bench's CPU-baseline
leg); the product library never imports this package.

Every matrix is built exactly as the paper writes it, with scipy.sparse:

* K_l      -- Eq. K_def: [[0, I_{n_l - 1}], [exp(i phi_l), 0]]
* H_1..H_3 -- Eq. H_def: H_1 = I (x) I (x) K_1, H_2 = I (x) K_2 (x) I, H_3 = K_3 (x) I (x) I
* S_d1..4  -- Eq. Sd_def: H3 H2 H1, H3^-1 H2 H1, H3 H2^-1 H1, H3^-1 H2^-1 H1
* D_dl     -- Eq. Dd_def: (S_dl - I) / h_d
* Dt_s     -- Eq. Dtilde_recon
* Dcal_m   -- Eqs. Dhat_def, Dcal_cartesian_transform
* B_h      -- Eq. B_discrete
* A_h, M_h -- Eq. discrete_GEP (C_h, M_h nodewise)
* P_sigma  -- Eq. Proj_sigma from Gamma_12, Gamma_13 (Eqs. Gamma12_13_sign_main, Gamma12_13_op_main)

Practical up to N ~ 48 (the matrices hold ~51 nonzeros per row).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

C_SIGNS = np.array([[1, 1, 1, 1], [1, 1, -1, -1], [1, -1, 1, -1]], dtype=np.float64)


def K_matrix(n: int, phi: float) -> sp.csr_matrix:
    """One-dimensional Bloch shift (Eq. K_def)."""
    rows = np.arange(n)
    cols = (rows + 1) % n
    vals = np.ones(n, dtype=np.complex128)
    vals[n - 1] = np.exp(1j * phi)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def H_matrices(dims, phi):
    """H_1, H_2, H_3 of Eq. H_def (node index l = i + n1 (j + n2 k))."""
    n1, n2, n3 = dims
    I1, I2, I3 = (sp.identity(m, dtype=np.complex128, format="csr") for m in dims)
    K1, K2, K3 = (K_matrix(m, p) for m, p in zip(dims, phi))
    H1 = sp.kron(I3, sp.kron(I2, K1), format="csr")
    H2 = sp.kron(I3, sp.kron(K2, I1), format="csr")
    H3 = sp.kron(K3, sp.kron(I2, I1), format="csr")
    return H1, H2, H3


def unitary_inverse(H: sp.csr_matrix) -> sp.csr_matrix:
    """Inverse of a phased permutation matrix (unitary): its conjugate transpose."""
    return H.conj().T.tocsr()


def S_matrices(dims, phi):
    """The four body-diagonal Bloch shifts (Eq. Sd_def)."""
    H1, H2, H3 = H_matrices(dims, phi)
    H2i, H3i = unitary_inverse(H2), unitary_inverse(H3)
    return [H3 @ H2 @ H1, H3i @ H2 @ H1, H3 @ H2i @ H1, H3i @ H2i @ H1]


def derivative_matrices(dims, phi, ainv):
    """Cartesian derivative matrices Dcal_1..3 (Eqs. Dd_def, Dtilde_recon, Dhat_def, Dcal_cartesian_transform).

    ainv is A_lat^{-1} with ainv[s, m] = (A_lat^{-1})_{s m}.
    """
    h = np.array([1.0 / m for m in dims])
    hd = np.sqrt(np.sum(h ** 2))
    n = int(np.prod(dims))
    Id = sp.identity(n, dtype=np.complex128, format="csr")
    S = S_matrices(dims, phi)
    D = [(Sl - Id) / hd for Sl in S]
    Dt = []
    for s in range(3):
        acc = sp.csr_matrix((n, n), dtype=np.complex128)
        for l in range(4):
            acc = acc + C_SIGNS[s, l] * D[l]
        Dt.append(hd / (4.0 * h[s]) * acc)
    Dhat = [-1j * Dt[s] for s in range(3)]
    Dcal = []
    for m in range(3):
        acc = sp.csr_matrix((n, n), dtype=np.complex128)
        for s in range(3):
            acc = acc + ainv[s, m] * Dhat[s]
        Dcal.append(acc.tocsr())
    return Dcal


def B_matrix(dims, phi, ainv) -> sp.csr_matrix:
    """Divergence-type matrix B_h(k), 3n x 6n (Eq. B_discrete)."""
    D1, D2, D3 = derivative_matrices(dims, phi, ainv)
    Z = None
    return sp.bmat([[D1, Z, Z, Z, D3, D2],
                    [Z, D2, Z, D3, Z, D1],
                    [Z, Z, D3, D2, D1, Z]], format="csr")


def C_matrix(node_C: np.ndarray) -> sp.csr_matrix:
    """Nodewise stiffness C_h, 6n x 6n, Voigt-component-major (row p*n + l)."""
    n = node_C.shape[0]
    rows, cols, vals = [], [], []
    base = np.arange(n)
    for p in range(6):
        for q in range(6):
            rows.append(p * n + base)
            cols.append(q * n + base)
            vals.append(node_C[:, p, q])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(6 * n, 6 * n))


def M_matrix(node_rho: np.ndarray) -> sp.csr_matrix:
    """Nodewise mass M_h, 3n x 3n."""
    return sp.diags(np.tile(node_rho, 3).astype(np.complex128), format="csr")


def A_matrix(dims, phi, ainv, node_C) -> sp.csr_matrix:
    """A_h(k) = B_h C_h B_h^H (Eq. discrete_GEP)."""
    B = B_matrix(dims, phi, ainv)
    return (B @ C_matrix(node_C) @ B.conj().T).tocsr()


def parity_signs(dims):
    """g_12 = (-1)^(i+j), g_13 = (-1)^(i+k) on the scalar grid (Eq. Gamma12_13_sign_main)."""
    n1, n2, n3 = dims
    k, j, i = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    g12 = ((-1.0) ** (i + j)).reshape(-1)
    g13 = ((-1.0) ** (i + k)).reshape(-1)
    return g12, g13


def block_signs(b: int):
    """Block b = 2 p12 + p13 <-> (sigma12, sigma13) = ((-1)^p12, (-1)^p13)."""
    return (1.0 if (b >> 1) == 0 else -1.0), (1.0 if (b & 1) == 0 else -1.0)


def projector_diag(dims, b: int) -> np.ndarray:
    """Diagonal of the scalar projector P_sigma = 1/4 (I + s12 G12)(I + s13 G13) (Eq. Proj_sigma)."""
    g12, g13 = parity_signs(dims)
    s12, s13 = block_signs(b)
    return 0.25 * (1.0 + s12 * g12) * (1.0 + s13 * g13)


def block_nodes(dims, b: int) -> np.ndarray:
    """Full-grid nodes spanning V_sigma, ascending: the range of the 0/1 projector P_sigma."""
    d = projector_diag(dims, b)
    return np.nonzero(d > 0.5)[0].astype(np.int64)


def Q_matrix(dims, b: int) -> sp.csr_matrix:
    """Orthonormal basis of the velocity block space (I_3 (x) selection of block nodes), 3n x 3n/4."""
    n = int(np.prod(dims))
    nodes = block_nodes(dims, b)
    nb = nodes.size
    rows = np.concatenate([a * n + nodes for a in range(3)])
    cols = np.arange(3 * nb)
    return sp.csr_matrix((np.ones(3 * nb, dtype=np.complex128), (rows, cols)), shape=(3 * n, 3 * nb))
