"""Two-phase phononic-crystal cells (seeded, synthetic).

The construction follows the paper's two-phase setting (Sec. 7.1: a matrix
phase with a spherical inclusion centred at reduced coordinate (1/2,1/2,1/2),
nodes at r = (i,j,k)/N, Voigt order [11,22,33,23,13,12] with engineering
shear).  The synthetic stand-in materials are:

* matrix: isotropic, Lame lambda = 40 GPa, mu = 30 GPa, rho = 1200 kg/m^3;
* inclusion: C = Q diag(u) Q^T with u ~ U[20, 200] GPa and Q a Haar-random
  6x6 orthogonal matrix (QR of a Gaussian matrix, column signs fixed so that
  diag(R) > 0), rho = 7800 kg/m^3.

Random draws, in this order, from ``numpy.random.default_rng(seed)``:
``G = standard_normal((6, 6))``, ``u = uniform(20, 200, 6)`` and, only when
the radius is drawn, ``R = uniform(0.2, 0.4)``.

A node (i, j, k) belongs to the inclusion iff
``(i - N/2)^2 + (j - N/2)^2 + (k - N/2)^2 <= (R N)^2 (1 + 1e-12)``: the left
side is an exact integer, the slack makes on-sphere nodes count as inside.

Arrays use the full-grid node order l = i + N (j + N k) (i fastest), the
order fixed by the shift operators H_1 = I (x) I (x) K_1 etc. (Eq. H_def).
"""

from __future__ import annotations

import dataclasses

import numpy as np

GPA = 1.0e9


def isotropic_voigt(lam: float, mu: float) -> np.ndarray:
    """6x6 Voigt stiffness of an isotropic solid (engineering shear)."""
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[0, 0] = C[1, 1] = C[2, 2] = lam + 2.0 * mu
    C[3, 3] = C[4, 4] = C[5, 5] = mu
    return C


def random_spd_voigt(rng: np.random.Generator, lo: float = 20.0, hi: float = 200.0) -> np.ndarray:
    """Seeded SPD 6x6 stiffness in Pa: Haar orthogonal basis, eigenvalues U[lo, hi] GPa."""
    G = rng.standard_normal((6, 6))
    Q, R = np.linalg.qr(G)
    Q = Q * np.sign(np.diag(R))[None, :]
    u = rng.uniform(lo, hi, 6) * GPA
    C = (Q * u[None, :]) @ Q.T
    return 0.5 * (C + C.T)


@dataclasses.dataclass
class TwoPhaseCell:
    """A discretised two-phase unit cell.

    C:     (2, 6, 6) float64 Voigt stiffness per phase, Pa (phase 0 = matrix).
    rho:   (2,) float64 density per phase, kg/m^3.
    phase: (N^3,) uint8 phase id per node (full-grid order), or None.
    theta: (N^3,) float32 inclusion fraction per node, or None.
    a_lat: (3, 3) float64 lattice basis A_lat = [a1 a2 a3] (columns), metres.
    """

    N: int
    C: np.ndarray
    rho: np.ndarray
    phase: np.ndarray | None
    theta: np.ndarray | None
    a_lat: np.ndarray
    seed: int | None = None
    radius: float | None = None

    @property
    def n(self) -> int:
        return self.N ** 3

    def theta_f64(self) -> np.ndarray:
        """Per-node inclusion fraction as float64 (0/1 for a binary cell)."""
        if self.theta is not None:
            return self.theta.astype(np.float64)
        if self.phase is not None:
            return self.phase.astype(np.float64)
        return np.zeros(self.n)

    def node_C(self) -> np.ndarray:
        """(n, 6, 6) nodewise stiffness (1 - theta) C0 + theta C1 (Eq. subpixel_material_average)."""
        t = self.theta_f64()[:, None, None]
        return (1.0 - t) * self.C[0][None] + t * self.C[1][None]

    def node_rho(self) -> np.ndarray:
        t = self.theta_f64()
        return (1.0 - t) * self.rho[0] + t * self.rho[1]


def sphere_mask(N: int, radius: float) -> np.ndarray:
    """uint8 (N^3,) mask of nodes inside the centred sphere of reduced radius ``radius``."""
    idx = np.arange(N, dtype=np.int64) - N // 2
    k, j, i = np.meshgrid(idx, idx, idx, indexing="ij")  # k slowest, i fastest
    d2 = i * i + j * j + k * k
    rN = float(radius) * N
    inside = d2.astype(np.float64) <= rN * rN * (1.0 + 1e-12)
    return inside.reshape(-1).astype(np.uint8)


def two_phase_sphere(N: int, radius: float, seed: int, a: float = 1.0) -> TwoPhaseCell:
    """Seeded two-phase simple-cubic cell with an anisotropic spherical inclusion."""
    if N % 2 != 0 or N < 4:
        raise ValueError("N must be even and >= 4")
    rng = np.random.default_rng(seed)
    C1 = random_spd_voigt(rng)
    C0 = isotropic_voigt(40.0 * GPA, 30.0 * GPA)
    C = np.stack([C0, C1])
    rho = np.array([1200.0, 7800.0])
    return TwoPhaseCell(N=N, C=C, rho=rho, phase=sphere_mask(N, radius), theta=None,
                        a_lat=np.eye(3) * a, seed=seed, radius=radius)


def config_cell(name: str, N: int | None = None) -> TwoPhaseCell:
    """The named synthetic workloads.

    ``tiny``: N=8, R=0.35, seed 1.  ``fp64``: N=48, R=0.35, seed 2.
    ``precision``: N=160, R=0.3, seed 3.  ``diff``: N=64, R=0.35, seed 4.
    ``batch``: N in {32, 48, 64, 96, 128} with seed 10+i and R ~ U[0.2, 0.4]
    drawn after the stiffness from the same generator.
    """
    table = {"tiny": (8, 0.35, 1), "fp64": (48, 0.35, 2), "precision": (160, 0.3, 3),
             "diff": (64, 0.35, 4)}
    if name in table:
        n0, r, s = table[name]
        return two_phase_sphere(N or n0, r, s)
    if name == "batch":
        sizes = [32, 48, 64, 96, 128]
        if N not in sizes:
            raise ValueError("batch grids are N in %s" % sizes)
        i = sizes.index(N)
        seed = 10 + i
        rng = np.random.default_rng(seed)
        C1 = random_spd_voigt(rng)
        radius = float(rng.uniform(0.2, 0.4))
        C0 = isotropic_voigt(40.0 * GPA, 30.0 * GPA)
        return TwoPhaseCell(N=N, C=np.stack([C0, C1]), rho=np.array([1200.0, 7800.0]),
                            phase=sphere_mask(N, radius), theta=None, a_lat=np.eye(3),
                            seed=seed, radius=radius)
    raise KeyError(name)


def quartz_silicon_constants():
    """Low-quartz matrix and silicon inclusion of the paper's FCC example (Sec. 7.1).

    Returns (C_quartz, rho_quartz, C_si, rho_si) in Pa and kg/m^3; unlisted
    entries follow from symmetry or are zero.
    """
    Cq = np.zeros((6, 6))
    Cq[0, 0] = Cq[1, 1] = 86.6
    Cq[0, 1] = 6.9
    Cq[0, 2] = Cq[1, 2] = 13.6
    Cq[2, 2] = 106.7
    Cq[0, 3] = -17.7
    Cq[1, 3] = 17.7
    Cq[3, 3] = Cq[4, 4] = 57.7
    Cq[4, 5] = -17.7
    Cq[5, 5] = 39.85
    Cq = np.triu(Cq) + np.triu(Cq, 1).T
    Cs = np.zeros((6, 6))
    Cs[0, 0] = Cs[1, 1] = Cs[2, 2] = 166.0
    Cs[0, 1] = Cs[0, 2] = Cs[1, 2] = 64.0
    Cs[3, 3] = Cs[4, 4] = Cs[5, 5] = 79.6
    Cs = np.triu(Cs) + np.triu(Cs, 1).T
    return Cq * GPA, 2650.0, Cs * GPA, 2329.0


FCC_A0 = 3.0e-2  # lattice constant of the paper's FCC example, m


def fcc_lattice(a0: float = FCC_A0) -> np.ndarray:
    """FCC primitive basis a1 = (0, a0/2, a0/2), a2 = (a0/2, 0, a0/2), a3 = (a0/2, a0/2, 0) as the
    columns of A_lat (Sec. 7.1, Eq. num_lattice_vectors)."""
    h = a0 / 2
    return np.array([[0.0, h, h], [h, 0.0, h], [h, h, 0.0]]).T


def fcc_quartz_silicon_cell(N: int, supersample: int = 8, radius: float = 0.25) -> TwoPhaseCell:
    """The paper's FCC example (Sec. 7.1): low-quartz matrix, silicon sphere of radius
    ``radius`` * a0 centred at reduced coordinate (1/2, 1/2, 1/2), sub-pixel inclusion fractions
    (Eq. subpixel_material_average).

    The cell of node r = (i, j, k) / N is read as the reduced cube of side 1/N centred on the
    node, mapped to Cartesian space by A_lat; its silicon fraction theta is the share of
    ``supersample``^3 equally spaced sub-samples inside the sphere.  Nodes farther from the
    sphere surface than the cell's circumradius get 0 or 1 directly.
    """
    Cq, rq, Cs, rs = quartz_silicon_constants()
    A = fcc_lattice()
    n = N ** 3
    idx = np.arange(n)
    r = np.stack([idx % N, (idx // N) % N, idx // (N * N)], axis=1).astype(np.float64) / N
    centre = A @ np.full(3, 0.5)
    R = radius * FCC_A0
    x = r @ A.T
    d = np.linalg.norm(x - centre, axis=1)
    # circumradius of a cell: half the longest diagonal of the parallelepiped spanned by A / N
    diag = max(np.linalg.norm(A @ np.array(sgn)) for sgn in
               [(1, 1, 1), (1, 1, -1), (1, -1, 1), (-1, 1, 1)]) / (2 * N)
    theta = (d <= R).astype(np.float64)
    cut = np.nonzero(np.abs(d - R) <= diag)[0]
    off = (np.arange(supersample) + 0.5) / supersample - 0.5
    sub = np.stack(np.meshgrid(off, off, off, indexing="ij"), axis=-1).reshape(-1, 3) / N  # reduced offsets
    sub_x = sub @ A.T
    for lo in range(0, cut.size, 4096):
        c = cut[lo:lo + 4096]
        pts = x[c][:, None, :] + sub_x[None, :, :]
        inside = np.linalg.norm(pts - centre, axis=2) <= R
        theta[c] = inside.mean(axis=1)
    return TwoPhaseCell(N=N, C=np.stack([Cq, Cs]), rho=np.array([rq, rs]), phase=None,
                        theta=theta.astype(np.float32), a_lat=A)
