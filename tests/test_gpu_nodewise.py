"""Nodewise material (every node its own symmetric stiffness and density) through the C ABI,
and the autograd functions whose inputs are that material, against the oracle.

* The complex128 apply of a grid made by pc_grid_create_nodewise equals the oracle's nodewise
  pencil (A - s M) x element-wise (1e-12), in the four parity blocks and the full space, on a
  cubic and an FCC lattice; complex64 applies and mixed precision are refused (PC_EINVAL).
* A two-phase material entered node by node gives the same eigenvalues as the two-phase grid.
* The lowest eigenvalues of a randomly perturbed nodewise material equal dense LAPACK (1e-10).
* NodewiseBandEigenvalues: the gradient with respect to the (N^3, 21) stiffness and (N^3,)
  density equals the oracle's dense-eigenvector Hellmann-Feynman gradient (1e-7), and central
  differences with a relative step of 1e-6 along seeded random directions in (C, rho) (the
  forward evaluated by the GPU solver on the perturbed nodewise material).
* NodewiseBandGap: the gap-width gradient against central differences along seeded directions.
* NodewiseBandStructure (lockstep over several Bloch vectors) = NodewiseBandEigenvalues per
  Bloch vector, eigenvalues and summed gradients.
"""

import numpy as np
import pytest

from oracle import oracle as O
from oracle.oracle import Problem
from workloads import complex_gaussian, two_phase_sphere

pytestmark = pytest.mark.gpu

IU = np.triu_indices(6)
KAPPA = (0.13, 0.27, 0.41)
FCC = np.array([[0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]])


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


def perturbed_material(N, seed, a_lat=None):
    """A two-phase cell with every node's stiffness and density perturbed (SI units): the nodewise
    (C21, rho) and the oracle's Problem of the same material in units C / 1e9, rho / 1e3, L."""
    rng = np.random.default_rng(seed)
    cell = two_phase_sphere(N, 0.35, 3)
    n = N ** 3
    th = cell.theta_f64()
    C = np.asarray(cell.C)
    Cn = (1 - th)[:, None, None] * C[0][None] + th[:, None, None] * C[1][None]
    G = rng.standard_normal((n, 6, 6))
    Cn = Cn + 4e9 * (G + np.transpose(G, (0, 2, 1)))  # symmetric, +-10 % of the matrix stiffness
    rho = ((1 - th) * cell.rho[0] + th * cell.rho[1]) * (1 + 0.2 * rng.uniform(size=n))
    A = np.eye(3) if a_lat is None else np.asarray(a_lat, dtype=np.float64)
    L = abs(np.linalg.det(A)) ** (1 / 3)
    pb = Problem(dims=(N,) * 3, ainv=np.linalg.inv(A / L), C=C / 1e9, rho=np.asarray(cell.rho) / 1e3, theta=th,
                 C_nodes=Cn / 1e9, rho_nodes=rho / 1e3)
    return Cn[:, IU[0], IU[1]], rho, pb, A, L


@pytest.mark.parametrize("lattice", ["cubic", "fcc"])
@pytest.mark.parametrize("block", [0, 1, 2, 3, -1])
def test_nodewise_apply_matches_oracle(pc, lattice, block):
    import torch
    N = 8
    C21, rho, pb, A, L = perturbed_material(N, 11, None if lattice == "cubic" else FCC)
    g = pc.pc_grid_create_nodewise(N, C21, rho, a_lat=A)
    try:
        C0, rho0, Lg = pc.pc_grid_units(g)
        assert (C0, rho0) == (1e9, 1e3) and abs(Lg - L) < 1e-14
        kappa = [0.3, 0.1, 0.2]
        pc.pc_set_k(g, kappa)
        m = N ** 3 // 4 if block >= 0 else N ** 3
        x = complex_gaussian((3, m), 21 + block)
        xd = torch.from_numpy(x.reshape(-1)).cuda()
        y = torch.full_like(xd, complex(float("nan"), float("nan")))
        pc.pc_block_apply(g, block, xd, y, shift=0.6)
        Ao, Mo = O.sparse_pencil(pb, kappa, block if block >= 0 else None)
        ref = (Ao - 0.6 * Mo) @ x.reshape(-1)
        got = y.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    finally:
        pc.pc_grid_destroy(g)


def test_nodewise_refuses_complex64_and_mixed(pc):
    import torch
    N = 8
    C21, rho, _, _, _ = perturbed_material(N, 12)
    g = pc.pc_grid_create_nodewise(N, C21, rho)
    try:
        pc.pc_set_k(g, KAPPA)
        x = torch.zeros(3 * N ** 3 // 4, dtype=torch.complex64, device="cuda")
        with pytest.raises(pc.PcError) as ei:
            pc.pc_block_apply(g, 0, x, torch.zeros_like(x))
        assert ei.value.code == pc.PC_EINVAL
        with pytest.raises(pc.PcError) as ei:
            pc.pc_eigs(g, KAPPA, 4, opt=pc.pc_options_default(precision=pc.PC_PREC_MIXED))
        assert ei.value.code == pc.PC_EINVAL
    finally:
        pc.pc_grid_destroy(g)
    with pytest.raises(pc.PcError):  # a non-positive density is refused
        bad = rho.copy()
        bad[5] = 0.0
        pc.pc_grid_create_nodewise(N, C21, bad)


def test_two_phase_entered_node_by_node_matches_the_two_phase_grid(pc, ad):
    N = 12
    cell = two_phase_sphere(N, 0.35, 2)
    C21, rho = ad.two_phase_nodewise(cell)
    g1 = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    g2 = pc.pc_grid_create_nodewise(N, C21, rho, a_lat=cell.a_lat)
    try:
        for kappa in ([0.3, 0.1, 0.2], [0.0, 0.0, 0.0]):
            e1, _, _ = pc.pc_eigs(g1, kappa, 12)
            e2, _, _ = pc.pc_eigs(g2, kappa, 12)
            assert np.abs(e1 - e2).max() <= 1e-10 * e1.max()
    finally:
        pc.pc_grid_destroy(g1)
        pc.pc_grid_destroy(g2)


@pytest.mark.parametrize("kappa", [[0.3, 0.1, 0.2], [0.0, 0.0, 0.0]])
def test_nodewise_eigenvalues_match_dense(pc, kappa):
    N = 8
    C21, rho, pb, A, _ = perturbed_material(N, 13)
    g = pc.pc_grid_create_nodewise(N, C21, rho, a_lat=A)
    try:
        for full in (0, 1):
            ev, _, info = pc.pc_eigs(g, kappa, 12, opt=pc.pc_options_default(full_space=full))
            assert info["max_rel_resid"] <= 1e-8
            ref = O.lowest_nonzero(O.dense_eigvals(pb, kappa), 12) * 1e9 / 1e3
            assert np.abs(ev - ref).max() <= 1e-10 * ref.max()
    finally:
        pc.pc_grid_destroy(g)


def _weighted_sum(ev, w):
    return float(np.dot(w, ev))


def test_nodewise_autograd_matches_the_dense_gradient(pc, ad):
    import torch
    N = 8
    C21, rho, pb, A, L = perturbed_material(N, 14)
    nev = 6
    w = np.array([1.0, -0.5, 0.75, 2.0, -1.25, 0.3])
    Ct = torch.tensor(C21, dtype=torch.float64, requires_grad=True)
    rt = torch.tensor(rho, dtype=torch.float64, requires_grad=True)
    lam = ad.band_eigenvalues_nodewise(Ct, rt, N, KAPPA, nev, a_lat=A)
    (lam * torch.as_tensor(w)).sum().backward()
    # the oracle's gradient from dense M-normalised eigenvectors (hat units -> SI)
    vals, vecs = O.dense_eigpairs(pb, KAPPA)
    assert np.abs(vals[:nev] * 1e6 - lam.detach().numpy()).max() <= 1e-10 * vals[nev - 1] * 1e6
    dC, drho = np.zeros((N ** 3, 21)), np.zeros(N ** 3)
    for v in range(nev):
        gC, grho = O.eigpair_gradients(pb, KAPPA, vecs[v], vals[v])
        dC += w[v] * gC[:, IU[0], IU[1]] / (1e3 * L ** 2)
        drho += w[v] * grho * 1e6 / 1e3
    gc = Ct.grad.numpy()
    gr = rt.grad.numpy()
    assert np.abs(gc - dC).max() <= 1e-7 * np.abs(dC).max()
    assert np.abs(gr - drho).max() <= 1e-7 * np.abs(drho).max()


def test_nodewise_autograd_matches_central_differences(pc, ad):
    import torch
    N = 8
    C21, rho, _, A, _ = perturbed_material(N, 15)
    nev = 6
    w = np.array([0.4, 1.0, -0.7, 0.2, 1.5, -0.9])
    Ct = torch.tensor(C21, dtype=torch.float64, requires_grad=True)
    rt = torch.tensor(rho, dtype=torch.float64, requires_grad=True)
    lam = ad.band_eigenvalues_nodewise(Ct, rt, N, KAPPA, nev, a_lat=A)
    (lam * torch.as_tensor(w)).sum().backward()
    gc, gr = Ct.grad.numpy(), rt.grad.numpy()
    h = 1e-6  # relative step: entries move by h times their scale
    sC, sr = np.abs(C21[:, [0, 6, 11]]).mean(), rho.mean()
    rng = np.random.default_rng(77)
    for _ in range(6):
        dCd = sC * rng.standard_normal(C21.shape)
        drd = sr * rng.standard_normal(rho.shape)
        vals = []
        for sgn in (1.0, -1.0):
            ev, _ = ad._solve_nodewise(C21 + sgn * h * dCd, rho + sgn * h * drd, N, KAPPA, nev, A, None)
            vals.append(_weighted_sum(ev, w))
        fd = (vals[0] - vals[1]) / (2 * h)
        an = float(np.sum(gc * dCd) + np.sum(gr * drd))
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-9 * np.abs(w).sum() * 1e8


def test_nodewise_band_gap_matches_central_differences(pc, ad):
    import torch
    N = 8
    C21, rho, _, A, _ = perturbed_material(N, 16)
    kappas = [[0.0, 0.0, 0.0], [0.25, 0.0, 0.0], [0.5, 0.0, 0.0], [0.5, 0.5, 0.0]]
    lo = 4
    Ct = torch.tensor(C21, dtype=torch.float64, requires_grad=True)
    rt = torch.tensor(rho, dtype=torch.float64, requires_grad=True)
    gap = ad.band_gap_nodewise(Ct, rt, N, kappas, lo, a_lat=A)
    gap.backward()
    gc, gr = Ct.grad.numpy(), rt.grad.numpy()
    h = 1e-6
    sC, sr = np.abs(C21[:, [0, 6, 11]]).mean(), rho.mean()
    rng = np.random.default_rng(78)
    for _ in range(3):
        dCd = sC * rng.standard_normal(C21.shape)
        drd = sr * rng.standard_normal(rho.shape)
        vals = []
        for sgn in (1.0, -1.0):
            with torch.no_grad():
                v = ad.band_gap_nodewise(torch.tensor(C21 + sgn * h * dCd), torch.tensor(rho + sgn * h * drd), N,
                                         kappas, lo, a_lat=A)
            vals.append(float(v))
        fd = (vals[0] - vals[1]) / (2 * h)
        an = float(np.sum(gc * dCd) + np.sum(gr * drd))
        assert abs(fd - an) <= 1e-5 * abs(an) + 1e-6


def test_band_structure_autograd_equals_per_bloch_vector_autograd(pc, ad):
    """NodewiseBandStructure (all Bloch vectors in one lockstep solve, eigenvectors from
    pc_eigs_multi) gives the per-Bloch-vector eigenvalues and the summed gradient of
    NodewiseBandEigenvalues called once per Bloch vector."""
    import torch
    N = 8
    C21, rho, _, A, _ = perturbed_material(N, 17)
    kappas = [[0.0, 0.0, 0.0], [0.3, 0.1, 0.2], [0.5, 0.5, 0.0]]
    nev = 6
    w = np.array([[1.0, -0.5, 0.75, 2.0, -1.25, 0.3], [0.2, 0.4, -1.0, 0.5, 0.9, -0.3],
                  [1.5, 0.1, 0.6, -0.8, 0.25, 1.1]])
    Ct = torch.tensor(C21, dtype=torch.float64, requires_grad=True)
    rt = torch.tensor(rho, dtype=torch.float64, requires_grad=True)
    lam = ad.band_structure_nodewise(Ct, rt, N, kappas, nev, a_lat=A)
    (lam * torch.as_tensor(w)).sum().backward()
    gc_sum, gr_sum = 0.0, 0.0
    for i, k in enumerate(kappas):
        C1 = torch.tensor(C21, dtype=torch.float64, requires_grad=True)
        r1 = torch.tensor(rho, dtype=torch.float64, requires_grad=True)
        l1 = ad.band_eigenvalues_nodewise(C1, r1, N, k, nev, a_lat=A)
        assert np.abs(l1.detach().numpy() - lam[i].detach().numpy()).max() <= 1e-10 * l1.detach().numpy().max()
        (l1 * torch.as_tensor(w[i])).sum().backward()
        gc_sum = gc_sum + C1.grad.numpy()
        gr_sum = gr_sum + r1.grad.numpy()
    assert np.abs(Ct.grad.numpy() - gc_sum).max() <= 1e-8 * np.abs(gc_sum).max()
    assert np.abs(rt.grad.numpy() - gr_sum).max() <= 1e-8 * np.abs(gr_sum).max()
