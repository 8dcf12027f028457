"""Parity at the workloads' full grid sizes (N = 48: the FP64 band workload; N = 160: the
apply and precision workloads), where the oracle's dense and ARPACK solves are out of reach.

* The block apply exactly as the bench times it (all four blocks in one launch, N = 160) on
  sampled outputs the oracle computes node by node.

* A homogeneous medium has a closed-form spectrum at any size: the union over all modes of
  eig(B_hat(m) C B_hat(m)^H) / rho (Sec. 5.3, App. B), evaluated by the oracle plane by plane.
  The solver's lowest 20 eigenvalues must equal it to 1e-10 relative, in FP64 and in mixed
  precision with FP64 refinement.
* On the heterogeneous N = 48 workload cell, every returned eigenpair is checked with the
  oracle's matrix-free C apply: true residual ||A x - lambda M x|| <= 1e-8 |lambda| ||M x||
  (which bounds the eigenvalue's distance to the spectrum), M-orthonormality to 1e-9.
* On the heterogeneous N = 160 precision cell, mixed precision returns the FP64 solve's 20
  eigenvalues band by band to 1e-10, and FP64 eigenpairs across the band range pass the
  oracle's residual test and M-normalisation.
* On the N = 48 grid, a right-hand side holding a NaN ends the inner solve with PC_ENAN and
  leaves x at its zero start (the status path of the reductions, no device fault).
* Guard bands: outputs written into views of larger buffers leave a sentinel on both sides
  untouched (no write outside the caller's vector), for the benchmarked launches.
* Below those sizes, where the oracle's ARPACK shift-invert solve (exact sparse LU, pinned
  to dense LAPACK) still takes seconds: a heterogeneous cell spanning several tiles
  (N = 16), lowest 20 non-zero eigenvalues to 1e-10, at a generic Bloch vector and at Gamma.
"""

import numpy as np
import pytest

from oracle import oracle as O
from workloads import complex_gaussian, two_phase_sphere
from workloads.materials import TwoPhaseCell

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_03599_gb300 as pc
    return pc


class Grid:
    def __init__(self, pc, cell):
        self.pc = pc
        self.h = pc.pc_grid_create(cell.N, cell.C, cell.rho, phase=cell.phase, theta=cell.theta,
                                   a_lat=cell.a_lat)
        self.C0, self.rho0, self.L = pc.pc_grid_units(self.h)
        self.pb = O.problem_from_cell(cell, C0=self.C0, rho0=self.rho0, L=self.L)
        self.to_si = self.C0 / (self.rho0 * self.L ** 2)

    def close(self):
        self.pc.pc_grid_destroy(self.h)


def _homogeneous_cell(N):
    rng = np.random.default_rng(4)
    G = rng.standard_normal((6, 6))
    C = (G @ G.T + 6 * np.eye(6)) * 1e10
    return TwoPhaseCell(N=N, C=np.stack([C, C]), rho=np.array([2000.0, 2000.0]), phase=None, theta=None,
                        a_lat=np.eye(3))


TOL = {"c128": 1e-12, "c64": 2e-6}


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_four_block_batch_apply_n160_as_benchmarked(pc, dtype):
    """N = 160 (R = 0.3, seed 3), all four parity blocks in one pc_apply_batch launch with
    shift 0.5 at kappa = (0.3, 0.1, 0.2), as the bench times it; per block, random nodes plus
    the quarter grid's faces (the Bloch-wrap paths) against the oracle."""
    import torch
    N = 160
    g = Grid(pc, two_phase_sphere(N, 0.3, 3))
    try:
        kappa = [0.3, 0.1, 0.2]
        pc.pc_set_k(g.h, kappa)
        nb, X = N ** 3 // 4, N // 2
        td = torch.complex64 if dtype == "c64" else torch.complex128
        xs_host = [complex_gaussian((3, nb), 20 + b) for b in range(4)]
        xs = [torch.from_numpy(x.reshape(-1)).to(td).cuda() for x in xs_host]
        ys = [torch.empty_like(x) for x in xs]
        pc.pc_apply_batch(g.h, [0, 1, 2, 3], xs, ys, [0.5] * 4)
        torch.cuda.synchronize()
        rng = np.random.default_rng(12)
        for b in range(4):
            y = ys[b].cpu().numpy().astype(np.complex128).reshape(3, -1)
            t = rng.integers(0, nb, 1000)
            a, bb, k = rng.integers(0, X, 200), rng.integers(0, X, 200), rng.integers(0, N, 200)
            faces = np.concatenate([0 + X * (bb + X * k), (X - 1) + X * (bb + X * k),
                                    a + X * (0 + X * k), a + X * ((X - 1) + X * k),
                                    a + X * (bb + X * 0), a + X * (bb + X * (N - 1))])
            ts = np.unique(np.concatenate([t, faces]))
            ref = O.apply_block_at(g.pb, kappa, b, xs_host[b], ts, 0.5)
            assert np.abs(y[:, ts].T - ref).max() <= TOL[dtype] * np.abs(ref).max(), b
    finally:
        g.close()


@pytest.mark.parametrize("kappa", [[0.3, 0.1, 0.2], [0.0, 0.0, 0.0]])
def test_n48_workload_eigenpairs_pass_the_oracle_residual(pc, kappa):
    import torch
    N, nev = 48, 20
    g = Grid(pc, two_phase_sphere(N, 0.35, 2))
    try:
        evecs = torch.empty(nev * 3 * N ** 3, dtype=torch.complex128, device="cuda")
        ev, blocks, info = pc.pc_eigs(g.h, kappa, nev, evecs=evecs)
        assert np.all(np.diff(ev) >= 0) and np.all(ev > 0)
        V = evecs.cpu().numpy().reshape(nev, 3, -1)
        rho = g.pb.node_rho()
        for i in range(nev):
            lam = ev[i] / g.to_si
            Mv = rho[None, :] * V[i]
            r = O.apply_full(g.pb, kappa, V[i]) - lam * Mv
            assert np.linalg.norm(r) <= 1e-8 * abs(lam) * np.linalg.norm(Mv), i
        W = V.reshape(nev, -1)
        gram = (W.conj() * np.tile(rho, 3)[None, :]) @ W.T
        assert np.abs(gram - np.eye(nev)).max() <= 1e-9
    finally:
        g.close()


def test_n160_precision_cell_mixed_equals_fp64_and_passes_the_oracle_residual(pc):
    """The heterogeneous precision workload (N = 160, R = 0.3, seed 3) at kappa = (0.3, 0.1, 0.2):
    the mixed-precision solve (complex64 inner PCG, FP64 refinement and outer loop) returns the
    FP64 solve's 20 eigenvalues band by band to 1e-10, and FP64 eigenpairs spread over the band
    range pass the oracle's own FP64 residual (1e-8) and M-normalisation."""
    import torch
    N, nev = 160, 20
    kappa = [0.3, 0.1, 0.2]
    g = Grid(pc, two_phase_sphere(N, 0.3, 3))
    try:
        evecs = torch.empty(nev * 3 * N ** 3, dtype=torch.complex128, device="cuda")
        ev64, _, info64 = pc.pc_eigs(g.h, kappa, nev, evecs=evecs)
        evm, _, infom = pc.pc_eigs(g.h, kappa, nev, opt=pc.pc_options_default(precision=pc.PC_PREC_MIXED))
        assert info64["max_rel_resid"] <= 1e-8 and infom["max_rel_resid"] <= 1e-8
        assert np.abs(evm - ev64).max() <= 1e-10 * ev64.max()
        rho = g.pb.node_rho()
        for i in (0, 9, 19):
            v = evecs[i * 3 * N ** 3:(i + 1) * 3 * N ** 3].cpu().numpy().reshape(3, -1)
            lam = ev64[i] / g.to_si
            Mv = rho[None, :] * v
            r = O.apply_full(g.pb, kappa, v) - lam * Mv
            assert np.linalg.norm(r) <= 1e-8 * abs(lam) * np.linalg.norm(Mv), i
            assert abs(np.real(np.vdot(v, Mv)) - 1.0) <= 1e-9
    finally:
        g.close()


_CLOSED_FORM = {}


@pytest.mark.parametrize("N,precision", [(48, "fp64"), (160, "fp64"), (160, "mixed")])
def test_homogeneous_closed_form_at_workload_sizes(pc, N, precision):
    kappa = [0.21, 0.13, 0.05]
    g = Grid(pc, _homogeneous_cell(N))
    try:
        prec = pc.PC_PREC_MIXED if precision == "mixed" else pc.PC_PREC_FP64
        ev, blocks, info = pc.pc_eigs(g.h, kappa, 20, opt=pc.pc_options_default(precision=prec))
        key = (N, tuple(kappa))
        if key not in _CLOSED_FORM:
            _CLOSED_FORM[key] = O.homogeneous_spectrum_planes(g.pb.dims, kappa, g.pb.ainv, g.pb.C[0], g.pb.rho[0])
        cf = _CLOSED_FORM[key][:20] * g.to_si
        assert np.abs(ev - cf).max() / cf.max() <= 1e-10
        assert info["max_rel_resid"] <= 1e-8
    finally:
        g.close()


def test_n48_pcg_with_nan_right_hand_side_reports_enan(pc):
    import torch
    N = 48
    g = Grid(pc, two_phase_sphere(N, 0.35, 2))
    try:
        pc.pc_set_k(g.h, [0.3, 0.1, 0.2])
        rhs = torch.from_numpy(complex_gaussian(3 * N ** 3 // 4, 31)).cuda()
        rhs[1234] = complex(float("nan"), 0.0)
        x = torch.empty_like(rhs)
        r = pc.pc_shift_invert_pcg(g.h, 0, pc.pc_default_sigma(g.h), rhs, x, tol=1e-10, maxit=50,
                                   raise_on_fail=False)
        torch.cuda.synchronize()
        assert r["rc"] == pc.PC_ENAN and r["status"] == pc.PC_ENAN
        assert torch.count_nonzero(x).item() == 0
    finally:
        g.close()


GUARD = 1024  # elements on each side of a guarded vector (keeps 16-byte and larger alignments)
SENTINEL = complex(12345.0, -678.0)


def _guarded(torch, n, dtype):
    buf = torch.full((GUARD + n + GUARD,), SENTINEL, dtype=dtype, device="cuda")
    return buf, buf[GUARD:GUARD + n]


def _guards_intact(buf, n):
    head, tail = buf[:GUARD], buf[GUARD + n:]
    return bool(((head == SENTINEL).all() & (tail == SENTINEL).all()).item())


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_outputs_stay_inside_the_callers_vectors(pc, dtype):
    import torch
    td = torch.complex64 if dtype == "c64" else torch.complex128
    # N = 160: all four blocks in one launch, as the bench times it
    N = 160
    nb = N ** 3 // 4
    g = Grid(pc, two_phase_sphere(N, 0.3, 3))
    try:
        pc.pc_set_k(g.h, [0.3, 0.1, 0.2])
        xs = [torch.from_numpy(complex_gaussian(3 * nb, 40 + b)).to(td).cuda() for b in range(4)]
        guarded = [_guarded(torch, 3 * nb, td) for _ in range(4)]
        pc.pc_apply_batch(g.h, [0, 1, 2, 3], xs, [v for _, v in guarded], [0.5] * 4)
        torch.cuda.synchronize()
        for buf, v in guarded:
            assert _guards_intact(buf, 3 * nb)
            assert bool(torch.isfinite(torch.view_as_real(v)).all().item())
    finally:
        g.close()
    # N = 48: eight vectors of one block in one launch (the solver's batched apply)
    N, count = 48, 8
    nb = N ** 3 // 4
    g = Grid(pc, two_phase_sphere(N, 0.35, 2))
    try:
        pc.pc_set_k(g.h, [0.3, 0.1, 0.2])
        x = torch.from_numpy(complex_gaussian(count * 3 * nb, 50)).to(td).cuda()
        buf, y = _guarded(torch, count * 3 * nb, td)
        pc.pc_block_apply_many(g.h, 2, count, x, y, 0.5)
        torch.cuda.synchronize()
        assert _guards_intact(buf, count * 3 * nb)
        assert bool(torch.isfinite(torch.view_as_real(y)).all().item())
    finally:
        g.close()


@pytest.mark.parametrize("kappa", [[0.3, 0.1, 0.2], [0.0, 0.0, 0.0]])
def test_n16_heterogeneous_eigenvalues_match_the_arpack_oracle(pc, kappa):
    N, nev, per_block = 16, 20, 12
    g = Grid(pc, two_phase_sphere(N, 0.35, 2))
    try:
        ev, blocks, info = pc.pc_eigs(g.h, kappa, nev)
        assert info["max_rel_resid"] <= 1e-8
        sigma = pc.pc_default_sigma(g.h)
        parts = [O.eigs_oracle(g.pb, kappa, per_block, sigma=sigma, b=b) for b in range(4)]
        union = np.sort(np.concatenate(parts))[:nev]
        # every block's computed eigenvalues reach past the union's 20th: the reference is complete
        assert all(p.max() >= union[-1] for p in parts)
        ref = union * g.to_si
        assert np.abs(ev - ref).max() / ref.max() <= 1e-10
    finally:
        g.close()
