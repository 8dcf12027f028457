"""The fused stencil kernel's tile logic, run by the host emulator, against the oracle (CPU only).

The emulator executes the kernel's own per-thread phase functions for every
simulated thread of every CTA, with bounds checks on each shared-memory and
global access, so these tests check the tiling, halo, chunking and Bloch-wrap
arithmetic of the CUDA kernel without a GPU.
"""

import ctypes
import importlib.util
import os

import numpy as np
import pytest

from oracle import oracle as O
from oracle.oracle import Problem
from workloads import complex_gaussian, two_phase_sphere

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def emu():
    spec = importlib.util.spec_from_file_location(
        "pcband_build", os.path.join(ROOT, "paper_2606_03599_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    lib = ctypes.CDLL(mod.build_emulator())
    dp = ctypes.POINTER(ctypes.c_double)
    lib.pc_emu_apply.argtypes = [ctypes.c_int] * 5 + [dp, dp, dp, ctypes.c_int, dp, ctypes.c_void_p,
                                                      ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                      ctypes.c_double]
    lib.pc_emu_apply.restype = ctypes.c_int
    return lib


def run_emu(lib, pb, block, dtype, shape, tz, kappa, x, shift, matkind):
    N = pb.dims[0]
    dp = ctypes.POINTER(ctypes.c_double)
    Chat = np.ascontiguousarray(pb.C.reshape(72))
    rho = np.ascontiguousarray(pb.rho)
    ainv = np.ascontiguousarray(pb.ainv.reshape(9))
    cubic = int(np.abs(pb.ainv - np.eye(3)).max() < 1e-12)
    phi = np.ascontiguousarray(2 * np.pi * (np.asarray(kappa, dtype=float) - np.floor(kappa)))
    th = pb.theta if block < 0 else pb.theta[O.block_index(pb.dims, block)]
    mat = np.ascontiguousarray(th.astype(np.float32) if matkind else th.astype(np.uint8))
    ct = np.complex64 if dtype == 1 else np.complex128
    xx = np.ascontiguousarray(x.astype(ct))
    y = np.zeros_like(xx)
    f = lambda a: a.ctypes.data_as(dp)  # noqa: E731
    rc = lib.pc_emu_apply(N, block, dtype, shape, tz, f(Chat), f(rho), f(ainv), cubic, f(phi),
                          mat.ctypes.data, matkind, xx.ctypes.data, y.ctypes.data, shift)
    assert rc == 0
    return y


CASES = [
    # N, block, dtype, shape, tz
    (4, 0, 2, 3, 1), (4, 3, 2, 3, 4), (4, -1, 2, 3, 3),
    (8, 1, 2, 3, 3), (8, 2, 1, 3, 2), (8, -1, 2, 2, 5), (8, 3, 2, 2, 8),
    (12, 0, 2, 1, 5), (12, 2, 1, 0, 4), (12, -1, 2, 2, 7),
    # TMA-staged kernel (codes 10: 16x16 / 16x8 tiles, 11: 8x8 tiles)
    (16, 0, 1, 10, 3), (16, 3, 2, 10, 5), (16, -1, 1, 10, 4), (16, 1, 2, 11, 16),
    (8, 2, 1, 11, 2), (8, -1, 2, 11, 3), (12, 1, 1, 11, 6), (4, 0, 2, 11, 4), (20, 3, 1, 10, 7),
    # row-tile kernel (code 20, complex64 blocks; tz = persistent CTAs): single tile with both row
    # wraps, several tiles (N >= 48), ragged tile heights (N = 68: 11, 11, 12 rows), CTA ranges that
    # split tiles, and more CTAs than planes
    (4, 0, 1, 20, 1), (4, 3, 1, 20, 5), (8, 1, 1, 20, 3), (8, 2, 1, 20, 64), (12, 3, 1, 20, 7),
    (16, 0, 1, 20, 2), (20, 2, 1, 20, 9), (48, 1, 1, 20, 13), (56, 3, 1, 20, 40), (68, 0, 1, 20, 17),
    # row-tile kernel with compile-time widths (code 21): X = 16, 24, 32 (N = 32, 48, 64)
    (32, 2, 1, 21, 5), (48, 0, 1, 21, 152), (64, 3, 1, 21, 31),
    # plane-pipelined kernel (code 40, complex64 blocks; tz = persistent CTAs): one tile with both
    # row wraps, several tiles, ragged tile heights, CTA ranges that split tiles, more CTAs than
    # planes; code 41: compile-time widths X = 16, 24, 32; codes 51-53: 1, 2, 3 thread rows (tiles
    # of 1, 3, 5 rows, so that most tiles touch a wrap or a neighbour tile)
    (4, 0, 1, 40, 1), (4, 3, 1, 40, 5), (8, 1, 1, 40, 3), (8, 2, 1, 40, 64), (12, 3, 1, 40, 7),
    (16, 0, 1, 40, 2), (20, 2, 1, 40, 9), (48, 1, 1, 40, 13), (56, 3, 1, 40, 40), (68, 0, 1, 40, 17),
    (32, 2, 1, 41, 5), (48, 0, 1, 41, 152), (64, 3, 1, 41, 31),
    (4, 1, 1, 51, 3), (12, 2, 1, 51, 5), (20, 2, 1, 52, 9), (24, 1, 1, 51, 11), (28, 3, 1, 53, 6),
    # two-pass complex128 kernels (code 30): every block, the full grid, the smallest grids
    (4, 0, 2, 30, 0), (4, 3, 2, 30, 0), (4, -1, 2, 30, 0), (8, 1, 2, 30, 0), (8, 2, 2, 30, 0),
    (8, -1, 2, 30, 0), (12, 3, 2, 30, 0), (16, 0, 2, 30, 0),
    (8, 1, 1, 30, 0), (12, -1, 1, 30, 0), (16, 2, 1, 30, 0),
    # odd quarter-grid widths (X = N/2 = 3, 5, 7): two-pass and register-staged kernels
    (6, 3, 2, 30, 0), (10, 1, 2, 30, 0), (10, -1, 2, 30, 0), (14, 2, 1, 30, 0),
    (6, 0, 2, 3, 2), (10, 2, 1, 3, 3), (14, -1, 2, 2, 5), (10, 3, 2, 1, 4),
]


@pytest.mark.parametrize("N,block,dtype,shape,tz", CASES)
@pytest.mark.parametrize("kappa", [[0.3, 0.1, 0.2], [0.0, 0.0, 0.0], [1.3, 0.1, -0.8]])
def test_emulated_kernel_matches_oracle(emu, N, block, dtype, shape, tz, kappa):
    pb = O.problem_from_cell(two_phase_sphere(N, 0.35, 1), C0=1e9, rho0=1e3)
    m = N ** 3 // 4 if block >= 0 else N ** 3
    x = complex_gaussian((3, m), 7)
    ref = (O.apply_block(pb, kappa, block, x, shift=0.37) if block >= 0
           else O.apply_full(pb, kappa, x, shift=0.37))
    y = run_emu(emu, pb, block, dtype, shape, tz, kappa, x, 0.37, 0)
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err < (1e-13 if dtype == 2 else 2e-6)


@pytest.mark.parametrize("block", [1, -1])
def test_emulated_kernel_general_lattice_and_fractions(emu, block):
    """Non-cubic (FCC) lattice mixing and fractional (sub-pixel) material."""
    N = 8
    cell = two_phase_sphere(N, 0.3, 2)
    A = np.array([[0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]])
    Ah = A / abs(np.linalg.det(A)) ** (1 / 3)
    theta = np.random.default_rng(0).uniform(0, 1, N ** 3).astype(np.float32).astype(np.float64)
    pb = Problem(dims=(N,) * 3, ainv=np.linalg.inv(Ah), C=cell.C / 1e9, rho=cell.rho / 1e3, theta=theta)
    kappa = [0.21, -0.33, 0.4]
    m = N ** 3 // 4 if block >= 0 else N ** 3
    x = complex_gaussian((3, m), 9)
    ref = (O.apply_block(pb, kappa, block, x, shift=0.5) if block >= 0
           else O.apply_full(pb, kappa, x, shift=0.5))
    for dtype, shape, tz in ((2, 2, 3), (1, 3, 4), (2, 11, 5), (1, 10, 3), (1, 20, 3), (1, 40, 3), (1, 52, 5),
                             (2, 30, 0)):
        if shape in (20, 40, 52) and block < 0:
            continue
        y = run_emu(emu, pb, block, dtype, shape, tz, kappa, x, 0.5, 1)
        err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
        assert err < (1e-13 if dtype == 2 else 2e-6)


@pytest.mark.parametrize("block", [2, -1])
@pytest.mark.parametrize("lattice", ["cubic", "fcc"])
def test_emulated_two_pass_nodewise_material(emu, block, lattice):
    """Nodewise material (every node its own symmetric stiffness and density) in the two-pass
    complex128 kernels, against the oracle's nodewise pencil."""
    N = 8
    n = N ** 3
    rng = np.random.default_rng(5)
    cell = two_phase_sphere(N, 0.35, 3)
    base = O.problem_from_cell(cell, C0=1e9, rho0=1e3)
    G = rng.standard_normal((n, 6, 6))
    Cn = base.node_C() + 0.1 * (G + np.transpose(G, (0, 2, 1)))
    rn = base.node_rho() * (1.0 + 0.2 * rng.uniform(size=n))
    A = np.eye(3) if lattice == "cubic" else np.array([[0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]])
    Ah = A / abs(np.linalg.det(A)) ** (1 / 3)
    pb = Problem(dims=(N,) * 3, ainv=np.linalg.inv(Ah), C=base.C, rho=base.rho, theta=base.theta,
                 C_nodes=Cn, rho_nodes=rn)
    kappa = [0.21, -0.33, 0.4]
    m = n // 4 if block >= 0 else n
    x = complex_gaussian((3, m), 11)
    # the oracle's sparse pencil reads the nodewise material (its C apply takes two phases only)
    A, M = O.sparse_pencil(pb, kappa, block if block >= 0 else None)
    ref = ((A - 0.7 * M) @ x.reshape(-1)).reshape(3, m)
    # the library's device layout: [22][m], the 21 upper entries times (N/4)^2 on a cubic lattice
    iu = np.triu_indices(6)
    q2 = (N / 4.0) ** 2 if lattice == "cubic" else 1.0
    lay = np.concatenate([Cn[:, iu[0], iu[1]].T * q2, rn[None, :]], axis=0)
    if block >= 0:
        lay = lay[:, O.block_index(pb.dims, block)]
    mat = np.ascontiguousarray(lay)
    dp = ctypes.POINTER(ctypes.c_double)
    Chat = np.ascontiguousarray(base.C.reshape(72))
    rho = np.ascontiguousarray(base.rho)
    ainv = np.ascontiguousarray(pb.ainv.reshape(9))
    phi = np.ascontiguousarray(2 * np.pi * (np.asarray(kappa, dtype=float) - np.floor(kappa)))
    xx = np.ascontiguousarray(x.astype(np.complex128))
    y = np.zeros_like(xx)
    f = lambda a: a.ctypes.data_as(dp)  # noqa: E731
    rc = emu.pc_emu_apply(N, block, 2, 30, 0, f(Chat), f(rho), f(ainv), int(lattice == "cubic"), f(phi),
                          mat.ctypes.data, 2, xx.ctypes.data, y.ctypes.data, 0.7)
    assert rc == 0
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err < 1e-13


@pytest.mark.parametrize("L", list(range(1, 17)))
def test_small_dft_with_compile_time_roots_matches_numpy(emu, L):
    """The L-point DFT inside the Bloch transform kernels (roots from constant expressions, paired
    inputs) equals numpy's FFT, forward and unnormalised inverse, to rounding."""
    rng = np.random.default_rng(L)
    v = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    fn = emu.pc_emu_small_dft
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    fn.restype = ctypes.c_int
    for inv, ref in ((0, np.fft.fft(v)), (1, np.fft.ifft(v) * L)):
        inp = np.ascontiguousarray(np.stack([v.real, v.imag], axis=1).reshape(-1))
        out = np.zeros(2 * L)
        assert fn(L, inv, inp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == 0
        got = out[0::2] + 1j * out[1::2]
        assert np.abs(got - ref).max() <= 4e-16 * L * np.abs(v).sum()


@pytest.mark.parametrize("dims", [(2, 2, 4), (3, 4, 6), (24, 24, 48), (30, 30, 60), (5, 7, 3)])
def test_ghost_cell_numbering_is_a_bijection_with_its_inverse(emu, dims):
    """The two-pass kernels number the one-cell ghost layer around the grid (planes, then rows,
    then columns); the flux pass finds a wrapped neighbour's cell by the inverse map.  Every layer
    cell is numbered exactly once, no interior cell is, and the inverse returns the number."""
    fn = emu.pc_emu_ghost_cells
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    fn.restype = ctypes.c_longlong
    assert fn(*dims) == 0
