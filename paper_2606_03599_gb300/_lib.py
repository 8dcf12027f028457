"""ctypes binding of ``libpcband.so``: argument marshalling only.

Every function mirrors the C entry point of the same name declared in
``include/pcband.h``; status codes become exceptions.  Device vectors are
passed as torch CUDA tensors (or raw integer device addresses); nothing here
computes any part of the method.  A missing library raises at import.
"""

from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpcband.so")

PC_OK, PC_EINVAL, PC_ENOMEM, PC_ECUDA, PC_ENOCONV, PC_EBREAKDOWN, PC_ENAN, PC_ESTATE = \
    0, -1, -2, -3, -4, -5, -6, -7
PC_C64, PC_C128 = 1, 2
PC_PREC_FP64, PC_PREC_MIXED = 0, 1

EXPORTED = [
    "pc_grid_create", "pc_grid_destroy", "pc_grid_units", "pc_set_k", "pc_block_index",
    "pc_block_apply", "pc_block_apply_many", "pc_block_mass", "pc_block_transfer",
    "pc_block_fourier", "pc_block_precond", "pc_shift_invert_pcg", "pc_options_default", "pc_default_sigma",
    "pc_eigs", "pc_last_error", "pc_version", "pc_apply_batch", "pc_stats_timing", "pc_stats_reset",
    "pc_stats_get", "pc_block_apply_dot_noalloc", "pc_eig_grad", "pc_autotune", "pc_tuned_config",
    "pc_grid_clone", "pc_eigs_batch", "pc_device_status", "pc_fp64_peak", "pc_grid_create_nodewise",
    "pc_eigs_multi", "pc_eigs_multi_max", "pc_set_k_multi", "pc_apply_batch_k",
]


class PcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (status %d)" % (msg, code))
        self.code = code


class PcNoConvergence(PcError):
    pass


class PcBreakdown(PcError):
    pass


class c_material(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double * 2), ("C", (ctypes.c_double * 36) * 2),
                ("phase", ctypes.POINTER(ctypes.c_uint8)), ("theta", ctypes.POINTER(ctypes.c_float)),
                ("a_lat", ctypes.c_double * 9)]


class c_pcg_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("rel_resid", ctypes.c_double)]


class c_options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("inner_tol", ctypes.c_double), ("precision", ctypes.c_int),
                ("full_space", ctypes.c_int), ("block_size", ctypes.c_int), ("max_basis", ctypes.c_int),
                ("max_restarts", ctypes.c_int), ("inner_maxit", ctypes.c_int), ("guard", ctypes.c_int),
                ("verbose", ctypes.c_int), ("stream", ctypes.c_void_p), ("autotune", ctypes.c_int),
                ("precond_fp32", ctypes.c_int), ("kbatch", ctypes.c_int)]


class c_batch_job(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_void_p), ("nk", ctypes.c_int), ("kappas", ctypes.POINTER(ctypes.c_double)),
                ("nev", ctypes.c_int), ("sigma", ctypes.c_double), ("evals", ctypes.POINTER(ctypes.c_double)),
                ("block_of", ctypes.POINTER(ctypes.c_int)), ("status", ctypes.POINTER(ctypes.c_int))]


class c_batch_info(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int), ("kpoints", ctypes.c_int), ("failed", ctypes.c_int),
                ("pcg_iters", ctypes.c_longlong), ("max_rel_resid", ctypes.c_double), ("seconds", ctypes.c_double)]


class c_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("apply_launches", ctypes.c_longlong),
                ("apply_timed", ctypes.c_longlong * 2), ("apply_ms", ctypes.c_double * 2),
                ("apply_nodes", ctypes.c_double * 2),
                ("apply_nodes_launched", ctypes.c_double * 2)]


class c_eigs_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_iters", ctypes.c_int), ("inner_solves", ctypes.c_int),
                ("pcg_iters", ctypes.c_longlong), ("max_pcg_iters", ctypes.c_int),
                ("zero_modes", ctypes.c_int), ("max_rel_resid", ctypes.c_double),
                ("seconds", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libpcband.so is not built: run __graft_entry__.build() "
                          "(or python -m paper_2606_03599_gb300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "pc_grid_create": ([ci, ctypes.POINTER(c_material), ctypes.POINTER(vp)], ci),
        "pc_grid_destroy": ([vp], ci),
        "pc_grid_units": ([vp, dp, dp, dp], ci),
        "pc_set_k": ([vp, dp], ci),
        "pc_block_index": ([ci, ci, ctypes.POINTER(ctypes.c_int64)], ci),
        "pc_block_apply": ([vp, ci, ci, vp, vp, cd, vp], ci),
        "pc_block_apply_many": ([vp, ci, ci, ci, vp, vp, cd, vp], ci),
        "pc_block_mass": ([vp, ci, ci, vp, vp, vp], ci),
        "pc_block_transfer": ([vp, ci, ci, ci, vp, vp, vp], ci),
        "pc_block_fourier": ([vp, ci, ci, ci, vp, vp, vp], ci),
        "pc_block_precond": ([vp, ci, ci, ci, cd, vp, vp, vp], ci),
        "pc_shift_invert_pcg": ([vp, ci, ci, cd, vp, vp, cd, ci, ctypes.POINTER(c_pcg_info), vp], ci),
        "pc_options_default": ([ctypes.POINTER(c_options)], ci),
        "pc_default_sigma": ([vp], cd),
        "pc_eigs": ([vp, dp, ci, cd, ctypes.POINTER(c_options), dp, vp, ctypes.POINTER(ci),
                     ctypes.POINTER(c_eigs_info)], ci),
        "pc_eigs_multi": ([vp, ci, dp, ci, cd, ctypes.POINTER(c_options), dp, vp, ctypes.POINTER(ci),
                           ctypes.POINTER(c_eigs_info)], ci),
        "pc_eigs_multi_max": ([vp], ci),
        "pc_set_k_multi": ([vp, ci, dp], ci),
        "pc_apply_batch_k": ([vp, ci, ci, ctypes.POINTER(ci), ctypes.POINTER(ci), ctypes.POINTER(vp),
                              ctypes.POINTER(vp), dp, vp], ci),
        "pc_apply_batch": ([vp, ci, ci, ctypes.POINTER(ci), ctypes.POINTER(vp), ctypes.POINTER(vp), dp, vp], ci),
        "pc_block_apply_dot_noalloc": ([vp, ci, ci, vp, vp, cd, vp, vp], ci),
        "pc_eig_grad": ([vp, ci, ci, vp, dp, dp, vp, vp, vp], ci),
        "pc_autotune": ([vp, ci, ci, ci, vp], ci),
        "pc_grid_clone": ([vp, ctypes.POINTER(vp)], ci),
        "pc_eigs_batch": ([ctypes.POINTER(c_batch_job), ci, ctypes.POINTER(c_options), ci,
                           ctypes.POINTER(c_batch_info)], ci),
        "pc_tuned_config": ([vp, ci, ci, ci] + [ctypes.POINTER(ci)] * 4, ci),
        "pc_stats_timing": ([ci], ci),
        "pc_stats_reset": ([], ci),
        "pc_stats_get": ([ctypes.POINTER(c_stats)], ci),
        "pc_device_status": ([vp, vp], ci),
        "pc_grid_create_nodewise": ([ci, dp, dp, dp, ctypes.POINTER(vp)], ci),
        "pc_fp64_peak": ([cd, dp, dp], ci),
        "pc_last_error": ([], ctypes.c_char_p),
        "pc_version": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()


def _check(rc):
    if rc == PC_OK:
        return
    msg = lib.pc_last_error().decode()
    if rc == PC_ENOCONV:
        raise PcNoConvergence(rc, msg)
    if rc == PC_EBREAKDOWN:
        raise PcBreakdown(rc, msg)
    raise PcError(rc, msg)


def _ptr(t):
    """Device address of a torch tensor (or an int address)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("vector arguments must be contiguous")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dtype_code(t):
    import torch
    if t.dtype == torch.complex64:
        return PC_C64
    if t.dtype == torch.complex128:
        return PC_C128
    raise TypeError("vectors must be complex64 or complex128")


def make_material(C, rho, phase=None, theta=None, a_lat=None):
    """pc_material from per-phase stiffness (2,6,6) Pa, densities (2,), optional phase/theta arrays.

    Returns (struct, keepalive) -- keep ``keepalive`` referenced until the create call returns.
    """
    m = c_material()
    C = np.asarray(C, dtype=np.float64).reshape(2, 36)
    for p in range(2):
        m.rho[p] = float(rho[p])
        for e in range(36):
            m.C[p][e] = float(C[p, e])
    keep = []
    if phase is not None:
        ph = np.ascontiguousarray(np.asarray(phase, dtype=np.uint8))
        keep.append(ph)
        m.phase = ph.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    if theta is not None:
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float32))
        keep.append(th)
        m.theta = th.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    A = np.eye(3) if a_lat is None else np.asarray(a_lat, dtype=np.float64)
    for l in range(3):
        for r in range(3):
            m.a_lat[3 * l + r] = float(A[r, l])
    return m, keep


def pc_grid_create(N, C, rho, phase=None, theta=None, a_lat=None):
    m, keep = make_material(C, rho, phase, theta, a_lat)
    h = ctypes.c_void_p()
    _check(lib.pc_grid_create(int(N), ctypes.byref(m), ctypes.byref(h)))
    del keep
    return h.value


def pc_grid_create_nodewise(N, C21, rho, a_lat=None):
    """Grid with a nodewise material: C21 (N^3, 21) upper-triangular Voigt entries per node (Pa, row
    order p <= r), rho (N^3,) kg/m^3, both in full-grid node order; host arrays (numpy or CPU tensors)."""
    C21 = np.ascontiguousarray(np.asarray(C21, dtype=np.float64))
    rho = np.ascontiguousarray(np.asarray(rho, dtype=np.float64))
    n = int(N) ** 3
    if C21.shape != (n, 21) or rho.shape != (n,):
        raise ValueError("C21 must be (N^3, 21) and rho (N^3,)")
    A = np.eye(3) if a_lat is None else np.asarray(a_lat, dtype=np.float64)
    a = np.ascontiguousarray(A.T.reshape(9))  # column-major
    dp = ctypes.POINTER(ctypes.c_double)
    h = ctypes.c_void_p()
    _check(lib.pc_grid_create_nodewise(int(N), C21.ctypes.data_as(dp), rho.ctypes.data_as(dp), a.ctypes.data_as(dp),
                                       ctypes.byref(h)))
    return h.value


def pc_grid_destroy(g):
    _check(lib.pc_grid_destroy(g))


def pc_grid_units(g):
    c0, r0, L = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib.pc_grid_units(g, ctypes.byref(c0), ctypes.byref(r0), ctypes.byref(L)))
    return c0.value, r0.value, L.value


def pc_set_k(g, kappa):
    k = (ctypes.c_double * 3)(*[float(v) for v in kappa])
    _check(lib.pc_set_k(g, k))


def pc_block_index(N, block):
    out = np.empty(int(N) ** 3 // 4, dtype=np.int64)
    _check(lib.pc_block_index(int(N), int(block), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return out


def pc_block_apply(g, block, x, y, shift=0.0, stream=None):
    _check(lib.pc_block_apply(g, int(block), _dtype_code(x), _ptr(x), _ptr(y), float(shift),
                              _stream(stream)))


def pc_block_apply_many(g, block, count, x, y, shift=0.0, stream=None):
    _check(lib.pc_block_apply_many(g, int(block), _dtype_code(x), int(count), _ptr(x), _ptr(y),
                                   float(shift), _stream(stream)))


def pc_block_mass(g, block, x, y, stream=None):
    _check(lib.pc_block_mass(g, int(block), _dtype_code(x), _ptr(x), _ptr(y), _stream(stream)))


def pc_block_transfer(g, block, direction, src, dst, stream=None):
    _check(lib.pc_block_transfer(g, int(block), _dtype_code(src), int(direction), _ptr(src), _ptr(dst),
                                 _stream(stream)))


def pc_block_fourier(g, block, inverse, w, what, stream=None):
    _check(lib.pc_block_fourier(g, int(block), _dtype_code(w), int(inverse), _ptr(w), _ptr(what),
                                _stream(stream)))


def pc_block_precond(g, block, sigma, r, z, fp32_transforms=False, stream=None):
    """z = P_ref r (reference-medium preconditioner, Sec. 5.4); block -1 = full space."""
    _check(lib.pc_block_precond(g, int(block), _dtype_code(r), int(bool(fp32_transforms)), float(sigma), _ptr(r),
                                _ptr(z), _stream(stream)))


def pc_shift_invert_pcg(g, block, sigma, rhs, x, tol=1e-10, maxit=400, stream=None, raise_on_fail=True):
    info = c_pcg_info()
    rc = lib.pc_shift_invert_pcg(g, int(block), _dtype_code(rhs), float(sigma), _ptr(rhs), _ptr(x),
                                 float(tol), int(maxit), ctypes.byref(info), _stream(stream))
    if raise_on_fail:
        _check(rc)
    return {"rc": rc, "iters": info.iters, "status": info.status, "rel_resid": info.rel_resid}


def pc_options_default(**overrides):
    o = c_options()
    _check(lib.pc_options_default(ctypes.byref(o)))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def pc_default_sigma(g):
    return float(lib.pc_default_sigma(g))


def pc_eigs(g, kappa, nev, sigma=float("nan"), opt=None, evecs=None, raise_on_fail=True):
    """Returns (evals SI ascending, block_of, info dict)."""
    opt = opt if opt is not None else pc_options_default()
    k = (ctypes.c_double * 3)(*[float(v) for v in kappa])
    ev = np.empty(int(nev), dtype=np.float64)
    bo = (ctypes.c_int * int(nev))()
    info = c_eigs_info()
    rc = lib.pc_eigs(g, k, int(nev), float(sigma), ctypes.byref(opt),
                     ev.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(evecs), bo,
                     ctypes.byref(info))
    if raise_on_fail:
        _check(rc)
    d = {f: getattr(info, f) for f, _ in c_eigs_info._fields_}
    d["rc"] = rc
    return ev, np.array(list(bo)), d


def pc_eigs_multi(g, kappas, nev, sigma=float("nan"), opt=None, evecs=None, raise_on_fail=True):
    """Several Bloch vectors of one grid in lockstep.  Returns (evals [nk][nev], block_of [nk][nev],
    list of per-vector info dicts); evecs: optional device complex128 buffer of nk * nev * 3 N^3."""
    ks = np.ascontiguousarray(np.asarray(kappas, dtype=np.float64).reshape(-1, 3))
    nk = ks.shape[0]
    opt = opt if opt is not None else pc_options_default()
    ev = np.empty((nk, int(nev)), dtype=np.float64)
    bo = np.empty((nk, int(nev)), dtype=np.int32)
    infos = (c_eigs_info * nk)()
    rc = lib.pc_eigs_multi(g, nk, ks.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(nev), float(sigma),
                           ctypes.byref(opt), ev.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(evecs),
                           bo.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), infos)
    if raise_on_fail:
        _check(rc)
    out = []
    for i in range(nk):
        d = {f: getattr(infos[i], f) for f, _ in c_eigs_info._fields_}
        d["rc"] = rc
        out.append(d)
    return ev, bo, out


def pc_set_k_multi(g, kappas):
    """Bloch slots 0 .. nk - 1 of the grid at the reduced vectors kappas ([nk][3])."""
    ks = np.ascontiguousarray(np.asarray(kappas, dtype=np.float64).reshape(-1, 3))
    _check(lib.pc_set_k_multi(g, ks.shape[0], ks.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))


def pc_apply_batch_k(g, blocks, kslots, xs, ys, shifts, stream=None):
    """pc_apply_batch with each item at the Bloch vector of its slot."""
    n = len(blocks)
    bl = (ctypes.c_int * n)(*[int(b) for b in blocks])
    kl = (ctypes.c_int * n)(*[int(k) for k in kslots])
    xp = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    yp = (ctypes.c_void_p * n)(*[_ptr(y) for y in ys])
    sh = (ctypes.c_double * n)(*[float(v) for v in shifts])
    _check(lib.pc_apply_batch_k(g, _dtype_code(xs[0]), n, bl, kl, xp, yp, sh, _stream(stream)))


def pc_eigs_multi_max(g):
    """Largest number of Bloch vectors pc_eigs_multi solves together on this grid."""
    r = int(lib.pc_eigs_multi_max(g))
    if r < 0:
        _check(r)
    return r


def pc_apply_batch(g, blocks, xs, ys, shifts, stream=None):
    n = len(blocks)
    bl = (ctypes.c_int * n)(*[int(b) for b in blocks])
    xp = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    yp = (ctypes.c_void_p * n)(*[_ptr(y) for y in ys])
    sh = (ctypes.c_double * n)(*[float(v) for v in shifts])
    _check(lib.pc_apply_batch(g, _dtype_code(xs[0]), n, bl, xp, yp, sh, _stream(stream)))


def pc_block_apply_dot_noalloc(g, block, x, y, dot, shift=0.0, stream=None):
    """y = (A - shift M) x and dot[0] = Re <x, y> without any device allocation by the library.

    ``dot`` is a caller-owned device tensor holding one float64.
    """
    import torch
    if not (isinstance(dot, torch.Tensor) and dot.is_cuda and dot.dtype == torch.float64 and dot.numel() >= 1):
        raise ValueError("dot must be a float64 CUDA tensor with at least one element")
    if x.dtype != y.dtype or x.numel() != y.numel():
        raise ValueError("x and y must have the same dtype and size")
    _check(lib.pc_block_apply_dot_noalloc(g, int(block), _dtype_code(x), _ptr(x), _ptr(y), float(shift),
                                          _ptr(dot), _stream(stream)))


def pc_fp64_peak(seconds=0.5):
    """Measured FP64 FMA throughput of the current device: (TFLOP/s, FMA instructions/s)."""
    t, f = ctypes.c_double(), ctypes.c_double()
    _check(lib.pc_fp64_peak(float(seconds), ctypes.byref(t), ctypes.byref(f)))
    return t.value, f.value


def pc_device_status(g, stream=None):
    """Synchronise the stream and raise PcError (PC_ECUDA) if a kernel's bounded copy wait expired."""
    _check(lib.pc_device_status(g, _stream(stream)))


def pc_eig_grad(g, block, X, lambdas, weights, dC, drho, stream=None):
    """Accumulate weighted eigenvalue gradients into dC ([21, n] float64 device) and drho ([n])."""
    lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64))
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    _check(lib.pc_eig_grad(g, int(block), int(lam.size), _ptr(X),
                           lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(dC), _ptr(drho),
                           _stream(stream)))


def pc_grid_clone(g):
    h = ctypes.c_void_p()
    _check(lib.pc_grid_clone(g, ctypes.byref(h)))
    return h.value


def pc_eigs_batch(grids, kappas, nev, opt=None, workers=4, sigma=float("nan"), raise_on_noconv=True):
    """Solve every (grid, Bloch vector): grids is a list of handles, kappas a list of [nk][3] arrays.
    Returns (evals list of [nk][nev] arrays, block_of list, status list, info dict)."""
    n = len(grids)
    jobs = (c_batch_job * n)()
    keep = []
    out_ev, out_bl, out_st = [], [], []
    for j, (g, ks) in enumerate(zip(grids, kappas)):
        ks = np.ascontiguousarray(np.asarray(ks, dtype=np.float64).reshape(-1, 3))
        ev = np.zeros((ks.shape[0], nev))
        bl = np.zeros((ks.shape[0], nev), dtype=np.int32)
        st = np.zeros(ks.shape[0], dtype=np.int32)
        keep += [ks, ev, bl, st]
        out_ev.append(ev)
        out_bl.append(bl)
        out_st.append(st)
        jobs[j].grid = g
        jobs[j].nk = ks.shape[0]
        jobs[j].kappas = ks.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        jobs[j].nev = int(nev)
        jobs[j].sigma = float(sigma)
        jobs[j].evals = ev.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        jobs[j].block_of = bl.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        jobs[j].status = st.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    o = opt if opt is not None else pc_options_default()
    info = c_batch_info()
    rc = lib.pc_eigs_batch(jobs, n, ctypes.byref(o), int(workers), ctypes.byref(info))
    if rc != PC_OK and (rc != PC_ENOCONV or raise_on_noconv):
        _check(rc)
    d = {f[0]: getattr(info, f[0]) for f in c_batch_info._fields_}
    return out_ev, out_bl, out_st, d


def pc_autotune(g, dtype, layout, nitems, stream=None):
    """Time the stencil launch shapes for batches of `nitems` (layout 0 blocks, 1 full, 2 both)."""
    _check(lib.pc_autotune(g, int(dtype), int(layout), int(nitems), _stream(stream)))


def pc_tuned_config(g, dtype, layout, nitems):
    """(kind, shape, tz, ctas) of the launch the library uses; kind 0 registers, 1 TMA tile, 2 row, 3 two-pass."""
    v = [ctypes.c_int() for _ in range(4)]
    _check(lib.pc_tuned_config(g, int(dtype), int(layout), int(nitems), *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def pc_stats_timing(enable):
    _check(lib.pc_stats_timing(int(bool(enable))))


def pc_stats_reset():
    _check(lib.pc_stats_reset())


def pc_stats_get():
    st = c_stats()
    _check(lib.pc_stats_get(ctypes.byref(st)))
    return {"launches": st.launches, "apply_launches": st.apply_launches,
            "apply_timed": list(st.apply_timed), "apply_ms": list(st.apply_ms),
            "apply_nodes": list(st.apply_nodes),
            "apply_nodes_launched": list(st.apply_nodes_launched)}


def pc_version():
    return lib.pc_version().decode()


def nan():
    return math.nan
