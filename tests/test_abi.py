"""C-ABI checks that need no GPU: the library loads, exports every declared symbol,
its host-side index map is bit-exact, and argument errors are reported."""

import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "pcband.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pc_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def pc():
    import paper_2606_03599_gb300 as pc
    return pc


def test_library_exports_every_declared_symbol(pc):
    names = _declared_symbols()
    assert len(names) >= 15
    for name in names:
        assert hasattr(pc.lib, name), name
    assert set(names) == set(pc.EXPORTED)


@pytest.mark.parametrize("N", [4, 6, 8, 12])
def test_block_index_bit_exact(pc, N):
    for b in range(4):
        assert np.array_equal(pc.pc_block_index(N, b), O.block_index((N, N, N), b))


def test_block_index_rejects_bad_arguments(pc):
    out = np.empty(64, dtype=np.int64)
    p = out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    assert pc.lib.pc_block_index(5, 0, p) == pc.PC_EINVAL
    assert "even" in pc.lib.pc_last_error().decode()
    assert pc.lib.pc_block_index(2, 0, p) == pc.PC_EINVAL
    assert pc.lib.pc_block_index(8, 4, p) == pc.PC_EINVAL
    assert pc.lib.pc_block_index(8, 0, None) == pc.PC_EINVAL


def test_options_defaults(pc):
    o = pc.pc_options_default()
    assert o.tol == 1e-8 and o.block_size == 2 and o.precision == pc.PC_PREC_FP64
    assert o.max_basis == 24 and o.kbatch == 0 and o.precond_fp32 == 1


def test_lockstep_entry_points_reject_bad_arguments(pc):
    import ctypes as ct
    k = (ct.c_double * 6)(0, 0, 0, 0.5, 0, 0)
    ev = (ct.c_double * 8)()
    assert pc.lib.pc_eigs_multi(None, 2, k, 4, float("nan"), None, ev, None, None, None) == pc.PC_EINVAL
    assert pc.lib.pc_set_k_multi(None, 2, k) == pc.PC_EINVAL
    assert pc.lib.pc_eigs_multi_max(None) == pc.PC_EINVAL
    assert pc.lib.pc_apply_batch_k(None, pc.PC_C64, 0, None, None, None, None, None, None) == pc.PC_EINVAL


def test_null_grid_is_rejected(pc):
    assert pc.lib.pc_set_k(None, None) == pc.PC_EINVAL
    assert pc.lib.pc_block_apply(None, 0, pc.PC_C64, None, None, 0.0, None) == pc.PC_EINVAL
    assert pc.lib.pc_grid_destroy(None) == pc.PC_OK


def test_stats_counters_need_no_device(pc):
    """The launch and apply counters reset and read back on a host without a GPU (no apply has run,
    so nothing was counted on a device): every counter is zero after a reset."""
    pc.pc_stats_reset()
    st = pc.pc_stats_get()
    assert st["launches"] == 0 and st["apply_launches"] == 0
    for k in ("apply_timed", "apply_ms", "apply_nodes", "apply_nodes_launched"):
        assert st[k] == [0, 0], (k, st[k])
    assert pc.lib.pc_stats_get(None) == pc.PC_EINVAL
