"""Bounded device waits: a kernel whose wait on its own copies runs out reports it.

The row-tile and TMA-tile apply kernels stage x through bulk / tensor copies and wait on
them with a bounded number of mbarrier polls.  With PC_WAIT_LIMIT=0 every such wait gives up
at once: the kernel lets its copies in flight land, records the event in the grid's device
error word and returns.  Nothing faults and nothing hangs; the host sees the event through
the synchronising calls.  Each case runs in a child process (the limit is read once per
process); afterwards this process, at the default limit, still matches the oracle.
"""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

from workloads import complex_gaussian, two_phase_sphere

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, %(root)r)
import paper_2606_03599_gb300 as pc
from workloads import complex_gaussian, two_phase_sphere

N = 32
cell = two_phase_sphere(N, 0.35, 2)
g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
pc.pc_set_k(g, [0.3, 0.1, 0.2])
nb = N ** 3 // 4
out = {}
x = torch.from_numpy(complex_gaussian(3 * nb, 5)).to(torch.complex64).cuda()
y = torch.zeros_like(x)

def status():
    try:
        pc.pc_device_status(g)
        return 0
    except pc.PcError as e:
        return e.code

pc.pc_block_apply(g, 0, x, y, 0.5)
out["apply"] = status()
out["after_clear"] = status()          # the word was cleared by the previous check
dot = torch.zeros(1, dtype=torch.float64, device="cuda")
pc.pc_block_apply_dot_noalloc(g, 1, x, y, dot, 0.5)
torch.cuda.synchronize()
out["noalloc_dot_nan"] = bool(np.isnan(dot.item()))
out["noalloc"] = status()
rhs = x.clone()
xs = torch.zeros_like(x)
try:
    pc.pc_shift_invert_pcg(g, 2, pc.pc_default_sigma(g), rhs, xs, tol=1e-6, maxit=4)
    out["pcg"] = 0
except pc.PcError as e:
    out["pcg"] = e.code
out["final"] = status()
pc.pc_grid_destroy(g)
print("RESULT " + json.dumps(out))
"""


def _child(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    p = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT}], env=env, capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    line = [ln for ln in p.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


@pytest.mark.parametrize("kernel", ["default", "tma"])
def test_expired_waits_are_reported(kernel):
    import paper_2606_03599_gb300 as pc
    env = {"PC_WAIT_LIMIT": "0"}
    if kernel == "tma":
        env["PC_APPLY_KERNEL"] = "tma"
    r = _child(env)
    assert r["apply"] == pc.PC_ECUDA
    assert r["after_clear"] == pc.PC_OK
    assert r["noalloc_dot_nan"] and r["noalloc"] == pc.PC_ECUDA
    assert r["pcg"] == pc.PC_ECUDA
    assert r["final"] == pc.PC_OK


def test_default_limit_child_reports_nothing():
    import paper_2606_03599_gb300 as pc
    r = _child({})
    assert r["apply"] == pc.PC_OK and r["noalloc"] == pc.PC_OK and not r["noalloc_dot_nan"]
    assert r["final"] == pc.PC_OK


def test_apply_still_matches_the_oracle_after_expired_waits():
    import torch
    import paper_2606_03599_gb300 as pc
    from oracle import oracle as O
    N = 32
    cell = two_phase_sphere(N, 0.35, 2)
    g = pc.pc_grid_create(N, cell.C, cell.rho, phase=cell.phase, a_lat=cell.a_lat)
    try:
        C0, rho0, L = pc.pc_grid_units(g)
        pb = O.problem_from_cell(cell, C0=C0, rho0=rho0, L=L)
        kappa = [0.3, 0.1, 0.2]
        pc.pc_set_k(g, kappa)
        nb = N ** 3 // 4
        xh = complex_gaussian(3 * nb, 5)
        x = torch.from_numpy(xh).to(torch.complex64).cuda()
        y = torch.full_like(x, complex(float("nan"), float("nan")))
        pc.pc_block_apply(g, 0, x, y, 0.5)
        pc.pc_device_status(g)
        ref = O.apply_block(pb, kappa, 0, xh.astype(np.complex64).astype(np.complex128).reshape(3, nb), shift=0.5)
        got = y.cpu().numpy().astype(np.complex128).reshape(3, nb)
        assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()
    finally:
        pc.pc_grid_destroy(g)
