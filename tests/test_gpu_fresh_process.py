"""Standalone kernel entry points must work as the first library call of a process (no
handle created before): each is run in a fresh interpreter."""
import os
import subprocess
import sys

import pytest

from gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, ctypes, torch
sys.path.insert(0, {root!r})
import paper_2502_02294_gb300 as dh
n = 40
u = torch.zeros(5, n, n, n, device="cuda"); u[0] = 1.0; u[4] = 1.0; u[1] = 0.1
lam = torch.ones_like(u)
for axis in range(3):
    out = dh.sweep(u, axis, 0.3)
    lin, dnu = dh.sweep_adjoint(u, lam, axis, 0.3)
torch.cuda.synchronize()
assert torch.isfinite(out).all() and torch.isfinite(lin).all()
print("ok")
"""


def test_sweep_entry_points_in_fresh_process():
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT)], capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
