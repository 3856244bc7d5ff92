"""Programmatic dependent launch changes when a kernel starts, never what it computes: the cycle
and a Krylov solve give bitwise the same results with it (default) and without it (SMG_PDL=0,
read once per process, so the second run is a child process)."""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RUN = r"""
import os, sys
import numpy as np
sys.path.insert(0, os.environ["SMG_ROOT"])
import torch
from paper_1212_6680_gb300 import build, inputs
build.build()
from paper_1212_6680_gb300 import smg
out = {}
for prec in ("fp32", "fp64"):
    n = 48
    r = torch.from_numpy(inputs.rhs(n, n, n, seed=3).ravel().copy()).cuda()
    s = torch.empty_like(r)
    h = smg.smg_setup(n, n, n, 1, 0)
    smg.smg_set_precision(h, prec)
    smg.smg_apply(h, r, s)
    x = torch.zeros_like(r)
    rc, it, rr = smg.krylov_solve(h, "fpcg", r, x, 1e-8, 100)
    torch.cuda.synchronize()
    out[prec + "_apply"] = s.cpu().numpy()
    out[prec + "_x"] = x.cpu().numpy()
    out[prec + "_it"] = np.array([it])
    smg.smg_destroy(h)
np.savez(sys.argv[1], **out)
"""


def _run(path, pdl):
    env = dict(os.environ, SMG_ROOT=ROOT, SMG_PDL="1" if pdl else "0")
    p = subprocess.run([sys.executable, "-c", _RUN, path], env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return np.load(path)


def test_dependent_launch_is_bitwise_neutral():
    with tempfile.TemporaryDirectory() as d:
        on = _run(os.path.join(d, "on.npz"), True)
        off = _run(os.path.join(d, "off.npz"), False)
        for k in on.files:
            assert np.array_equal(on[k], off[k]), k
