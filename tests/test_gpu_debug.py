"""The bounds-checked build (GW_CHI0_DEBUG=1 loads it): the pair kernels of both stage (a) routes
and the contraction run with every plan-derived index checked on the device; no violation may be
recorded, and the results still match the oracle.  Runs in a child process (the library is loaded
once per process)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch
import gwgen, oracle
import paper_2509_23018_gb300 as gw
from paper_2509_23018_gb300 import _lib
assert _lib.library_path().endswith("libgwchi0_debug.so")
for grid, nv, nc, ngpsi, ng in (((48, 48, 48), 16, 20, 900, 300), ((24, 24, 24), 6, 9, 400, 100)):
    p = gwgen.make_problem(grid, nv, nc, ngpsi, ng, seed=9)
    h = gw.from_problem(p, prec="ozaki", nslices=7, mtxel="twofloat", pair_chunk=96)
    (chi,) = h.compute(0, [0.0])
    h.sync()                                    # raises on a recorded bounds violation
    M = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    ref = oracle.chi0(M, oracle.delta(p.ev, p.ec, 0.0))
    err = np.linalg.norm(chi[0].cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < 1e-11, err
print("debug ok")
"""


def test_bounds_checked_build_runs_clean():
    env = dict(os.environ, GW_CHI0_DEBUG="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0 and "debug ok" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]
