"""Index maps of the pair kernels, on the CPU: the radix plans of every configured grid and the
sphere tables the library builds (csrc/sphere_plan.h, the builder gw_chi0_set_gsphere uses),
walked index by index against the extents of the buffers they address (tests/host/plan_check.cu).
This stands in for a device-side bounds checker: every index the kernels derive from the plans
is enumerated here for each workload's grid and G-sphere (and for spheres at finite q and on
non-cubic grids)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import gwgen

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("plans") / "plan_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-o", exe,
                    os.path.join(HERE, "host", "plan_check.cu")], check=True, capture_output=True)
    return exe


def run(checker, grid, g):
    inp = f"{grid[0]} {grid[1]} {grid[2]} {len(g)}\n" + "\n".join(" ".join(str(int(x)) for x in r) for r in g) + "\n"
    r = subprocess.run([checker], input=inp, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout


@pytest.mark.parametrize("name", ["c1_24cube", "c2_48cube", "c3_72cube", "c5_adjoint"])
def test_workload_spheres(checker, name):
    cfg = gwgen.CONFIGS[name]
    out = run(checker, cfg.grid, gwgen.gsphere(cfg.ng, exclude_zero=True))
    assert out.startswith("OK")


def test_batched_spheres_at_finite_q(checker):
    """The 40^3 batched workload: spheres of 300 .. 3000 points at q on the 4x4x4 grid."""
    qs = gwgen.qgrid(4)
    rng = np.random.default_rng(3)
    for i in rng.choice(len(qs), 6, replace=False):
        ng = int(rng.integers(300, 3001))
        run(checker, (40, 40, 40), gwgen.gsphere(ng, q=qs[i], exclude_zero=bool(np.all(qs[i] == 0))))


@pytest.mark.parametrize("grid,ng", [((16, 15, 18), 77), ((12, 12, 12), 27), ((20, 24, 30), 300), ((48, 48, 48), 1)])
def test_other_grids_and_degenerate_spheres(checker, grid, ng):
    run(checker, grid, gwgen.gsphere(ng))


def test_checker_catches_a_bad_table(checker):
    """The checker itself: with two cells of the built tables swapped (a plausible ordering slip)
    it must report a violation."""
    g = gwgen.gsphere(200)
    r = subprocess.run([checker, "--corrupt"], input="48 48 48 200\n" + "\n".join(" ".join(map(str, x)) for x in g)
                       + "\n", capture_output=True, text=True)
    assert r.returncode != 0 and "FAIL" in r.stdout


def test_bounds_checked_build_compiles_and_exports():
    """The bounds-checked build (-DGW_DEBUG) compiles and exports every symbol the header declares."""
    import ctypes
    import re
    from paper_2509_23018_gb300 import build as b
    if not os.path.exists(b.nvcc()):
        pytest.skip("nvcc not available")
    lib = ctypes.CDLL(b.build(debug=True))
    names = set(re.findall(r"GW_API[^;(]*?\b(gw_chi0_\w+)\s*\(", open(os.path.join(HERE, "..", "include",
                                                                                    "gw_chi0.h")).read()))
    for n in names:
        assert hasattr(lib, n), n
