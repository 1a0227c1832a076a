"""Stage (a) in two-float arithmetic (FP32 pairs on the FP32 pipes) against the CPU oracle."""
import numpy as np
import pytest

import gwgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def gw():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_2509_23018_gb300 as gw
    return gw


@pytest.mark.parametrize("grid,nv,nc,ngpsi,ng", [((8, 9, 10), 2, 3, 57, 19), ((12, 10, 9), 3, 4, 93, 27),
                                                 ((16, 16, 16), 4, 5, 200, 81), ((20, 18, 15), 2, 7, 150, 64),
                                                 ((24, 24, 24), 16, 64, 600, 200)])
def test_pair_elements_twofloat(gw, grid, nv, nc, ngpsi, ng):
    p = gwgen.make_problem(grid, nv, nc, ngpsi, ng, seed=11, exclude_head=False)
    h = gw.from_problem(p, mtxel="twofloat")
    M = h.pair_elements(0, 0, nv * nc).cpu().numpy()
    h.sync()
    assert rel(M, oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)) < 1e-12


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("ozaki", 1e-9)])
def test_compute_c1_twofloat(gw, prec, tol):
    cfg = gwgen.CONFIGS["c1_24cube"]
    p = gwgen.config_problem(cfg)
    h = gw.from_problem(p, prec=prec, nslices=6, mtxel="twofloat", pair_chunk=300)
    (chi,) = h.compute(0, [0.0, 4.0])
    chi = chi.cpu().numpy()
    h.sync()
    M = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    for i, w in enumerate([0.0, 4.0]):
        assert rel(chi[i], oracle.chi0(M, oracle.delta(p.ev, p.ec, w))) <= tol


@pytest.mark.parametrize("n,nv,nc,ngpsi,ng", [(24, 2, 5, 300, 120), (40, 2, 5, 900, 400), (48, 2, 4, 1200, 500),
                                              (72, 2, 3, 2500, 900)])
def test_pair_elements_cubic_specialised(gw, n, nv, nc, ngpsi, ng):
    """The grid-specialised two-float kernel on each cubic grid it is built for: all pairs (whole
    valence rows, valence-fastest block order) and a range that starts and ends mid-row."""
    p = gwgen.make_problem((n, n, n), nv, nc, ngpsi, ng, seed=13, exclude_head=False)
    h = gw.from_problem(p, mtxel="twofloat")
    Mo = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    M = h.pair_elements(0, 0, nv * nc).cpu().numpy()
    Mr = h.pair_elements(0, 1, nv * nc - 2).cpu().numpy()
    h.sync()
    assert rel(M, Mo) < 1e-12
    assert rel(Mr, Mo[1:nv * nc - 1]) < 1e-12


@pytest.mark.parametrize("gchi", [[(1, 0, 0)], [(0, 0, 0), (1, 0, 0), (0, 1, 0), (-1, 0, 0), (-2, 1, 0)]])
def test_pair_elements_one_plane_sphere(gw, gchi):
    """Degenerate spheres on a specialised grid: one point, and points in one z-plane (one kept
    i2-frequency).  (G = 0 alone would compare rounding noise: M_vc(0) = 0 for v != c.)"""
    p = gwgen.make_problem((24, 24, 24), 2, 3, 300, 1, seed=17, exclude_head=False)
    p.gchi = np.asarray(gchi, np.int32)
    h = gw.from_problem(p, mtxel="twofloat")
    M = h.pair_elements(0, 0, 6).cpu().numpy()
    h.sync()
    assert rel(M, oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)) < 1e-12
