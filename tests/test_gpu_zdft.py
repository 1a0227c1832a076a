"""Stage (a) with the last-axis transform on the tensor cores (the route gw_chi0_compute takes for
two-float stage (a) on the 48^3 grid): pair elements of a conduction block against the oracle,
element by element, and chi through that route, on shapes that exercise its tiles: a partial row
tile (few valence bands), two row tiles, few kept z-frequencies (four conduction bands per tile),
ragged conduction blocks, and the 2000-G sphere of the benchmark's workload; and bands whose
scales span many orders of magnitude on a sphere with G = 0, on both routes of stage (a)."""
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


SHAPES = [(5, 7, 600, 200, 8192), (130, 9, 900, 300, 8192), (16, 64, 6000, 2000, 8192), (12, 23, 1200, 400, 60)]


@pytest.mark.parametrize("nv,nc,ngpsi,ng,chunk", SHAPES)
def test_block_pair_elements_match_oracle(gw, nv, nc, ngpsi, ng, chunk):
    p = gwgen.make_problem((48, 48, 48), nv, nc, ngpsi, ng, seed=41)
    h = gw.from_problem(p, prec="ozaki", nslices=7, mtxel="twofloat", pair_chunk=chunk)
    c0, cb = nc // 3, nc - nc // 3          # a block that does not start at 0
    M = h.pair_elements_block(0, c0, cb).cpu().numpy()
    h.sync()
    Mo = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc[c0:c0 + cb], p.gchi)       # rows v * cb + cl
    Mo = Mo.reshape(nv, cb, ng).transpose(1, 0, 2).reshape(cb * nv, ng)    # rows cl * nv + v
    assert rel(M, Mo) < 1e-12
    # row by row too: no pair may carry a large relative error hidden by the others
    rows = np.linalg.norm(M - Mo, axis=1) / np.linalg.norm(Mo, axis=1)
    assert rows.max() < 1e-11


@pytest.mark.parametrize("nv,nc,ngpsi,ng,chunk", SHAPES[:2] + SHAPES[3:])
@pytest.mark.parametrize("single", [False, True])
def test_chi_on_tensor_route_matches_oracle(gw, nv, nc, ngpsi, ng, chunk, single):
    p = gwgen.make_problem((48, 48, 48), nv, nc, ngpsi, ng, seed=43)
    h = gw.from_problem(p, prec="ozaki", nslices=7, mtxel="twofloat", pair_chunk=chunk, single_stream=single)
    assert h.streams(0) == 1
    om = [0.0, 2.5]
    chis = h.compute(0, om)[0].cpu().numpy()
    h.sync()
    M = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    for i, w in enumerate(om):
        assert rel(chis[i], oracle.chi0(M, oracle.delta(p.ev, p.ec, w))) < 1e-11
        assert np.array_equal(chis[i], chis[i].conj().T)


def test_block_entry_rejects_other_routes(gw):
    from paper_2509_23018_gb300 import _lib
    p = gwgen.make_problem((24, 24, 24), 4, 6, 300, 80, seed=5)
    h = gw.from_problem(p, prec="ozaki", nslices=7, mtxel="twofloat")
    with pytest.raises(gw.GwError) as e:
        h.pair_elements_block(0, 0, 2)
    assert e.value.status == _lib.GW_ERR_UNSUPPORTED
    h.destroy()
    p = gwgen.make_problem((48, 48, 48), 4, 6, 300, 80, seed=5)
    h = gw.from_problem(p, prec="ozaki", nslices=7, mtxel="twofloat")
    with pytest.raises(gw.GwError) as e:
        h.pair_elements_block(0, 4, 3)   # outside [0, nc)
    assert e.value.status == _lib.GW_ERR_ARG
    h.pair_elements_block(0, 0, 6)       # still usable
    h.sync()


@pytest.mark.parametrize("block", [True, False])
def test_pair_elements_wide_dynamic_range(gw, block):
    """Bands scaled over many orders of magnitude (valence 1e-3 .. 1e3, conduction 1e-6 .. 1e6,
    so the rows of M span 1e-9 .. 1e9) on a sphere that includes G = 0, where M_vc(0) = <v|c>
    vanishes for the orthonormal bands by cancellation over the grid: every row matches the
    oracle to its own scale on the tensor-core route (block entry) and on the two-float FFT
    route (general entry); M_vc(0) stays at rounding level relative to the row."""
    import dataclasses
    p = gwgen.make_problem((48, 48, 48), 6, 10, 900, 300, seed=47)
    sv = 10.0 ** np.linspace(-3, 3, 6)
    sc = 10.0 ** np.linspace(-6, 6, 10)
    g = np.vstack([np.zeros((1, 3), np.int32), p.gchi]).astype(np.int32)
    p = dataclasses.replace(p, cv=p.cv * sv[:, None], cc=p.cc * sc[:, None], gchi=g)
    h = gw.from_problem(p, prec="ozaki", nslices=7, mtxel="twofloat")
    Mo = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)              # rows v * nc + c
    if block:
        M = h.pair_elements_block(0, 0, 10).cpu().numpy()               # rows c * nv + v
        M = M.reshape(10, 6, -1).transpose(1, 0, 2).reshape(60, -1)
    else:
        M = h.pair_elements(0, 0, 60).cpu().numpy()
    h.sync()
    scale = np.outer(sv, sc).reshape(-1)                                # |M_vc| ~ sv sc
    rows = np.linalg.norm(M - Mo, axis=1) / np.linalg.norm(Mo, axis=1)
    assert rows.max() < 1e-11, rows.max()
    assert np.all(np.abs(M[:, 0]) < 1e-12 * scale)                      # <v|c> = 0 for v != c


@pytest.mark.parametrize("gzmax,route", [(15, True), (16, False)])
def test_route_edge_kept_frequencies(gw, gzmax, route):
    """The widest sphere the tensor-core route takes, K2 = 32 kept z-frequencies (one conduction
    band per 64-column tile), and one more (K2 = 33), which must fall back to the FFT route:
    chi against the oracle on both, and the route each took."""
    import dataclasses
    from paper_2509_23018_gb300 import _lib
    p = gwgen.make_problem((48, 48, 48), 6, 10, 900, 200, seed=53)
    g = np.array([(x, y, z) for z in range(-16, gzmax + 1) for y in (-1, 0, 1) for x in (-1, 0, 1)
                  if (x, y, z) != (0, 0, 0)], np.int32)
    p = dataclasses.replace(p, gchi=g)
    h = gw.from_problem(p, prec="ozaki", nslices=7, mtxel="twofloat")
    (chi,) = h.compute(0, [0.0])
    h.sync()
    M = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    assert rel(chi[0].cpu().numpy(), oracle.chi0(M, oracle.delta(p.ev, p.ec, 0.0))) < 1e-11
    if route:
        Mb = h.pair_elements_block(0, 0, 10).cpu().numpy().reshape(10, 6, -1).transpose(1, 0, 2).reshape(60, -1)
        h.sync()
        assert rel(Mb, M) < 1e-12
    else:
        with pytest.raises(gw.GwError) as e:
            h.pair_elements_block(0, 0, 10)
        assert e.value.status == _lib.GW_ERR_UNSUPPORTED
