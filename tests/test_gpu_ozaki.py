"""Split-precision (Ozaki, BF16 tensor cores) contraction against the CPU oracle.

Bar for the split path: relative Frobenius error <= 1e-9 at the default slice count,
error 0 when every input is a small integer that one slice holds exactly, and an
error that falls as slices are added.
"""
import numpy as np
import pytest

import gwgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_SPLIT = 1e-9


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def gw():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_2509_23018_gb300 as gw
    return gw


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


@pytest.fixture(scope="module")
def c1():
    cfg = gwgen.CONFIGS["c1_24cube"]
    p = gwgen.config_problem(cfg)
    M = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    return p, M


@pytest.mark.parametrize("ng,nv,nc", [(40, 3, 37), (200, 16, 64), (129, 5, 77)])
def test_small_integers_exact(gw, ng, nv, nc):
    """Integer M and Delta = -1 (x = -4 at w = 0): the split is exact, so is the result."""
    rng = np.random.default_rng(ng)
    M = rng.integers(-3, 4, (nv * nc, ng)) + 1j * rng.integers(-3, 4, (nv * nc, ng))
    ev, ec = np.full(nv, -2.0), np.full(nc, 2.0)
    want = -(np.conj(M).T @ M)  # exact in float64 (small integers)
    h = gw.Chi0((8, 8, 8), prec="ozaki", nslices=4)
    chi = h.contract(dev(ev), dev(ec), dev(M), [0.0]).cpu().numpy()[0]
    h.sync()
    assert np.array_equal(chi, want)


def test_split_c1_matches_oracle(gw, c1):
    p, M = c1
    errs = {}
    for s in (3, 4, 5, 6, 7, 8):
        h = gw.Chi0(p.grid, prec="ozaki", nslices=s)
        chi = h.contract(dev(p.ev), dev(p.ec), dev(M), [0.0, 5.0]).cpu().numpy()
        h.sync()
        e = []
        for i, w in enumerate([0.0, 5.0]):
            ref = oracle.chi0(M, oracle.delta(p.ev, p.ec, w))
            e.append(rel(chi[i], ref))
            assert np.array_equal(chi[i], chi[i].conj().T)
        errs[s] = max(e)
    print("split error per slice count:", errs)
    assert errs[6] <= TOL_SPLIT
    for s in (3, 4, 5, 6):
        assert errs[s + 1] <= errs[s] * 1.01 or errs[s + 1] < 1e-14


@pytest.mark.parametrize("chunk", [8192, 100])
def test_split_full_path_c1(gw, c1, chunk):
    p, M = c1
    h = gw.from_problem(p, prec="ozaki", nslices=6, pair_chunk=chunk)
    (chi,) = h.compute(0, [0.0, 2.0])
    chi = chi.cpu().numpy()
    h.sync()
    for i, w in enumerate([0.0, 2.0]):
        assert rel(chi[i], oracle.chi0(M, oracle.delta(p.ev, p.ec, w))) <= TOL_SPLIT


@pytest.mark.parametrize("ng", [1, 7, 64, 65, 129, 300])
def test_split_ragged(gw, ng):
    p = gwgen.make_problem((16, 15, 18), 3, 9, 150, ng, seed=5)
    h = gw.from_problem(p, prec="ozaki", nslices=6, pair_chunk=10)
    (chi,) = h.compute(0, [0.0])
    chi = chi.cpu().numpy()[0]
    h.sync()
    Mo = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    assert rel(chi, oracle.chi0(Mo, oracle.delta(p.ev, p.ec, 0.0))) <= TOL_SPLIT


@pytest.mark.parametrize("ng", [65, 300, 2000])
def test_split_tile_widths_agree(gw, ng, monkeypatch):
    """The split contraction gives the same bits at tile widths 128, 240 and 256 real columns
    (every entry sums the same slice products in the same K order), on spheres that leave ragged
    row and column tiles at each width."""
    rng = np.random.default_rng(1000 + ng)
    nv, nc = 8, 40
    M = rng.standard_normal((nv * nc, ng)) + 1j * rng.standard_normal((nv * nc, ng))
    ev, ec = -1.0 - rng.random(nv), 1.0 + rng.random(nc)
    outs = []
    for width in (128, 240, 256):
        monkeypatch.setenv("GW_CHI0_SPLIT_TILE", str(width))
        h = gw.Chi0((8, 8, 8), prec="ozaki", nslices=7)
        outs.append(h.contract(dev(ev), dev(ec), dev(M), [0.0, 1.5]).cpu().numpy())
        h.sync()
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2])
    assert np.array_equal(outs[0][0], outs[0][0].conj().T)


def test_streams_query(gw):
    """The overlapped path is taken for a 24^3 slot in split precision and not in
    FP64 mode or with single_stream; an unset slot is an error."""
    cfg = gwgen.CONFIGS["c1_24cube"]
    p = gwgen.config_problem(cfg)
    for prec, single, want in (("ozaki", False, 2), ("ozaki", True, 1), ("fp64", False, 1)):
        h = gw.from_problem(p, prec=prec, nslices=7, mtxel="twofloat", single_stream=single)
        assert h.streams(0) == want
        with pytest.raises(gw.GwError):
            h.streams(5)
        h.destroy()


@pytest.mark.parametrize("mtxel", ["twofloat", "fp64"])
def test_frequency_group_slicing(gw, mtxel):
    """Nine frequencies in one call (sliced in groups of up to eight from one read of M) against
    nine single-frequency calls (sliced one by one), and against the oracle."""
    cfg = gwgen.CONFIGS["c1_24cube"]
    p = gwgen.config_problem(cfg)
    om = [0.0, 0.5, 1.0, 2.0, 3.5, 5.0, 8.0, 13.0, 21.0]
    h = gw.from_problem(p, prec="ozaki", nslices=7, mtxel=mtxel, pair_chunk=300)
    (many,) = h.compute(0, om)
    many = many.cpu().numpy()
    one = np.stack([h.compute(0, [w])[0][0].cpu().numpy() for w in om])
    h.sync()
    assert np.abs(many - one).max() <= 1e-14 * np.abs(one).max()
    M = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    for i in (0, 4, 8):
        ref = oracle.chi0(M, oracle.delta(p.ev, p.ec, om[i]))
        assert np.linalg.norm(many[i] - ref) <= 1e-9 * np.linalg.norm(ref)
    h.destroy()


@pytest.mark.parametrize("spread", [0.0, 1e-3])
def test_split_correlated_rows(gw, spread):
    """Correlated inputs, the worst case for the FP32 sums of the slice groups: every pair
    carries (nearly) the same row, so the digits of all 8192 pairs of a chunk share their signs
    and the group sums reach their largest magnitudes (t >= 4 may then round in FP32; the
    rounding sits at least 2^-36 below the leading group).  The result must still meet the
    split bar against the oracle."""
    rng = np.random.default_rng(23)
    ng, nv, nc = 160, 8, 1024
    m0 = rng.standard_normal(ng) + 1j * rng.standard_normal(ng)
    noise = rng.standard_normal((nv * nc, ng)) + 1j * rng.standard_normal((nv * nc, ng))
    M = m0[None, :] * (1.0 + spread * noise)
    ev = rng.uniform(-10, -1, nv)
    ec = rng.uniform(1, 30, nc)
    h = gw.Chi0((8, 8, 8), prec="ozaki", nslices=7, pair_chunk=8192)
    for w in (0.0, 4.0):
        chi = h.contract(dev(ev), dev(ec), dev(M), [w]).cpu().numpy()[0]
        assert rel(chi, oracle.chi0(M, oracle.delta(ev, ec, w))) <= TOL_SPLIT
    h.sync()
