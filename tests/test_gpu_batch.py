"""Batched chi0 over many q-points with uneven spheres and several frequencies (graph path)."""
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


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


@pytest.fixture(scope="module")
def batch():
    b = gwgen.make_batch((24, 24, 24), 8, 32, 600, 40, 200, 2, 3, seed=gwgen.BASE_SEED + 3)
    refs = []
    for iq in range(len(b.qs)):
        M = oracle.m_conv(b.gpsi, b.cv[iq], b.gpsi, b.cc, b.gchi[iq])
        refs.append([oracle.chi0(M, oracle.delta(b.ev[iq], b.ec, w)) for w in b.omega])
    return b, refs


def load(gw, b, **kw):
    h = gw.Chi0(b.grid, nq=len(b.qs), **kw)
    g = dev(b.gpsi)
    h.set_bands(0, 1, g, dev(b.cc), dev(b.ec))
    for iq in range(len(b.qs)):
        h.set_bands(iq, 0, g, dev(b.cv[iq]), dev(b.ev[iq]))
        h.set_gsphere(iq, dev(b.gchi[iq]))
    return h


@pytest.mark.parametrize("prec,mtxel,tol", [("fp64", "fp64", 1e-11), ("ozaki", "twofloat", 1e-9),
                                            ("fp64", "twofloat", 1e-11)])
def test_batch_matches_oracle(gw, batch, prec, mtxel, tol):
    b, refs = batch
    h = load(gw, b, prec=prec, nslices=6, mtxel=mtxel)
    slots = list(range(len(b.qs)))
    res, dg = h.compute_batch(slots, list(b.omega), diag=True)
    for _ in range(2):  # replays of the captured graph give the same values
        res2 = h.compute_batch(slots, list(b.omega))
    h.sync()
    for iq in slots:
        got, got2, d = res[iq].cpu().numpy(), res2[iq].cpu().numpy(), dg[iq].cpu().numpy()
        assert np.array_equal(got, got2)
        for w in range(len(b.omega)):
            assert rel(got[w], refs[iq][w]) <= tol, (iq, w)
            assert np.array_equal(got[w], got[w].conj().T)
            assert rel(d[w], np.real(np.diag(refs[iq][w]))) < 1e-11
    t = h.tuning()
    assert t["shapes_tuned"] == 1
    assert t["tile_f64"] in (32, 64) and t["tile_split"] in (128, 240, 256)


def test_batch_equals_streamed(gw, batch):
    """The graph path and the chunked streaming path agree (subset of slots, reordered)."""
    b, _ = batch
    h = load(gw, b, pair_chunk=100)
    slots = [5, 2, 7]
    a = h.compute_batch(slots, list(b.omega))
    c = h.compute(slots, list(b.omega))
    h.sync()
    for x, y in zip(a, c):
        assert rel(x.cpu().numpy(), y.cpu().numpy()) < 1e-13
