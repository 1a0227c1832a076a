"""Parity of the native FP64 CUDA path with the CPU oracle (same seeded inputs).

Bar: relative Frobenius error <= 1e-11 (the FP64 target of the method's statement).
"""
import numpy as np
import pytest

import gwgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11


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


def handle(gw, prob, **kw):
    return gw.from_problem(prob, **kw)


C1 = gwgen.CONFIGS["c1_24cube"]


@pytest.fixture(scope="module")
def c1():
    p = gwgen.config_problem(C1)
    M = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    return p, M


@pytest.mark.parametrize("grid,nv,nc,ngpsi,ng", [((8, 9, 10), 2, 3, 57, 19), ((12, 10, 9), 3, 4, 93, 27),
                                                 ((16, 16, 16), 4, 5, 200, 81), ((20, 18, 15), 2, 7, 150, 64)])
def test_pair_elements_tiny_two_routes(gw, grid, nv, nc, ngpsi, ng):
    p = gwgen.make_problem(grid, nv, nc, ngpsi, ng, seed=11, exclude_head=False)
    h = handle(gw, p)
    M = h.pair_elements(0, 0, nv * nc).cpu().numpy()
    h.sync()
    assert rel(M, oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)) < 1e-12
    if np.prod(grid) <= 4000:
        assert rel(M, oracle.m_dft(grid, p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)) < 1e-12


def test_pair_elements_c1(gw, c1):
    p, Mo = c1
    h = handle(gw, p)
    M = h.pair_elements(0, 0, C1.npairs).cpu().numpy()
    assert rel(M, Mo) < 1e-12
    # ragged sub-range
    M2 = h.pair_elements(0, 37, 101).cpu().numpy()
    assert rel(M2, Mo[37:138]) < 1e-12
    h.sync()


def test_contract_given_oracle_M(gw, c1):
    p, Mo = c1
    h = gw.Chi0(C1.grid)
    om = [0.0, 1.5, 40.0]
    chi = h.contract(dev(p.ev), dev(p.ec), dev(Mo), om).cpu().numpy()
    h.sync()
    for i, w in enumerate(om):
        ref = oracle.chi0(Mo, oracle.delta(p.ev, p.ec, w))
        assert rel(chi[i], ref) < TOL
        assert np.array_equal(chi[i], chi[i].conj().T)


@pytest.mark.parametrize("chunk", [8192, 300, 64])
def test_compute_c1(gw, c1, chunk):
    p, Mo = c1
    h = handle(gw, p, pair_chunk=chunk)
    om = [0.0, 2.0]
    (chi,), (dg,) = h.compute(0, om, diag=True)
    chi, dg = chi.cpu().numpy(), dg.cpu().numpy()
    h.sync()
    for i, w in enumerate(om):
        ref = oracle.chi0(Mo, oracle.delta(p.ev, p.ec, w))
        assert rel(chi[i], ref) < TOL
        assert np.array_equal(chi[i], chi[i].conj().T)
        assert np.all(np.diag(chi[i]).imag == 0)
        assert rel(dg[i], np.real(np.diag(ref))) < TOL


@pytest.mark.parametrize("ng", [1, 7, 64, 65, 129])
def test_compute_ragged_sphere(gw, ng):
    p = gwgen.make_problem((16, 15, 18), 3, 9, 150, ng, seed=5)
    h = handle(gw, p, pair_chunk=10)
    (chi,) = h.compute(0, [0.0])
    chi = chi.cpu().numpy()[0]
    h.sync()
    Mo = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    assert rel(chi, oracle.chi0(Mo, oracle.delta(p.ev, p.ec, 0.0))) < TOL


def test_single_pair(gw):
    p = gwgen.make_problem((12, 12, 12), 1, 1, 57, 27, seed=9)
    h = handle(gw, p)
    (chi,) = h.compute(0, [0.0])
    chi = chi.cpu().numpy()[0]
    h.sync()
    m = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)[0]
    assert rel(chi, 4.0 / (p.ev[0] - p.ec[0]) * np.outer(np.conj(m), m)) < TOL


def test_errors_are_reported(gw):
    import ctypes
    p = gwgen.make_problem((12, 12, 12), 2, 3, 57, 27, seed=9)
    h = gw.Chi0((12, 12, 12))
    buf = torch.empty(27 * 27, dtype=torch.complex128, device="cuda")
    st = h.lib.gw_chi0_compute(h.h, 1, (ctypes.c_int * 1)(0), 1, (ctypes.c_double * 1)(0.0),
                               ctypes.c_void_p(buf.data_ptr()), None)
    assert st == 2  # GW_ERR_STATE: nothing set yet
    g = dev(p.gpsi)
    h.set_bands(0, 1, g, dev(p.cc), dev(p.ec))
    with pytest.raises(gw.GwError) as e:  # valence above conduction
        h.set_bands(0, 0, g, dev(p.cv), dev(p.ec[:2] + 100.0))
    assert e.value.status == 1
    h.set_bands(0, 0, g, dev(p.cv), dev(p.ev))
    # |K| <= 5 bands with a |G| <= 2 sphere alias on a 12-grid: 5 + 5 + 2 >= 12
    wide = gwgen.make_problem((12, 12, 12), 2, 3, 500, 18, seed=9)  # |G| <= 1
    h2 = handle(gw, wide)
    with pytest.raises(gw.GwError) as e:
        h2.set_gsphere(0, dev(gwgen.gsphere(57)))
    assert e.value.status == 1
    with pytest.raises(gw.GwError) as e:  # a component outside (-n/2, n/2)
        h2.set_gsphere(0, dev(np.array([[6, 0, 0]], np.int32)))
    assert e.value.status == 1
    with pytest.raises(gw.GwError) as e:
        h.set_gsphere(0, dev(np.zeros((0, 3), np.int32)))
    assert e.value.status == 1
    # the handle stays usable after errors
    h.set_gsphere(0, dev(p.gchi))
    (chi,) = h.compute(0, [0.0])
    h.sync()
    assert chi.shape == (1, 27, 27)


def test_memory_budget(gw):
    p = gwgen.make_problem((12, 12, 12), 2, 3, 57, 27, seed=9)
    h = gw.Chi0((12, 12, 12), mem_budget_bytes=64 * 1024)
    with pytest.raises(gw.GwError) as e:
        h.set_bands(0, 1, dev(p.gpsi), dev(p.cc), dev(p.ec))
    assert e.value.status == 3  # GW_ERR_OOM


def test_watchdog_timeout_is_reported(gw):
    """A bounded device wait that nothing satisfies reports GW_ERR_TIMEOUT; the handle stays usable."""
    p = gwgen.make_problem((12, 12, 12), 2, 3, 57, 27, seed=9)
    h = handle(gw, p)
    assert h.lib.gw_chi0_check_watchdog(h.h, 2000) == 0
    with pytest.raises(gw.GwError) as e:
        h.sync()
    assert e.value.status == 6  # GW_ERR_TIMEOUT
    (chi,) = h.compute(0, [0.0])
    h.sync()  # status was cleared by the previous sync
    Mo = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    assert rel(chi.cpu().numpy()[0], oracle.chi0(Mo, oracle.delta(p.ev, p.ec, 0.0))) < TOL


def test_host_fault_injection(gw, monkeypatch):
    """An injected host-side failure before chunk 2 is reported; the next call succeeds."""
    p = gwgen.make_problem((12, 12, 12), 2, 3, 57, 27, seed=9)
    h = handle(gw, p, pair_chunk=2)
    monkeypatch.setenv("GW_CHI0_FAULT_AT_CHUNK", "2")
    with pytest.raises(gw.GwError) as e:
        h.compute(0, [0.0])
    assert e.value.status == 4 and "injected" in str(e.value)
    monkeypatch.delenv("GW_CHI0_FAULT_AT_CHUNK")
    (chi,) = h.compute(0, [0.0])
    h.sync()
    Mo = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    assert rel(chi.cpu().numpy()[0], oracle.chi0(Mo, oracle.delta(p.ev, p.ec, 0.0))) < TOL
