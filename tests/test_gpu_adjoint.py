"""Adjoint of L = Re Tr(W chi0): CUDA path against the oracle adjoint and finite differences."""
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


CASES = [((12, 12, 12), 3, 5, 93, 27, 0.0, 1000), ((16, 15, 18), 4, 9, 150, 64, 2.5, 12),
         ((24, 24, 24), 16, 64, 600, 200, 0.0, 256),
         # the grid-specialised back-projections of the 40^3 and 48^3 workloads
         ((40, 40, 40), 2, 4, 600, 150, 1.0, 5), ((48, 48, 48), 2, 3, 900, 200, 0.0, 6)]


@pytest.mark.parametrize("mtxel", ["fp64", "twofloat"])
@pytest.mark.parametrize("grid,nv,nc,ngpsi,ng,w,chunk", CASES)
def test_adjoint_matches_oracle(gw, mtxel, grid, nv, nc, ngpsi, ng, w, chunk):
    p = gwgen.make_problem(grid, nv, nc, ngpsi, ng, seed=31)
    W = gwgen.hermitian(np.random.default_rng(5), ng)
    Lo, dEvo, dEco, dcvo, dcco = oracle.adjoint(p.gpsi, p.cv, p.ev, p.gpsi, p.cc, p.ec, p.gchi, W, w)
    h = gw.from_problem(p, mtxel=mtxel, pair_chunk=chunk)
    L, dEv, dEc, dcv, dcc = h.adjoint(0, dev(W), omega=w)
    h.sync()
    assert abs(L - Lo) <= 1e-11 * abs(Lo)
    assert rel(dEv.cpu().numpy(), dEvo) < 1e-10
    assert rel(dEc.cpu().numpy(), dEco) < 1e-10
    assert rel(dcv.cpu().numpy(), dcvo) < 1e-10
    assert rel(dcc.cpu().numpy(), dcco) < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_adjoint_takes_hermitian_part_of_w(gw, prec):
    """A non-Hermitian W: the library uses (W + W^H)/2, which is all Re Tr(W chi) sees."""
    p = gwgen.make_problem((16, 15, 18), 4, 9, 150, 64, seed=33)
    rng = np.random.default_rng(8)
    W = rng.standard_normal((64, 64)) + 1j * rng.standard_normal((64, 64))
    Wh = 0.5 * (W + W.conj().T)
    Lo, dEvo, dEco, dcvo, dcco = oracle.adjoint(p.gpsi, p.cv, p.ev, p.gpsi, p.cc, p.ec, p.gchi, Wh, 1.5)
    h = gw.from_problem(p, prec=prec, nslices=7, pair_chunk=12)
    L, dEv, dEc, dcv, dcc = h.adjoint(0, dev(W), omega=1.5)
    h.sync()
    tol = 1e-10 if prec == "fp64" else 1e-9
    assert abs(L - Lo) <= tol * abs(Lo)
    for a, b in ((dEv, dEvo), (dEc, dEco), (dcv, dcvo), (dcc, dcco)):
        assert rel(a.cpu().numpy(), b) < tol


def _L_forward(gw, p, W, cv, cc, ev, ec, w):
    """L = Re Tr(W chi) with chi from the forward path."""
    pp = gwgen.Problem(p.grid, p.gpsi, cv, cc, ev, ec, p.gchi, np.array([w]))
    h = gw.from_problem(pp, mtxel="twofloat")
    (chi,) = h.compute(0, [w])
    L = float(torch.real(torch.trace(dev(W) @ chi[0])).item())
    h.destroy()
    return L


def test_adjoint_central_differences(gw):
    """h = 1e-6 central differences of the forward L on random coefficients and energies."""
    p = gwgen.make_problem((20, 20, 20), 6, 24, 300, 120, seed=77)
    W = gwgen.hermitian(np.random.default_rng(9), 120)
    w = 1.5
    hnd = gw.from_problem(p, mtxel="twofloat")
    L0, dEv, dEc, dcv, dcc = hnd.adjoint(0, dev(W), omega=w)
    dEv, dEc, dcv, dcc = (x.cpu().numpy() for x in (dEv, dEc, dcv, dcc))
    hnd.destroy()
    hstep = 1e-6
    rng = np.random.default_rng(4)
    for _ in range(8):
        which = rng.integers(2)
        arr = p.cv if which == 0 else p.cc
        b, k = rng.integers(arr.shape[0]), rng.integers(arr.shape[1])
        for unit in (1.0, 1j):
            ap, am = arr.copy(), arr.copy()
            ap[b, k] += hstep * unit
            am[b, k] -= hstep * unit
            if which == 0:
                fd = (_L_forward(gw, p, W, ap, p.cc, p.ev, p.ec, w) - _L_forward(gw, p, W, am, p.cc, p.ev, p.ec, w))
                an = dcv[b, k]
            else:
                fd = (_L_forward(gw, p, W, p.cv, ap, p.ev, p.ec, w) - _L_forward(gw, p, W, p.cv, am, p.ev, p.ec, w))
                an = dcc[b, k]
            fd /= 2 * hstep
            comp = an.real if unit == 1.0 else an.imag
            assert abs(fd - comp) < 1e-5 * max(1.0, abs(comp)), (which, b, k, unit, fd, comp)
    for i in range(2):
        e = p.ev.copy(); e[i] += hstep; Lp = _L_forward(gw, p, W, p.cv, p.cc, e, p.ec, w)
        e[i] -= 2 * hstep; Lm = _L_forward(gw, p, W, p.cv, p.cc, e, p.ec, w)
        assert abs((Lp - Lm) / (2 * hstep) - dEv[i]) < 1e-5 * max(1.0, abs(dEv[i]))
        e = p.ec.copy(); e[i] += hstep; Lp = _L_forward(gw, p, W, p.cv, p.cc, p.ev, e, w)
        e[i] -= 2 * hstep; Lm = _L_forward(gw, p, W, p.cv, p.cc, p.ev, e, w)
        assert abs((Lp - Lm) / (2 * hstep) - dEc[i]) < 1e-5 * max(1.0, abs(dEc[i]))


def test_adjoint_dot_product(gw):
    """<grad, dc> equals the directional derivative of L along a random complex direction dc."""
    p = gwgen.make_problem((16, 16, 16), 4, 12, 200, 81, seed=21)
    W = gwgen.hermitian(np.random.default_rng(8), 81)
    hnd = gw.from_problem(p)
    _, _, _, dcv, dcc = hnd.adjoint(0, dev(W))
    dcv, dcc = dcv.cpu().numpy(), dcc.cpu().numpy()
    hnd.destroy()
    rng = np.random.default_rng(1)
    dv = rng.standard_normal(p.cv.shape) + 1j * rng.standard_normal(p.cv.shape)
    dc = rng.standard_normal(p.cc.shape) + 1j * rng.standard_normal(p.cc.shape)
    t = 1e-5
    Lp = _L_forward(gw, p, W, p.cv + t * dv, p.cc + t * dc, p.ev, p.ec, 0.0)
    Lm = _L_forward(gw, p, W, p.cv - t * dv, p.cc - t * dc, p.ev, p.ec, 0.0)
    fd = (Lp - Lm) / (2 * t)
    an = np.sum(np.real(np.conj(dcv) * dv)) + np.sum(np.real(np.conj(dcc) * dc))
    assert abs(fd - an) < 1e-6 * abs(an)


def test_autograd_function(gw):
    """torch.autograd through Chi0Fn gives the oracle adjoint of L = Re Tr(W chi)."""
    p = gwgen.make_problem((16, 15, 18), 4, 9, 150, 64, seed=12)
    W = gwgen.hermitian(np.random.default_rng(3), 64)
    h = gw.Chi0(p.grid)
    cv = dev(p.cv).requires_grad_(True)
    cc = dev(p.cc).requires_grad_(True)
    ev = dev(p.ev).requires_grad_(True)
    ec = dev(p.ec).requires_grad_(True)
    chi = gw.Chi0Fn.apply(h, dev(p.gpsi), cv, ev, cc, ec, dev(p.gchi), 0.7)
    L = torch.real(torch.trace(dev(W) @ chi))
    L.backward()
    Lo, dEvo, dEco, dcvo, dcco = oracle.adjoint(p.gpsi, p.cv, p.ev, p.gpsi, p.cc, p.ec, p.gchi, W, 0.7)
    assert abs(L.item() - Lo) < 1e-11 * abs(Lo)
    assert rel(cv.grad.cpu().numpy(), dcvo) < 1e-10
    assert rel(cc.grad.cpu().numpy(), dcco) < 1e-10
    assert rel(ev.grad.cpu().numpy(), dEvo) < 1e-10
    assert rel(ec.grad.cpu().numpy(), dEco) < 1e-10


def test_autograd_function_non_hermitian_w(gw):
    """The upstream gradient of L = Re Tr(W chi) for a non-Hermitian W reaches the library as it
    is (W^H in torch's convention); the gradients are those of the Hermitian part of W."""
    p = gwgen.make_problem((16, 15, 18), 4, 9, 150, 64, seed=12)
    rng = np.random.default_rng(4)
    W = rng.standard_normal((64, 64)) + 1j * rng.standard_normal((64, 64))
    h = gw.Chi0(p.grid)
    cv = dev(p.cv).requires_grad_(True)
    ev = dev(p.ev).requires_grad_(True)
    chi = gw.Chi0Fn.apply(h, dev(p.gpsi), cv, ev, dev(p.cc), dev(p.ec), dev(p.gchi), 0.7)
    torch.real(torch.trace(dev(W) @ chi)).backward()
    _, dEvo, _, dcvo, _ = oracle.adjoint(p.gpsi, p.cv, p.ev, p.gpsi, p.cc, p.ec, p.gchi,
                                         0.5 * (W + W.conj().T), 0.7)
    assert rel(cv.grad.cpu().numpy(), dcvo) < 1e-10
    assert rel(ev.grad.cpu().numpy(), dEvo) < 1e-10
