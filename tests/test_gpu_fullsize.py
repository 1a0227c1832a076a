"""Full-size parity, in the launch configuration bench.py times, on outputs the oracle can compute.

48^3 grid, 128 + 1024 bands on 6000 plane waves, N_G = 2000, 8192-pair chunks: a sampled
block of chi (all 131072 pairs contribute) and sampled rows of M against the oracle, plus
properties that hold at any size (Hermitian, negative semidefinite at w = 0, trace), and the
split-precision chi over the whole matrix against the library's FP64 mode.  A sampled block's
norm is dominated by its diagonal (sums of squares, with the smallest relative errors), so the
block error is weighted into an estimate for the whole matrix (`strat_rel`).  The same
for the 72^3 workload (524288 pairs, N_G = 6000) in split precision, and for the batched
workload (64 q-points x 16 frequencies, uneven spheres) in one graph-captured call.
"""
import numpy as np
import pytest

import gwgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# s = 6 slices: 4.1e-10 over the whole 48^3 matrix against the FP64 mode
TOL_S6 = 1e-9


def strat_rel(got, ref, ng):
    """Relative Frobenius error over the whole ng x ng matrix, estimated from a sampled n x n
    block: its diagonal and off-diagonal entries weighted by their shares of the whole matrix."""
    n = ref.shape[0]
    on = np.eye(n, dtype=bool)
    d = got - ref
    wd, wo = ng / n, ng * (ng - 1.0) / (n * (n - 1.0))
    e = wd * np.sum(np.abs(d[on]) ** 2) + wo * np.sum(np.abs(d[~on]) ** 2)
    r = wd * np.sum(np.abs(ref[on]) ** 2) + wo * np.sum(np.abs(ref[~on]) ** 2)
    return float(np.sqrt(e / r))


@pytest.fixture(scope="module")
def gw():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_2509_23018_gb300 as gw
    return gw


@pytest.fixture(scope="module")
def c2():
    cfg = gwgen.CONFIGS["c2_48cube"]
    p = gwgen.config_problem(cfg)
    rng = np.random.default_rng(17)
    idx = np.sort(rng.choice(cfg.ng, 16, replace=False))
    Mcols = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi[idx])   # all pairs, 16 columns
    ref = oracle.chi0(Mcols, oracle.delta(p.ev, p.ec, 0.0))
    prs = np.sort(rng.choice(cfg.npairs, 16, replace=False))
    return cfg, p, idx, ref, prs


@pytest.fixture(scope="module")
def c2_fp64(gw, c2):
    """chi(0) of the 48^3 workload in the library's FP64 mode (FP64 stage (a), DMMA contraction)."""
    cfg, p, idx, ref, _ = c2
    h = gw.from_problem(p, prec="fp64", mtxel="fp64", pair_chunk=cfg.pair_chunk)
    (chi,) = h.compute(0, [0.0])
    h.sync()
    h.destroy()
    chi = chi[0].cpu().numpy()
    assert strat_rel(chi[np.ix_(idx, idx)], ref, cfg.ng) <= 1e-13
    return chi


@pytest.mark.parametrize("prec,nslices,mtxel,tol", [("fp64", 6, "fp64", 1e-11), ("ozaki", 7, "twofloat", 1e-11),
                                                    ("ozaki", 6, "twofloat", TOL_S6)])
def test_c2_sampled(gw, c2, c2_fp64, prec, nslices, mtxel, tol):
    cfg, p, idx, ref, prs = c2
    h = gw.from_problem(p, prec=prec, nslices=nslices, mtxel=mtxel, pair_chunk=cfg.pair_chunk)
    (chi,), (dg,) = h.compute(0, [0.0], diag=True)
    chi_d = chi[0]
    # properties at full size, on the device
    assert torch.equal(chi_d, chi_d.conj().T)
    ev = torch.linalg.eigvalsh(chi_d)
    assert float(ev.max()) <= 50 * tol * float(ev.abs().max())  # NSD up to the mode's error level
    # trace of chi against the independent FP64 column reduction of Delta |M|^2
    assert abs(float(torch.trace(chi_d).real) - float(dg[0].sum())) <= max(tol, 1e-12) * abs(float(dg[0].sum()))
    chi_h = chi_d.cpu().numpy()
    e = strat_rel(chi_h[np.ix_(idx, idx)], ref, cfg.ng)
    assert e <= tol, e
    if prec == "ozaki":
        e = rel(chi_h, c2_fp64)  # the whole matrix
        assert e <= tol, e
    # sampled pair rows of M (stage a alone)
    for pr in prs[:4]:
        m = h.pair_elements(0, int(pr), 1).cpu().numpy()[0]
        v, c = divmod(int(pr), cfg.nc)
        mo = oracle.m_conv(p.gpsi, p.cv[v:v + 1], p.gpsi, p.cc[c:c + 1], p.gchi)[0]
        assert rel(m, mo) < 1e-12
    h.sync()
    h.destroy()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("ozaki", 1e-9)])
def test_c2_epsilon_inverse_full_size(gw, c2, prec, tol):
    """[I - v chi(w)]^-1 at N_G = 2000 for chi(0), chi(5 eV) and chi(20 eV) of the 48^3 workload
    (the bench's --epsilon workload), element by element against the oracle's dense inverse of
    the same chi blocks, v_G = 4 pi / |G|^2."""
    cfg, p, _, _, _ = c2
    h = gw.from_problem(p, prec="ozaki", nslices=7, mtxel="twofloat", pair_chunk=cfg.pair_chunk)
    (chi,) = h.compute(0, [0.0, 5.0, 20.0])
    h.destroy()
    v = torch.as_tensor(gwgen.coulomb(p.gchi), device="cuda")
    he = gw.Chi0(cfg.grid, prec=prec, nslices=7)
    einv = he.epsilon_inverse(chi, v).cpu().numpy()
    he.sync()
    chis, vv = chi.cpu().numpy(), v.cpu().numpy()
    for i in range(3):
        assert rel(einv[i], oracle.epsilon_inverse(chis[i], vv)) <= tol


@pytest.fixture(scope="module")
def c3():
    cfg = gwgen.CONFIGS["c3_72cube"]
    p = gwgen.config_problem(cfg)
    rng = np.random.default_rng(19)
    idx = np.sort(rng.choice(cfg.ng, 6, replace=False))
    Mcols = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi[idx])   # all 524288 pairs, 6 columns
    return cfg, p, idx, oracle.chi0(Mcols, oracle.delta(p.ev, p.ec, 0.0))


def test_c3_sampled_split(gw, c3):
    """72^3, 256 + 2048 bands on 20000 plane waves, N_G = 6000, 64 chunks of 8192 pairs, split
    precision (s = 7) with two-float stage (a): a sampled block against the oracle, Hermitian and
    trace at full size."""
    cfg, p, idx, ref = c3
    h = gw.from_problem(p, prec="ozaki", nslices=7, mtxel="twofloat", pair_chunk=cfg.pair_chunk)
    (chi,), (dg,) = h.compute(0, [0.0], diag=True)
    chi_d = chi[0]
    assert torch.equal(chi_d, chi_d.conj().T)
    assert abs(float(torch.trace(chi_d).real) - float(dg[0].sum())) <= 1e-9 * abs(float(dg[0].sum()))
    got = chi_d.cpu().numpy()[np.ix_(idx, idx)]
    h.sync()
    e = strat_rel(got, ref, cfg.ng)
    assert e <= 1e-11, e
    h.destroy()


def test_adjoint_40cube_reduced_bands(gw):
    """Adjoint on the 40^3 / 4500 / 1500 shapes with reduced bands (12 + 48) vs the oracle adjoint."""
    p = gwgen.make_problem((40, 40, 40), 12, 48, 4500, 1500, seed=gwgen.BASE_SEED + 4)
    W = gwgen.hermitian(np.random.default_rng(gwgen.BASE_SEED + 4), 1500)
    Lo, dEvo, dEco, dcvo, dcco = oracle.adjoint(p.gpsi, p.cv, p.ev, p.gpsi, p.cc, p.ec, p.gchi, W, 0.0)
    h = gw.from_problem(p, mtxel="twofloat", pair_chunk=192)
    L, dEv, dEc, dcv, dcc = h.adjoint(0, torch.as_tensor(W, device="cuda"))
    h.sync()
    assert abs(L - Lo) <= 1e-10 * abs(Lo)
    for a, b in ((dEv, dEvo), (dEc, dEco), (dcv, dcvo), (dcc, dcco)):
        assert rel(a.cpu().numpy(), b) < 1e-10


def test_adjoint_c5_central_differences(gw):
    """The adjoint at the full 40^3 / 96 + 768 bands / 4500 / 1500 size in the launch configuration
    the bench times (split precision, two-float stage (a)), against central differences of the
    FP64 forward L = Re Tr(W chi) on the coefficients with the largest gradients and on two
    energies."""
    cfg = gwgen.CONFIGS["c5_adjoint"]
    p = gwgen.config_problem(cfg)
    W = gwgen.hermitian(np.random.default_rng(gwgen.BASE_SEED + 4), cfg.ng)
    Wd = torch.as_tensor(W, device="cuda")
    h = gw.from_problem(p, prec="ozaki", nslices=7, mtxel="twofloat", pair_chunk=cfg.pair_chunk)
    L, dEv, dEc, dcv, dcc = h.adjoint(0, Wd)
    h.sync()
    h.destroy()
    dcv, dcc, dEv = dcv.cpu().numpy(), dcc.cpu().numpy(), dEv.cpu().numpy()
    hf = gw.from_problem(p, prec="fp64", mtxel="twofloat", pair_chunk=cfg.pair_chunk)
    g = torch.as_tensor(p.gpsi, device="cuda")

    def L_of(cv, cc, ev, ec):
        hf.set_bands(0, 0, g, torch.as_tensor(cv, device="cuda"), torch.as_tensor(ev, device="cuda"))
        hf.set_bands(0, 1, g, torch.as_tensor(cc, device="cuda"), torch.as_tensor(ec, device="cuda"))
        (chi,) = hf.compute(0, [0.0])
        return float(torch.real(torch.trace(Wd @ chi[0])).item())

    L0 = L_of(p.cv, p.cc, p.ev, p.ec)
    assert abs(L0 - L) <= 1e-12 * abs(L)
    step = 1e-5
    checks = []
    for which, grad, base in (("v", dcv, p.cv), ("c", dcc, p.cc)):
        for flat in np.argsort(-np.abs(grad).ravel())[:2]:
            n, k = np.unravel_index(flat, grad.shape)
            for part, unit in (("re", 1.0), ("im", 1j)):
                cp, cm = base.copy(), base.copy()
                cp[n, k] += step * unit
                cm[n, k] -= step * unit
                if which == "v":
                    fd = (L_of(cp, p.cc, p.ev, p.ec) - L_of(cm, p.cc, p.ev, p.ec)) / (2 * step)
                else:
                    fd = (L_of(p.cv, cp, p.ev, p.ec) - L_of(p.cv, cm, p.ev, p.ec)) / (2 * step)
                checks.append((fd, grad[n, k].real if part == "re" else grad[n, k].imag))
    for v in np.argsort(-np.abs(dEv))[:2]:
        ep, em = p.ev.copy(), p.ev.copy()
        ep[v] += step
        em[v] -= step
        checks.append(((L_of(p.cv, p.cc, ep, p.ec) - L_of(p.cv, p.cc, em, p.ec)) / (2 * step), dEv[v]))
    hf.destroy()
    for fd, an in checks:
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_adjoint_c5_sampled_bands_vs_oracle(gw):
    """The full-size adjoint (40^3, 96 + 768 bands on 4500 plane waves, N_G = 1500, split precision
    with two-float stage (a), as the bench runs it) against the oracle adjoint on sampled bands.
    L is a sum over pairs, so one valence band's gradient (coefficients and energy) involves only
    its pairs with every conduction band, and one conduction band's only its pairs with every
    valence band: the oracle runs those one-band problems, whose gradient rows are the full
    problem's."""
    cfg = gwgen.CONFIGS["c5_adjoint"]
    p = gwgen.config_problem(cfg)
    W = gwgen.hermitian(np.random.default_rng(gwgen.BASE_SEED + 4), cfg.ng)
    h = gw.from_problem(p, prec="ozaki", nslices=7, mtxel="twofloat", pair_chunk=cfg.pair_chunk)
    _, dEv, dEc, dcv, dcc = h.adjoint(0, torch.as_tensor(W, device="cuda"))
    h.sync()
    h.destroy()
    dEv, dEc, dcv, dcc = (x.cpu().numpy() for x in (dEv, dEc, dcv, dcc))
    v = int(np.random.default_rng(29).integers(cfg.nv))
    _, dEvo, _, dcvo, _ = oracle.adjoint(p.gpsi, p.cv[v:v + 1], p.ev[v:v + 1], p.gpsi, p.cc, p.ec, p.gchi, W, 0.0)
    assert rel(dcv[v], dcvo[0]) <= 1e-9
    assert abs(dEv[v] - dEvo[0]) <= 1e-9 * float(np.abs(dEv).max())  # against the largest energy derivative
    for c in np.random.default_rng(31).choice(cfg.nc, 2, replace=False):
        _, _, dEco, _, dcco = oracle.adjoint(p.gpsi, p.cv, p.ev, p.gpsi, p.cc[c:c + 1], p.ec[c:c + 1], p.gchi,
                                             W, 0.0)
        assert rel(dcc[c], dcco[0]) <= 1e-9
        assert abs(dEc[c] - dEco[0]) <= 1e-9 * float(np.abs(dEc).max())

@pytest.fixture(scope="module")
def c4():
    cfg = gwgen.CONFIGS["c4_batch"]
    b = gwgen.make_batch(cfg.grid, cfg.nv, cfg.nc, cfg.ngpsi, 300, 3000, 4, cfg.nw, seed=gwgen.BASE_SEED + cfg.index)
    ngs = np.array([len(x) for x in b.gchi])
    rng = np.random.default_rng(23)
    refs = {}
    for iq in dict.fromkeys([0, int(np.argmin(ngs)), int(np.argmax(ngs))]):  # q = 0, smallest, largest sphere
        idx = np.sort(rng.choice(int(ngs[iq]), 8, replace=False))
        Mcols = oracle.m_conv(b.gpsi, b.cv[iq], b.gpsi, b.cc, b.gchi[iq][idx])   # all 32768 pairs, 8 columns
        refs[iq] = (idx, [oracle.chi0(Mcols, oracle.delta(b.ev[iq], b.ec, w)) for w in b.omega])
    return cfg, b, refs


def test_c4_sampled_batch(gw, c4):
    """64 q-points (N_G uniform in [300, 3000]) x 16 imaginary frequencies on 40^3, 64 + 512 bands
    on 8000 plane waves, all in one graph-captured persistent call in split precision (s = 7) with
    two-float stage (a), as the batched benchmark runs it: sampled blocks of three slots (q = 0 and
    the smallest and largest spheres) at every frequency against the oracle, every block Hermitian."""
    cfg, b, refs = c4
    h = gw.Chi0(cfg.grid, nq=len(b.qs), prec="ozaki", nslices=7, mtxel="twofloat")
    t = lambda x: torch.as_tensor(np.ascontiguousarray(x), device="cuda")
    g = t(b.gpsi)
    h.set_bands(0, 1, g, t(b.cc), t(b.ec))
    for iq in range(len(b.qs)):
        h.set_bands(iq, 0, g, t(b.cv[iq]), t(b.ev[iq]))
        h.set_gsphere(iq, t(b.gchi[iq]))
    slots = list(range(len(b.qs)))
    res = h.compute_batch(slots, list(b.omega))
    for r in res:
        assert torch.equal(r, r.conj().transpose(-1, -2))
    got = {}
    for iq, (idx, _) in refs.items():
        it = torch.as_tensor(idx, device="cuda")
        got[iq] = res[iq].index_select(1, it).index_select(2, it).cpu().numpy()
    h.sync()
    for iq, (idx, ref) in refs.items():
        for w in range(len(b.omega)):
            assert rel(got[iq][w], ref[w]) <= 1e-9, (iq, w)
    h.destroy()
