"""Off-diagonal plasmon-pole self-energy (section on the off-diagonal GPP kernel) through the C ABI,
FP64 (DMMA) and split precision (BF16 tensor cores), against the oracle."""
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


def handle(gw, prec):
    return gw.Chi0((8, 8, 8), prec=prec, nslices=7)


def run(h, p):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = h.sigma_gpp(t(p.M), p.En, p.nocc, t(p.omega2), t(p.wtilde), t(p.vcoul), p.E)
    res = out.cpu().numpy()
    h.sync()
    return res


def want(p):
    return oracle.sigma_gpp(p.M, p.En, p.nocc, p.omega2, p.wtilde, p.vcoul, p.E)


CASES = [  # (nb, nocc, nsig, ng, ne)
    (5, 2, 9, 100, 3),
    (3, 1, 33, 257, 5),      # ragged: ng and nsig off every tile edge
    (2, 2, 1, 1, 2),         # one self-energy band, one plane wave, all bands occupied
    (4, 0, 130, 300, 20),    # two row tiles, more energies than one batch of the split path
    (2, 1, 16, 4500, 2),     # inner dimension 9000 real: two accumulation segments per slice group
]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("ozaki", 1e-9)])
@pytest.mark.parametrize("nb,nocc,nsig,ng,ne", CASES)
def test_sigma_gpp_parity(gw, prec, tol, nb, nocc, nsig, ng, ne):
    p = gwgen.make_gpp(nb, nocc, nsig, ng, ne, seed=gwgen.BASE_SEED + 41 + ng)
    h = handle(gw, prec)
    got = run(h, p)
    assert rel(got, want(p)) < tol
    h.destroy()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("ozaki", 1e-9)])
def test_sigma_gpp_two_thousand_plane_waves(gw, prec, tol):
    """A dielectric sphere of 2000 G (16 column tiles of the first product) and 64 bands."""
    p = gwgen.make_gpp(2, 1, 64, 2000, 2, seed=gwgen.BASE_SEED + 43)
    h = handle(gw, prec)
    got = run(h, p)
    w = want(p)
    assert rel(got, w) < tol
    for e in range(len(p.E)):  # entrywise, relative to the block's scale
        assert np.abs(got[e] - w[e]).max() < 10 * tol * np.abs(w[e]).max()
    h.destroy()


def test_sigma_gpp_hermitian_inputs(gw):
    """Real symmetric mode energies and a Hermitian residue give a Hermitian Sigma(E); the split path
    keeps it to its tolerance."""
    rng = np.random.default_rng(3)
    p = gwgen.make_gpp(3, 1, 40, 150, 3, seed=5)
    wt = p.wtilde.real.copy() + 0.0j
    H = gwgen.hermitian(rng, 150)
    p.omega2 = 2.0 * wt * H / p.vcoul[None, :]
    p.wtilde = wt
    # keep every energy off the real poles E_n +- wt
    p.E = np.array([-0.3, 0.2, 0.45])
    h = handle(gw, "ozaki")
    got = run(h, p)
    for e in range(3):
        assert np.abs(got[e] - got[e].conj().T).max() < 1e-9 * np.abs(got[e]).max()
    assert rel(got, want(p)) < 1e-9
    h.destroy()


def test_sigma_gpp_edges_and_errors(gw):
    p = gwgen.make_gpp(2, 1, 5, 20, 2, seed=7)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for prec in ("fp64", "ozaki"):
        h = handle(gw, prec)
        args = (t(p.omega2), t(p.wtilde), t(p.vcoul))
        z = h.sigma_gpp(t(p.M[:0]), [], 0, *args, p.E).cpu().numpy()
        assert z.shape == (2, 5, 5) and not np.any(z)
        assert h.sigma_gpp(t(p.M), p.En, 1, *args, []).shape == (0, 5, 5)
        with pytest.raises(gw.GwError):
            h.sigma_gpp(t(p.M), p.En, 3, *args, p.E)          # nocc > nb
        with pytest.raises(gw.GwError):
            h.sigma_gpp(t(p.M), p.En, 1, *args, [0.0, np.nan])
        a = h.sigma_gpp(t(p.M), p.En, 1, *args, p.E).cpu().numpy()
        b = h.sigma_gpp(t(p.M), p.En, 1, *args, p.E).cpu().numpy()
        h.sync()
        assert np.array_equal(a, b)                           # no atomics: replays are identical
        assert rel(a, want(p)) < (1e-11 if prec == "fp64" else 1e-9)
        h.destroy()


@pytest.mark.parametrize("nslices,tol", [(4, 1e-3), (5, 1e-5), (8, 1e-9)])
def test_sigma_gpp_slice_counts(gw, nslices, tol):
    """Every digit layout of the prep. kernel (the low/high split of the scaled pole falls
    inside, at and beyond the digits taken): error falls with the slice count."""
    p = gwgen.make_gpp(2, 1, 24, 400, 3, seed=gwgen.BASE_SEED + 44)
    h = gw.Chi0((8, 8, 8), prec="ozaki", nslices=nslices)
    got = run(h, p)
    assert rel(got, want(p)) < tol
    h.destroy()


def test_sigma_gpp_energy_batches_do_not_change_bits(gw):
    """A small memory budget (three energies of P slices per prep. launch) and the default one
    (all sixteen of an energy batch) give the same bits: 3 bands x 20 energies cross both the
    P batches and the 16-energy batches of the second product."""
    p = gwgen.make_gpp(3, 1, 20, 700, 20, seed=gwgen.BASE_SEED + 45)
    outs = []
    for budget in (0, 4 * 3 * 7 * 700 * 1408 * 2):  # kpad = 1408 for 700 G
        h = gw.Chi0((8, 8, 8), prec="ozaki", nslices=7, mem_budget_bytes=budget)
        outs.append(run(h, p))
        h.destroy()
    assert np.array_equal(outs[0], outs[1])
    assert rel(outs[0], want(p)) < 1e-9


def test_sigma_gpp_from_stage_a(gw):
    """The self-energy fed by stage (a): the summed bands n as the valence set and the self-energy
    bands l as the conduction set give M[n][l][G] = sum_K conj(c_n(K)) c_l(K - G) from
    gw_chi0_pair_elements (pair p = n N_Sigma + l), then Sigma from those elements."""
    nb, nocc, nsig, ng, ne = 6, 3, 10, 150, 4
    prob = gwgen.make_problem((24, 24, 24), nb, nsig, 400, ng, seed=gwgen.BASE_SEED + 46)
    gp = gwgen.make_gpp(nb, nocc, nsig, ng, ne, seed=gwgen.BASE_SEED + 47)
    h = gw.from_problem(prob, prec="ozaki", nslices=7, mtxel="twofloat")
    M = h.pair_elements(0, 0, nb * nsig).view(nb, nsig, ng)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    En = np.concatenate([prob.ev, prob.ec])[:nb]
    got = h.sigma_gpp(M, En, nocc, t(gp.omega2), t(gp.wtilde), t(gp.vcoul), gp.E).cpu().numpy()
    h.sync()
    Mo = oracle.m_conv(prob.gpsi, prob.cv, prob.gpsi, prob.cc, prob.gchi).reshape(nb, nsig, ng)
    want = oracle.sigma_gpp(Mo, En, nocc, gp.omega2, gp.wtilde, gp.vcoul, gp.E)
    assert rel(got, want) < 1e-9
    h.destroy()
