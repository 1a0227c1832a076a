"""Static subspace approximation (Eq. chi_mat_sub) against the oracle, and the split-precision
general product it uses (also Y = M W in the adjoint)."""
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


@pytest.fixture(scope="module")
def case():
    p = gwgen.make_problem((24, 24, 24), 6, 24, 600, 200, seed=gwgen.BASE_SEED + 31)
    M = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    chi_0 = oracle.chi0(M, oracle.delta(p.ev, p.ec, 0.0))
    lam = np.linalg.eigvalsh(chi_0)
    # a cut with a clear gap between kept and discarded eigenvalues
    neig = int(20 + np.argmax(lam[21:41] - lam[20:40]))
    return p, M, chi_0, neig


OMEGA = [0.0, 2.0, 9.0]


@pytest.mark.parametrize("prec,mtxel,tol", [("fp64", "fp64", 1e-11), ("fp64", "twofloat", 1e-11),
                                            ("ozaki", "twofloat", 1e-9)])
def test_compute_subspace_matches_oracle(gw, case, prec, mtxel, tol):
    """chi_BB'(w) on the oracle's basis, entry by entry (projection + contraction on the GPU)."""
    p, M, chi_0, neig = case
    C, _ = oracle.subspace_basis(chi_0, neig)
    h = gw.from_problem(p, prec=prec, nslices=7, mtxel=mtxel, pair_chunk=50)
    got = h.compute_subspace(0, torch.as_tensor(C, device="cuda"), OMEGA).cpu().numpy()
    h.sync()
    for i, w in enumerate(OMEGA):
        ref = oracle.chi0_subspace(M, oracle.delta(p.ev, p.ec, w), C)
        assert rel(got[i], ref) <= tol, (w, rel(got[i], ref))
        assert np.array_equal(got[i], got[i].conj().T)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("ozaki", 1e-9)])
def test_subspace_basis_and_backprojection(gw, case, prec, tol):
    """The GPU basis from the GPU chi(0): eigenvalues, the subspace projector, chi_BB'(0) =
    diag(lambda), and the back-projected C chi_BB'(w) C^H, all against the oracle's."""
    p, M, chi_0, neig = case
    C_o, lam_o = oracle.subspace_basis(chi_0, neig)
    h = gw.from_problem(p, prec=prec, nslices=7, mtxel="twofloat", pair_chunk=64)
    (chi,) = h.compute(0, [0.0])
    C, lam = h.subspace_basis(chi[0], neig)
    sub = h.compute_subspace(0, C, OMEGA)
    h.sync()
    C, lam, sub = C.cpu().numpy(), lam.cpu().numpy(), sub.cpu().numpy()
    assert rel(lam, lam_o) <= tol
    assert np.abs(C.conj().T @ C - np.eye(neig)).max() < 1e-12
    gap = (np.linalg.eigvalsh(chi_0)[neig] - lam_o[-1]) / abs(lam_o[0])
    assert rel(C @ C.conj().T, C_o @ C_o.conj().T) <= 10 * tol / gap
    assert rel(sub[0], np.diag(lam).astype(np.complex128)) <= 10 * tol
    for i, w in enumerate(OMEGA):
        ref = C_o @ oracle.chi0_subspace(M, oracle.delta(p.ev, p.ec, w), C_o) @ C_o.conj().T
        assert rel(C @ sub[i] @ C.conj().T, ref) <= 10 * tol / gap


def test_subspace_errors(gw, case):
    p, _, _, _ = case
    h = gw.from_problem(p)
    C = torch.zeros((len(p.gchi), 4), dtype=torch.complex128, device="cuda")
    with pytest.raises(gw.GwError) as e:
        h.compute_subspace(0, torch.zeros((len(p.gchi), 0), dtype=torch.complex128, device="cuda"), [0.0])
    assert e.value.status == 1
    with pytest.raises(gw.GwError) as e:
        h.subspace_basis(torch.zeros((8, 8), dtype=torch.complex128, device="cuda"), 9)
    assert e.value.status == 1
    h.compute_subspace(0, C, [0.0])  # the handle stays usable
    h.sync()


def test_adjoint_split_product(gw):
    """Adjoint with Y = M W as a split product (s = 7) against the oracle adjoint."""
    p = gwgen.make_problem((20, 20, 20), 6, 24, 300, 120, seed=77)
    W = gwgen.hermitian(np.random.default_rng(78), 120)
    Lo, dEvo, dEco, dcvo, dcco = oracle.adjoint(p.gpsi, p.cv, p.ev, p.gpsi, p.cc, p.ec, p.gchi, W, 1.5)
    h = gw.from_problem(p, prec="ozaki", nslices=7, mtxel="twofloat", pair_chunk=40)
    L, dEv, dEc, dcv, dcc = h.adjoint(0, torch.as_tensor(W, device="cuda"), omega=1.5)
    h.sync()
    assert abs(L - Lo) <= 1e-10 * abs(Lo)
    for a, b in ((dEv, dEvo), (dEc, dEco), (dcv, dcvo), (dcc, dcco)):
        assert rel(a.cpu().numpy(), b) < 1e-10


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("ozaki", 1e-9)])
def test_epsilon_inverse_matches_oracle(gw, prec, tol):
    """[I - v chi(w)]^-1 (Eq. epsilon_mat) for two frequency blocks of the oracle's chi."""
    p = gwgen.make_problem((24, 24, 24), 6, 24, 600, 200, seed=gwgen.BASE_SEED + 33)
    M = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    chis = np.stack([oracle.chi0(M, oracle.delta(p.ev, p.ec, w)) for w in (0.0, 5.0)])
    v = gwgen.coulomb(p.gchi)
    h = gw.from_problem(p, prec=prec, nslices=7)
    got = h.epsilon_inverse(torch.as_tensor(chis, device="cuda"), torch.as_tensor(v, device="cuda")).cpu().numpy()
    h.sync()
    for i in range(2):
        assert rel(got[i], oracle.epsilon_inverse(chis[i], v)) <= tol


def test_epsilon_inverse_rejects_bad_coulomb(gw):
    p = gwgen.make_problem((16, 16, 16), 2, 3, 57, 27, seed=3)
    h = gw.from_problem(p)
    chi = torch.zeros((27, 27), dtype=torch.complex128, device="cuda")
    v = torch.ones(27, dtype=torch.float64, device="cuda")
    v[3] = 0.0
    with pytest.raises(gw.GwError) as e:
        h.epsilon_inverse(chi, v)
    assert e.value.status == 1
    out = h.epsilon_inverse(chi, torch.ones(27, dtype=torch.float64, device="cuda"))  # still usable: chi = 0
    h.sync()
    assert torch.equal(out, torch.eye(27, dtype=torch.complex128, device="cuda"))


@pytest.mark.parametrize("prec,mtxel,tol", [("fp64", "fp64", 1e-11), ("ozaki", "twofloat", 1e-9)])
def test_compute_real_matches_oracle(gw, case, prec, mtxel, tol):
    """chi on the real axis with broadening, below, across and above the resonances."""
    p, M, _, _ = case
    om, eta = [0.5, 12.0, 40.0], 0.2
    h = gw.from_problem(p, prec=prec, nslices=7, mtxel=mtxel, pair_chunk=64)
    got = h.compute_real(0, om, eta).cpu().numpy()
    h.sync()
    for i, w in enumerate(om):
        assert rel(got[i], oracle.chi0_real(M, oracle.delta_real(p.ev, p.ec, w, eta))) <= tol, w


def test_compute_real_errors(gw, case):
    p = case[0]
    h = gw.from_problem(p)
    with pytest.raises(gw.GwError) as e:
        h.compute_real(0, [1.0], 0.0)
    assert e.value.status == 1
    with pytest.raises(gw.GwError) as e:
        h.compute_real(0, [1.0] * 22, 0.1)
    assert e.value.status == 1


@pytest.mark.parametrize("prec,mtxel,tol", [("fp64", "fp64", 1e-11), ("ozaki", "twofloat", 1e-9)])
def test_jvp_matches_oracle(gw, case, prec, mtxel, tol):
    """Forward derivative of chi0 along random band and energy perturbations."""
    p = case[0]
    rng = np.random.default_rng(91)
    dcv = (rng.standard_normal(p.cv.shape) + 1j * rng.standard_normal(p.cv.shape)) / np.sqrt(p.cv.shape[1])
    dcc = (rng.standard_normal(p.cc.shape) + 1j * rng.standard_normal(p.cc.shape)) / np.sqrt(p.cc.shape[1])
    dev, dec = rng.standard_normal(len(p.ev)), rng.standard_normal(len(p.ec))
    om = [0.0, 4.0]
    h = gw.from_problem(p, prec=prec, nslices=7, mtxel=mtxel, pair_chunk=64)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    got = h.jvp(0, om, t(dcv), t(dcc), t(dev), t(dec)).cpu().numpy()
    h.sync()
    for i, w in enumerate(om):
        ref = oracle.jvp(p.gpsi, p.cv, p.ev, p.cc, p.ec, p.gchi, dcv, dcc, dev, dec, w)
        assert rel(got[i], ref) <= tol, (w, rel(got[i], ref))
        assert np.array_equal(got[i], got[i].conj().T)


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_resident_pair_elements(gw, case, prec):
    """With the pair elements kept resident, the subspace, real-axis and forward-derivative calls
    that reuse them give the same bits as the ones that recompute them; new bands drop them
    (results follow the new bands)."""
    p, M, chi_0, neig = case
    C, _ = oracle.subspace_basis(chi_0, neig)
    Cd = torch.as_tensor(C, device="cuda")
    rng = np.random.default_rng(8)
    tan = lambda shape: torch.as_tensor((rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * 1e-2,
                                        device="cuda")
    dcv, dcc = tan(p.cv.shape), tan(p.cc.shape)
    dev_, dec_ = (torch.as_tensor(rng.standard_normal(n), device="cuda") for n in (len(p.ev), len(p.ec)))
    outs = {}
    for keep in (False, True):
        h = gw.from_problem(p, prec=prec, nslices=7, mtxel="twofloat")
        if keep:
            h.keep_pair_elements(True)
        h.compute(0, [0.0])
        sub = h.compute_subspace(0, Cd, OMEGA).cpu().numpy()
        real = h.compute_real(0, [3.0], 0.2).cpu().numpy()
        jv = h.jvp(0, [1.0], dcv, dcc, dev_, dec_).cpu().numpy()
        h.sync()
        outs[keep] = (sub, real, h, jv)
    assert np.array_equal(outs[False][0], outs[True][0])
    assert np.array_equal(outs[False][1], outs[True][1])
    assert np.array_equal(outs[False][3], outs[True][3])
    # new valence bands on the kept slot: the resident elements are dropped
    h = outs[True][2]
    q = gwgen.make_problem(p.grid, p.cv.shape[0], p.cc.shape[0], p.gpsi.shape[0], p.gchi.shape[0],
                           seed=gwgen.BASE_SEED + 32)
    h.set_bands(0, 0, torch.as_tensor(q.gpsi, device="cuda"), torch.as_tensor(q.cv, device="cuda"),
                torch.as_tensor(q.ev, device="cuda"))
    sub2 = h.compute_subspace(0, Cd, OMEGA).cpu().numpy()
    h.sync()
    Mq = oracle.m_conv(q.gpsi, q.cv, p.gpsi, p.cc, p.gchi)
    want = oracle.chi0_subspace(Mq, oracle.delta(q.ev, p.ec, OMEGA[1]), C)
    assert rel(sub2[1], want) < (1e-11 if prec == "fp64" else 1e-9)
    for k in outs:
        outs[k][2].destroy()
