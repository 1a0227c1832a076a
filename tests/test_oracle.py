"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a closed form,
an invariant, a second independent route, or finite differences.
"""
import numpy as np
import pytest

import gwgen
import oracle

GRID = (8, 9, 10)  # deliberately not cubic: axis mix-ups change the answer


def tiny(nv=2, nc=3, ngpsi=57, ng=19, seed=7, exclude_head=False, omega=(0.0,)):
    return gwgen.make_problem(GRID, nv, nc, ngpsi, ng, seed, omega=omega, exclude_head=exclude_head)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ------------------------------------------------------------------ M (a1-a4)

def test_sphere_alias_free():
    p = tiny()
    mk = np.abs(p.gpsi).max(0)
    mg = np.abs(p.gchi).max(0)
    assert np.all(2 * mk + mg < np.array(GRID))


def test_plane_wave_closed_form():
    """Single plane waves: M_vc(G) = 1 exactly when G = K_v - K_c (sign of e^{+iG.r})."""
    g = gwgen.gsphere(27)
    kv, kc = [3, 11], [5, 20]
    cv = np.zeros((2, 27), complex); cv[0, kv[0]] = 1; cv[1, kv[1]] = 1
    cc = np.zeros((2, 27), complex); cc[0, kc[0]] = 1; cc[1, kc[1]] = 1
    gchi = gwgen.gsphere(19)
    for M in (oracle.m_conv(g, cv, g, cc, gchi), oracle.m_dft(GRID, g, cv, g, cc, gchi)):
        for v in range(2):
            for c in range(2):
                want = np.array([np.all(gg == g[kv[v]] - g[kc[c]]) for gg in gchi], float)
                assert np.allclose(M[v * 2 + c], want, atol=1e-13)


def test_two_routes_agree():
    """G-space convolution vs direct real-space sums (brute force, tiny grid)."""
    p = tiny()
    a = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    b = oracle.m_dft(GRID, p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    assert rel(a, b) < 1e-13


def test_orthonormal_head():
    """M_mn(G=0) = <m|n> = delta_mn for orthonormal bands."""
    p = tiny()
    bands = np.concatenate([p.cv, p.cc])
    zero = np.zeros((1, 3), np.int32)
    M = oracle.m_conv(p.gpsi, bands, p.gpsi, bands, zero).reshape(5, 5)
    assert np.abs(M - np.eye(5)).max() < 1e-14
    Md = oracle.m_dft(GRID, p.gpsi, bands, p.gpsi, bands, zero).reshape(5, 5)
    assert np.abs(Md - np.eye(5)).max() < 1e-13


def test_parseval():
    """sum over all grid G of |F_p(G)|^2 = (1/N_r) sum_r |rho_p(r)|^2."""
    p = tiny()
    psv = oracle.psi_dft(GRID, p.gpsi, p.cv)
    psc = oracle.psi_dft(GRID, p.gpsi, p.cc)
    nr = np.prod(GRID)
    allg = np.stack(np.meshgrid(*[np.arange(n) for n in GRID], indexing="ij"), -1).reshape(-1, 3)
    F = oracle.m_from_psi(GRID, psv, psc, allg)
    for v in range(2):
        for c in range(3):
            rho = np.conj(psv[v]) * psc[c]
            lhs = np.sum(np.abs(F[v * 3 + c]) ** 2)
            rhs = np.sum(np.abs(rho) ** 2) / nr
            assert abs(lhs - rhs) < 1e-12 * rhs
    # the convolution route, summed over every difference vector, carries the same norm
    # (on a grid wide enough that the pair spectrum |K-K'| <= 4 does not alias)
    g2 = (9, 10, 11)
    psv, psc = oracle.psi_dft(g2, p.gpsi, p.cv), oracle.psi_dft(g2, p.gpsi, p.cc)
    d = (p.gpsi[:, None, :] - p.gpsi[None, :, :]).reshape(-1, 3)
    d = np.unique(d, axis=0)
    Fc = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, d)
    for v in range(2):
        for c in range(3):
            rho = np.conj(psv[v]) * psc[c]
            assert abs(np.sum(np.abs(Fc[v * 3 + c]) ** 2) - np.sum(np.abs(rho) ** 2) / np.prod(g2)) < 1e-12


def test_psi_normalisation():
    """(1/N_r) sum_r |psi|^2 = sum_K |c(K)|^2 = 1 (discrete Parseval for the band transform)."""
    p = tiny()
    ps = oracle.psi_dft(GRID, p.gpsi, p.cc)
    nr = np.prod(GRID)
    assert np.allclose(np.sum(np.abs(ps) ** 2, axis=(1, 2, 3)) / nr, 1.0, atol=1e-13)


def test_gauge_covariance():
    p = tiny()
    rng = np.random.default_rng(1)
    tv, tc = rng.uniform(0, 2 * np.pi, 2), rng.uniform(0, 2 * np.pi, 3)
    M = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    M2 = oracle.m_conv(p.gpsi, p.cv * np.exp(1j * tv)[:, None], p.gpsi, p.cc * np.exp(1j * tc)[:, None], p.gchi)
    ph = np.exp(1j * (tc[None, :] - tv[:, None])).reshape(-1)
    assert rel(M2, M * ph[:, None]) < 1e-14


@pytest.mark.parametrize("route", ["conv", "dft"])
def test_translation_covariance(route):
    """c(K) -> c(K) e^{-2pi i K.tau}  =>  M(G) -> e^{+2pi i G.tau} M(G)."""
    p = tiny()
    if route == "conv":
        tau = np.array([0.137, -0.41, 0.29])
        f = lambda a, b: oracle.m_conv(p.gpsi, a, p.gpsi, b, p.gchi)
    else:
        tau = np.array([3, 2, 7]) / np.array(GRID)  # a grid shift keeps the DFT route exact
        f = lambda a, b: oracle.m_dft(GRID, p.gpsi, a, p.gpsi, b, p.gchi)
    sh = np.exp(-2j * np.pi * p.gpsi @ tau)
    M = f(p.cv, p.cc)
    M2 = f(p.cv * sh[None], p.cc * sh[None])
    assert rel(M2, M * np.exp(2j * np.pi * p.gchi @ tau)[None, :]) < 1e-13


# ------------------------------------------------------------------ Delta (a5)

def test_delta_closed_form():
    rng = np.random.default_rng(3)
    ev, ec = rng.uniform(-10, -1, 5), rng.uniform(1, 30, 7)
    x = (ev[:, None] - ec[None, :]).reshape(-1)
    for w in (0.0, 0.5, 13.0, 100.0):
        d, resid = oracle.delta(ev, ec, w, return_resid=True)
        assert resid == 0.0
        assert np.allclose(d, 4 * x / (x * x + w * w), rtol=1e-15, atol=0)
        assert np.all(d < 0)
    assert np.allclose(oracle.delta(ev, ec, 0.0), 4.0 / x, rtol=1e-15)


# ------------------------------------------------------------------ chi0 (a6-a7)

@pytest.fixture(scope="module")
def chi_case():
    p = tiny(nv=2, nc=4, ngpsi=93, ng=27, omega=(0.0, 2.0, 9.0))
    M = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    return p, M


def test_chi_hermitian_nsd(chi_case):
    p, M = chi_case
    chi = oracle.chi0(M, oracle.delta(p.ev, p.ec, 0.0))
    assert np.abs(chi - chi.conj().T).max() == 0.0
    ev = np.linalg.eigvalsh(chi)
    assert ev.max() <= 1e-14 * np.abs(ev).max()


def test_chi_rank():
    p = tiny(nv=1, nc=3, ngpsi=93, ng=27)  # P = 3 < N_G = 27
    M = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    chi = oracle.chi0(M, oracle.delta(p.ev, p.ec, 0.0))
    s = np.linalg.svd(chi, compute_uv=False)
    assert np.sum(s > 1e-12 * s[0]) == 3


def test_chi_single_pair_closed_form():
    """One pair: chi_GG' = Delta conj(m_G) m_G' with Delta = 4/(E_v - E_c)."""
    p = tiny(nv=1, nc=1, ngpsi=57, ng=19)
    M = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    chi = oracle.chi0(M, oracle.delta(p.ev, p.ec, 0.0))
    m = M[0]
    assert rel(chi, 4.0 / (p.ev[0] - p.ec[0]) * np.outer(np.conj(m), m)) < 1e-15


def test_chi_plane_wave_diagonal():
    """Plane-wave bands: chi is diagonal with sum of Delta over pairs whose K_v - K_c = G."""
    g = gwgen.gsphere(57)
    kv, kc = [0, 1, 2], [3, 9, 20, 33]
    cv = np.zeros((3, 57), complex); cv[np.arange(3), kv] = 1
    cc = np.zeros((4, 57), complex); cc[np.arange(4), kc] = 1
    ev, ec = np.array([-3.0, -2.0, -5.5]), np.array([1.0, 4.0, 2.5, 7.0])
    gchi = gwgen.gsphere(57)
    M = oracle.m_conv(g, cv, g, cc, gchi)
    chi = oracle.chi0(M, oracle.delta(ev, ec, 1.5))
    want = np.zeros((57, 57), complex)
    for v in range(3):
        for c in range(4):
            d = g[kv[v]] - g[kc[c]]
            hit = np.where(np.all(gchi == d, axis=1))[0]
            x = ev[v] - ec[c]
            for h in hit:
                want[h, h] += 4 * x / (x * x + 1.5 ** 2)
    assert np.abs(chi - want).max() < 1e-15


def test_chi_trace(chi_case):
    p, M = chi_case
    d = oracle.delta(p.ev, p.ec, 2.0)
    chi = oracle.chi0(M, d)
    assert abs(np.trace(chi) - np.sum(d * np.sum(np.abs(M) ** 2, 1))) < 1e-14 * abs(np.trace(chi))


def test_chi_band_phase_invariance(chi_case):
    p, _ = chi_case
    rng = np.random.default_rng(5)
    cv2 = p.cv * np.exp(1j * rng.uniform(0, 6.3, len(p.cv)))[:, None]
    cc2 = p.cc * np.exp(1j * rng.uniform(0, 6.3, len(p.cc)))[:, None]
    d = oracle.delta(p.ev, p.ec, 0.0)
    a = oracle.chi0(oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi), d)
    b = oracle.chi0(oracle.m_conv(p.gpsi, cv2, p.gpsi, cc2, p.gchi), d)
    assert rel(b, a) < 1e-14


def test_chi_translation_pins_conjugate_side(chi_case):
    """M(G) -> e^{iG.tau} M(G) gives chi_GG' -> e^{i(G'-G).tau} chi_GG' (conj sits on the row G)."""
    p, M = chi_case
    tau = np.array([0.21, 0.05, -0.33])
    sh = np.exp(-2j * np.pi * p.gpsi @ tau)
    d = oracle.delta(p.ev, p.ec, 0.0)
    a = oracle.chi0(M, d)
    b = oracle.chi0(oracle.m_conv(p.gpsi, p.cv * sh, p.gpsi, p.cc * sh, p.gchi), d)
    ph = np.exp(2j * np.pi * p.gchi @ tau)
    assert rel(b, np.conj(ph)[:, None] * a * ph[None, :]) < 1e-13


def test_chi_frequency_monotone(chi_case):
    p, M = chi_case
    c1 = oracle.chi0(M, oracle.delta(p.ev, p.ec, 2.0))
    c2 = oracle.chi0(M, oracle.delta(p.ev, p.ec, 9.0))
    ev = np.linalg.eigvalsh(c2 - c1)
    assert ev.min() >= -1e-14 * np.abs(ev).max()


def test_chi_large_frequency_limit(chi_case):
    """w >> |x|: chi -> -(4/w^2) sum_p (E_c - E_v) conj(m_p) m_p^T."""
    p, M = chi_case
    w = 1e5
    chi = oracle.chi0(M, oracle.delta(p.ev, p.ec, w))
    x = (p.ev[:, None] - p.ec[None, :]).reshape(-1)
    lim = np.einsum("p,pg,ph->gh", 4 * x / w ** 2, np.conj(M), M)
    assert rel(chi, lim) < 1e-6


# ------------------------------------------------------------------ adjoint (a9)

@pytest.fixture(scope="module")
def adj_case():
    p = tiny(nv=2, nc=3, ngpsi=33, ng=19)
    W = gwgen.hermitian(np.random.default_rng(11), 19)
    return p, W


def _L(p, W, cv, cc, ev, ec, w=0.0):
    return oracle.adjoint(p.gpsi, cv, ev, p.gpsi, cc, ec, p.gchi, W, w)[0]


def test_adjoint_matches_trace(adj_case):
    p, W = adj_case
    for w in (0.0, 3.0):
        L = _L(p, W, p.cv, p.cc, p.ev, p.ec, w)
        chi = oracle.chi0(oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi), oracle.delta(p.ev, p.ec, w))
        assert abs(L - np.real(np.trace(W @ chi))) < 1e-13 * abs(L)


@pytest.mark.parametrize("w", [0.0, 3.0])
def test_adjoint_finite_differences(adj_case, w):
    p, W = adj_case
    L0, dEv, dEc, dcv, dcc = oracle.adjoint(p.gpsi, p.cv, p.ev, p.gpsi, p.cc, p.ec, p.gchi, W, w)
    h = 1e-6
    rng = np.random.default_rng(2)
    for _ in range(6):
        which = rng.integers(2)
        arr = p.cv if which == 0 else p.cc
        b, k = rng.integers(arr.shape[0]), rng.integers(arr.shape[1])
        for unit in (1.0, 1j):
            ap, am = arr.copy(), arr.copy()
            ap[b, k] += h * unit
            am[b, k] -= h * unit
            if which == 0:
                fd = (_L(p, W, ap, p.cc, p.ev, p.ec, w) - _L(p, W, am, p.cc, p.ev, p.ec, w)) / (2 * h)
                an = dcv[b, k]
            else:
                fd = (_L(p, W, p.cv, ap, p.ev, p.ec, w) - _L(p, W, p.cv, am, p.ev, p.ec, w)) / (2 * h)
                an = dcc[b, k]
            comp = an.real if unit == 1.0 else an.imag
            assert abs(fd - comp) < 1e-6 * max(1.0, abs(comp)), (which, b, k, unit, fd, comp)
    for i in range(2):
        e = p.ev.copy(); e[i] += h; Lp = _L(p, W, p.cv, p.cc, e, p.ec, w)
        e[i] -= 2 * h; Lm = _L(p, W, p.cv, p.cc, e, p.ec, w)
        assert abs((Lp - Lm) / (2 * h) - dEv[i]) < 1e-6 * max(1, abs(dEv[i]))
    for i in range(3):
        e = p.ec.copy(); e[i] += h; Lp = _L(p, W, p.cv, p.cc, p.ev, e, w)
        e[i] -= 2 * h; Lm = _L(p, W, p.cv, p.cc, p.ev, e, w)
        assert abs((Lp - Lm) / (2 * h) - dEc[i]) < 1e-6 * max(1, abs(dEc[i]))


def test_adjoint_rows_from_one_band_problems():
    """L = Re Tr(W chi) is a sum over pairs, so a valence band's gradient row (coefficients and
    energy) is that of the problem with this valence band alone and every conduction band, and a
    conduction band's that of the problem with it alone; the full-size GPU adjoint is checked on
    sampled bands through exactly these one-band problems."""
    p = gwgen.make_problem((12, 12, 12), 3, 5, 60, 30, seed=7)
    W = gwgen.hermitian(np.random.default_rng(3), 30)
    _, dEv, dEc, dcv, dcc = oracle.adjoint(p.gpsi, p.cv, p.ev, p.gpsi, p.cc, p.ec, p.gchi, W, 0.0)
    for v in range(3):
        _, a, _, b, _ = oracle.adjoint(p.gpsi, p.cv[v:v + 1], p.ev[v:v + 1], p.gpsi, p.cc, p.ec, p.gchi, W, 0.0)
        assert abs(a[0] - dEv[v]) <= 1e-13 * abs(dEv[v]) and np.allclose(b[0], dcv[v], rtol=0, atol=1e-13 * abs(dcv).max())
    for c in range(5):
        _, _, e, _, f = oracle.adjoint(p.gpsi, p.cv, p.ev, p.gpsi, p.cc[c:c + 1], p.ec[c:c + 1], p.gchi, W, 0.0)
        assert abs(e[0] - dEc[c]) <= 1e-13 * abs(dEc[c]) and np.allclose(f[0], dcc[c], rtol=0, atol=1e-13 * abs(dcc).max())


def test_adjoint_identity_W_energy_closed_form(adj_case):
    """W = I: L = sum_p Delta_p |m_p|^2 and dL/dE_v = sum_c |m_vc|^2 4(w^2-x^2)/(x^2+w^2)^2."""
    p, _ = adj_case
    w = 1.7
    L, dEv, dEc, _, _ = oracle.adjoint(p.gpsi, p.cv, p.ev, p.gpsi, p.cc, p.ec, p.gchi, np.eye(19), w)
    M = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    n2 = np.sum(np.abs(M) ** 2, 1).reshape(2, 3)
    x = p.ev[:, None] - p.ec[None, :]
    dd = 4 * (w * w - x * x) / (x * x + w * w) ** 2
    assert abs(L - np.sum(4 * x / (x * x + w * w) * n2)) < 1e-14 * abs(L)
    assert np.allclose(dEv, np.sum(n2 * dd, 1), rtol=1e-13)
    assert np.allclose(dEc, -np.sum(n2 * dd, 0), rtol=1e-13)


# ------------------------------------------------------------------ static subspace (next row f1)

@pytest.fixture(scope="module")
def sub_case():
    p = tiny(nv=3, nc=8, ngpsi=93, ng=27, seed=19)
    M = oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi)
    chi_0 = oracle.chi0(M, oracle.delta(p.ev, p.ec, 0.0))
    return p, M, chi_0


def test_subspace_basis_eigenpairs(sub_case):
    """C_s is orthonormal, chi(0) C_s = C_s diag(lambda), and the kept eigenvalues are the most
    negative ones (chi(0) is negative semidefinite: the most significant)."""
    _, _, chi_0 = sub_case
    C, lam = oracle.subspace_basis(chi_0, 8)
    assert np.abs(C.conj().T @ C - np.eye(8)).max() < 1e-13
    assert rel(chi_0 @ C, C * lam) < 1e-13
    rest = np.linalg.eigvalsh(chi_0)[8:]
    assert lam.max() <= rest.min() and lam.max() < 0


def test_subspace_chi_at_zero_is_diagonal(sub_case):
    """At w = 0 the subspace polarizability is the eigenvalue matrix: C_s^H chi(0) C_s = diag(lambda)."""
    p, M, chi_0 = sub_case
    C, lam = oracle.subspace_basis(chi_0, 8)
    cs = oracle.chi0_subspace(M, oracle.delta(p.ev, p.ec, 0.0), C)
    assert rel(cs, np.diag(lam).astype(np.complex128)) < 1e-12


@pytest.mark.parametrize("w", [2.0, 9.0])
def test_subspace_chi_is_projected_chi(sub_case, w):
    """chi_BB'(w) from M^B = M C_s equals C_s^H chi_GG'(w) C_s (the two representations the
    paper connects), and with the full basis the back-projection C_s chi_BB' C_s^H is chi(w)."""
    p, M, chi_0 = sub_case
    dl = oracle.delta(p.ev, p.ec, w)
    chi_w = oracle.chi0(M, dl)
    C, _ = oracle.subspace_basis(chi_0, 8)
    assert rel(oracle.chi0_subspace(M, dl, C), C.conj().T @ chi_w @ C) < 1e-12
    Cf, _ = oracle.subspace_basis(chi_0, chi_0.shape[0])
    assert rel(Cf @ oracle.chi0_subspace(M, dl, Cf) @ Cf.conj().T, chi_w) < 1e-12


# ------------------------------------------------------------------ dielectric inverse (next row f2)

def test_epsilon_diagonal_closed_form():
    """A diagonal chi gives eps^-1 = diag(1 / (1 - v_G chi_GG))."""
    c = -np.linspace(0.1, 2.0, 7)
    v = np.linspace(0.5, 3.0, 7)
    assert rel(oracle.epsilon_inverse(np.diag(c).astype(np.complex128), v), np.diag(1.0 / (1.0 - v * c))) < 1e-15


def test_epsilon_structure():
    """v^-1/2 eps^-1 v^1/2 = [I - v^1/2 chi v^1/2]^-1 is Hermitian with eigenvalues in (0, 1]
    (chi <= 0), and to first order in v, eps^-1 = I + v chi (v multiplies from the left)."""
    p = tiny(nv=3, nc=8, ngpsi=93, ng=27, seed=19, exclude_head=True)
    chi_0 = oracle.chi0(oracle.m_conv(p.gpsi, p.cv, p.gpsi, p.cc, p.gchi), oracle.delta(p.ev, p.ec, 0.0))
    v = gwgen.coulomb(p.gchi)
    e = oracle.epsilon_inverse(chi_0, v)
    s = np.sqrt(v)
    h = e * s[None, :] / s[:, None]
    assert rel(h, h.conj().T) < 1e-13
    lam = np.linalg.eigvalsh(0.5 * (h + h.conj().T))
    assert lam.min() > 0 and lam.max() <= 1 + 1e-13
    t = 1e-6
    e1 = oracle.epsilon_inverse(chi_0, t * v)
    assert rel((e1 - np.eye(len(v))) / t, v[:, None] * chi_0) < 1e-5


# ------------------------------------------------------------------ real axis (next row f3)

def test_delta_real_limits():
    """Away from the poles and for eta -> 0, Delta = 2/(x - w) + 2/(x + w); at w = 0 with
    eta = w' it is the imaginary-axis factor at w' (the continuation i w' -> w + i eta)."""
    ev, ec = np.array([-3.0, -1.5]), np.array([2.0, 4.5, 7.0])
    x = (ev[:, None] - ec[None, :]).ravel()
    d = oracle.delta_real(ev, ec, 0.7, 1e-12)
    assert np.abs(d - (2 / (x - 0.7) + 2 / (x + 0.7))).max() < 1e-10
    assert np.abs(oracle.delta_real(ev, ec, 0.0, 2.5) - oracle.delta(ev, ec, 2.5)).max() < 1e-15


@pytest.mark.parametrize("w", [0.5, 9.0])
def test_chi_real_absorptive_part(sub_case, w):
    """chi(w) = chi_R + i chi_I with chi_I = (chi - chi^H)/(2i) negative semidefinite for w >= 0
    (absorption), and chi_R = (chi + chi^H)/2 the contraction with Re Delta."""
    p, M, _ = sub_case
    dc = oracle.delta_real(p.ev, p.ec, w, 0.3)
    chi = oracle.chi0_real(M, dc)
    ci = (chi - chi.conj().T) / 2j
    assert np.linalg.eigvalsh(ci).max() <= 1e-13 * np.abs(ci).max()
    assert rel((chi + chi.conj().T) / 2, oracle.chi0(M, dc.real)) < 1e-14


@pytest.mark.parametrize("w", [0.0, 3.0])
def test_jvp_central_differences(w):
    """The forward derivative against central differences of chi0 along the same direction."""
    p = tiny(nv=2, nc=4, ngpsi=93, ng=27, seed=23)
    rng = np.random.default_rng(24)
    dcv = rng.standard_normal(p.cv.shape) + 1j * rng.standard_normal(p.cv.shape)
    dcc = rng.standard_normal(p.cc.shape) + 1j * rng.standard_normal(p.cc.shape)
    dev, dec = rng.standard_normal(len(p.ev)), rng.standard_normal(len(p.ec))
    got = oracle.jvp(p.gpsi, p.cv, p.ev, p.cc, p.ec, p.gchi, dcv, dcc, dev, dec, w)

    def chi(t):
        M = oracle.m_conv(p.gpsi, p.cv + t * dcv, p.gpsi, p.cc + t * dcc, p.gchi)
        return oracle.chi0(M, oracle.delta(p.ev + t * dev, p.ec + t * dec, w))

    h = 1e-6
    assert rel(got, (chi(h) - chi(-h)) / (2 * h)) < 1e-7


# ------------------------------------------------------------------ off-diagonal plasmon-pole self-energy

def _sigma_by_frequency_integral(B, eps, occupied, wt, eta, E, n=400001, scale=10.0):
    """(i/2pi) int dw G(E + w) W_c(w) for one band and one plane wave, by quadrature on the real
    axis (w = scale tan(theta), trapezoid in theta).  G(z) = 1/(z - eps + i eta sgn), sgn = -1 for
    an occupied band; W_c(w) = B [1/(w - wt + i eta) - 1/(w + wt - i eta)], the time-ordered
    plasmon-pole screened interaction whose spectral weight B sits at +-wt."""
    th = np.linspace(-np.pi / 2, np.pi / 2, n)[1:-1]
    w = scale * np.tan(th)
    jac = scale / np.cos(th) ** 2
    sg = -1.0 if occupied else 1.0
    G = 1.0 / (E + w - eps + 1j * eta * sg)
    W = B * (1.0 / (w - wt + 1j * eta) - 1.0 / (w + wt - 1j * eta))
    f = G * W * jac
    return 1j / (2 * np.pi) * np.trapezoid(f, th)


@pytest.mark.parametrize("occupied", [True, False])
def test_gpp_pole_matches_frequency_integral(occupied):
    """The pole factor is the frequency convolution of G and the plasmon-pole W: closing the contour
    puts an empty band at E - eps - wt and an occupied one at E - eps + wt (with the damping
    eta entering twice, wt -> wt - 2 i eta), both with residue B = v Omega^2 / (2 wt)."""
    B, wt, eta = 2.5, 12.0, 0.3
    eps = -3.0 if occupied else 4.0
    wc = wt - 2j * eta
    v = np.array([1.7])
    om2 = np.array([[2.0 * wc * B / v[0]]])
    for E in (-1.0, 0.5, 2.0, 9.0):
        want = _sigma_by_frequency_integral(B, eps, occupied, wt, eta, E)
        got = oracle.sigma_gpp(np.ones((1, 1, 1), complex), np.array([eps]), 1 if occupied else 0, om2,
                               np.array([[wc]]), v, np.array([E]))[0, 0, 0]
        assert abs(got - want) < 1e-6 * abs(want), (E, got, want)


def test_gpp_screened_exchange_coulomb_hole_brute_force():
    """Quadruple loop over (n, G, G') in the screened-exchange + Coulomb-hole form of the same model:
    CH = (1/2) Omega^2 v / (wt (d - wt)) for every band, SX - X = -Omega^2 v / (d^2 - wt^2) for the
    occupied ones.  Catches a wrong occupied/empty pole, a dropped 1/2, v on the wrong index and a
    conjugate on the wrong side."""
    p = gwgen.make_gpp(nb=3, nocc=1, nsig=2, ng=9, ne=2, seed=5)  # two |G| shells: v varies
    nb, nsig, ng = p.M.shape
    got = oracle.sigma_gpp(p.M, p.En, p.nocc, p.omega2, p.wtilde, p.vcoul, p.E)
    for e in range(len(p.E)):
        for l in range(nsig):
            for m in range(nsig):
                acc = 0j
                for n in range(nb):
                    d = p.E[e] - p.En[n]
                    for G in range(ng):
                        for Gp in range(ng):
                            o2, wt, v = p.omega2[G, Gp], p.wtilde[G, Gp], p.vcoul[Gp]
                            f = 0.5 * o2 * v / (wt * (d - wt))
                            if n < p.nocc:
                                f += -o2 * v / (d * d - wt * wt)
                            acc += np.conj(p.M[n, l, G]) * f * p.M[n, m, Gp]
                assert abs(got[e, l, m] - acc) < 1e-13 * max(1.0, abs(acc))


def test_gpp_hermitian_and_phase_covariance():
    """With a real symmetric mode energy and a Hermitian residue v_G' Omega^2_GG' / (2 wt), every
    P^n(E) is Hermitian at real E, so Sigma(E) is Hermitian; a phase on band l of the self-energy
    set multiplies Sigma_lm by e^{-i phi_l} e^{i phi_m}; a phase on a summed band n drops out."""
    rng = np.random.default_rng(9)
    p = gwgen.make_gpp(nb=5, nocc=2, nsig=4, ng=7, ne=3, seed=9)
    ng = p.M.shape[2]
    wt = p.wtilde.real.copy()
    H = gwgen.hermitian(rng, ng)
    om2 = 2.0 * wt * H / p.vcoul[None, :]
    s = oracle.sigma_gpp(p.M, p.En, p.nocc, om2, wt, p.vcoul, p.E)
    for e in range(len(p.E)):
        assert np.abs(s[e] - s[e].conj().T).max() < 1e-13 * np.abs(s[e]).max()
    s = oracle.sigma_gpp(p.M, p.En, p.nocc, p.omega2, p.wtilde, p.vcoul, p.E)
    phi = rng.uniform(0, 2 * np.pi, p.M.shape[1])
    th = rng.uniform(0, 2 * np.pi, p.M.shape[0])
    M2 = p.M * np.exp(1j * phi)[None, :, None] * np.exp(1j * th)[:, None, None]
    s2 = oracle.sigma_gpp(M2, p.En, p.nocc, p.omega2, p.wtilde, p.vcoul, p.E)
    want = s * np.exp(-1j * phi)[None, :, None] * np.exp(1j * phi)[None, None, :]
    assert np.abs(s2 - want).max() < 1e-13 * np.abs(s).max()
