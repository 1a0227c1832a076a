"""Plain FP64 CPU oracle for the chi0 path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it, shares
no code with it and has no fallback to it.

Every function follows the paper's statement of the problem (SC'25 BerkeleyGW
paper, "Overview of the Problem"):

* ``m_conv`` -- plane-wave matrix elements M_vc(G) (definition inline after
  Eq. ff-ch) in their G-space form  M_vc(G) = sum_K conj(c_v(K)) c_c(K-G);
* ``psi_dft`` / ``m_from_psi`` / ``m_dft`` -- the same M by the real-space route of
  the definition: psi on the grid by a direct sum, the pair product, a direct
  forward sum with e^{+iG.r} and 1/N_r (tiny grids only);
* ``delta`` -- the energy factor 2/(x-iw) + 2/(x+iw), x = E_v - E_c, left open by
  Eq. chi_mat and fixed by the hot-path statement (imaginary frequency);
* ``chi0`` -- Eq. chi_mat without the outer factor 2 (the factor is folded into
  Delta), every entry summed separately with Neumaier compensation;
* ``adjoint`` -- gradients of L = Re Tr(W chi0) (GWPT motivation, Eq. gwpt);
* ``jvp`` -- the forward derivative of chi0 along band and energy perturbations (the first-order
  change GWPT builds from d psi, Eq. gwpt);
* ``delta_real`` / ``chi0_real`` -- the energy factor continued to the real axis with
  broadening (i w -> w + i eta) and chi0 with that complex Delta;
* ``epsilon_inverse`` -- Eq. epsilon_mat, [I - v chi]^-1 by a dense inverse;
* ``subspace_basis`` / ``chi0_subspace`` -- the static subspace approximation
  (Eq. chi_mat_sub and the paragraph around it): the N_Eig most significant
  eigenvectors of chi(0) as C_s, M^B = M C_s, chi_BB' from M^B as in Eq. chi_mat;
* ``gpp_pole_matrix`` / ``sigma_gpp`` -- the full-matrix (off-diagonal) plasmon-pole
  self-energy on an energy grid (section on the off-diagonal GPP kernel, Eq.
  flop_count_fullmat): the prep. step P^n(E) and the two products per (n, E).  The
  pole factor is the Hybertsen-Louie model the paper cites for the frequency dependence
  (its working equation is in a figure the text lacks).

All functions are pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle.py``
(two independent routes to M, orthonormality, Parseval, gauge and translation
covariance, Hermiticity / semidefiniteness / rank / trace of chi0, the
large-frequency limit, finite differences of L; for the self-energy a numerical
frequency integral of G W, the screened-exchange + Coulomb-hole decomposition by
brute force, Hermiticity and phase covariance).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gw_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fno-fast-math", "-ffp-contract=off",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, I, LL, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
            lib.oracle_threads.restype = I
            lib.oracle_m_conv.argtypes = [I, I, P, P, I, I, P, P, I, P, P]
            lib.oracle_m_conv.restype = I
            lib.oracle_psi_dft.argtypes = [I, I, I, I, I, P, P, P]
            lib.oracle_psi_dft.restype = None
            lib.oracle_m_from_psi.argtypes = [I, I, I, I, P, I, P, I, P, P]
            lib.oracle_m_from_psi.restype = None
            lib.oracle_delta.argtypes = [I, P, I, P, D, P, P]
            lib.oracle_delta.restype = None
            lib.oracle_chi0.argtypes = [LL, I, P, P, P]
            lib.oracle_chi0.restype = None
            lib.oracle_adjoint.argtypes = [I, I, P, P, P, I, I, P, P, P, I, P, P, D, P, P, P, P, P]
            lib.oracle_adjoint.restype = I
            _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    return int(_load().oracle_threads())


def m_conv(gv, cv, gc, cc, gchi) -> np.ndarray:
    """M [nv*nc, ng] complex128, pair index p = v*nc + c."""
    lib = _load()
    gv, gc, gchi = _c(gv, np.int32), _c(gc, np.int32), _c(gchi, np.int32)
    cv, cc = _c(cv, np.complex128), _c(cc, np.complex128)
    nv, nc, ng = cv.shape[0], cc.shape[0], gchi.shape[0]
    out = np.empty((nv * nc, ng), np.complex128)
    rc = lib.oracle_m_conv(nv, gv.shape[0], _p(gv), _p(cv), nc, gc.shape[0], _p(gc), _p(cc), ng, _p(gchi), _p(out))
    if rc:
        raise MemoryError("oracle_m_conv")
    return out


def psi_dft(grid, gk, coef) -> np.ndarray:
    """psi [nb, n0, n1, n2] = sum_K c(K) e^{+iK.r} by a direct sum."""
    lib = _load()
    gk, coef = _c(gk, np.int32), _c(coef, np.complex128)
    n0, n1, n2 = grid
    out = np.empty((coef.shape[0], n0, n1, n2), np.complex128)
    lib.oracle_psi_dft(n0, n1, n2, coef.shape[0], gk.shape[0], _p(gk), _p(coef), _p(out))
    return out


def m_from_psi(grid, psiv, psic, gchi) -> np.ndarray:
    lib = _load()
    psiv, psic, gchi = _c(psiv, np.complex128), _c(psic, np.complex128), _c(gchi, np.int32)
    n0, n1, n2 = grid
    nv, nc, ng = psiv.shape[0], psic.shape[0], gchi.shape[0]
    out = np.empty((nv * nc, ng), np.complex128)
    lib.oracle_m_from_psi(n0, n1, n2, nv, _p(psiv), nc, _p(psic), ng, _p(gchi), _p(out))
    return out


def m_dft(grid, gv, cv, gc, cc, gchi) -> np.ndarray:
    """M by the real-space route (direct sums; tiny grids only)."""
    return m_from_psi(grid, psi_dft(grid, gv, cv), psi_dft(grid, gc, cc), gchi)


def delta(ev, ec, omega: float, return_resid: bool = False):
    """Delta [nv*nc] float64 for one imaginary frequency omega (eV)."""
    lib = _load()
    ev, ec = _c(ev, np.float64), _c(ec, np.float64)
    out = np.empty(ev.shape[0] * ec.shape[0], np.float64)
    resid = np.zeros(1, np.float64)
    lib.oracle_delta(ev.shape[0], _p(ev), ec.shape[0], _p(ec), float(omega), _p(out), _p(resid))
    return (out, float(resid[0])) if return_resid else out


def chi0(M, dl) -> np.ndarray:
    """chi [ng, ng] complex128 = sum_p conj(M[p,G]) dl[p] M[p,G']."""
    lib = _load()
    M, dl = _c(M, np.complex128), _c(dl, np.float64)
    P, ng = M.shape
    out = np.empty((ng, ng), np.complex128)
    lib.oracle_chi0(P, ng, _p(M), _p(dl), _p(out))
    return out


def chi0_bands(prob, omega=None) -> np.ndarray:
    """chi0 [nw, ng, ng] for a gwgen.Problem (M by convolution)."""
    M = m_conv(prob.gpsi, prob.cv, prob.gpsi, prob.cc, prob.gchi)
    ws = prob.omega if omega is None else np.atleast_1d(omega)
    return np.stack([chi0(M, delta(prob.ev, prob.ec, w)) for w in ws])


def adjoint(gv, cv, ev, gc, cc, ec, gchi, W, omega: float = 0.0):
    """Returns (L, dL/dE_v, dL/dE_c, grad c_v, grad c_c); grad = dL/dRe + i dL/dIm."""
    lib = _load()
    gv, gc, gchi = _c(gv, np.int32), _c(gc, np.int32), _c(gchi, np.int32)
    cv, cc, W = _c(cv, np.complex128), _c(cc, np.complex128), _c(W, np.complex128)
    ev, ec = _c(ev, np.float64), _c(ec, np.float64)
    nv, nc, ng = cv.shape[0], cc.shape[0], gchi.shape[0]
    L = np.zeros(1, np.float64)
    dEv, dEc = np.empty(nv), np.empty(nc)
    dcv, dcc = np.empty_like(cv), np.empty_like(cc)
    rc = lib.oracle_adjoint(nv, gv.shape[0], _p(gv), _p(cv), _p(ev), nc, gc.shape[0], _p(gc), _p(cc), _p(ec),
                            ng, _p(gchi), _p(W), float(omega), _p(L), _p(dEv), _p(dEc), _p(dcv), _p(dcc))
    if rc:
        raise MemoryError("oracle_adjoint")
    return float(L[0]), dEv, dEc, dcv, dcc


def subspace_basis(chi_w0, neig: int):
    """The static subspace basis (paragraph of Eq. chi_mat_sub): chi(w = 0) is diagonalised
    (numpy eigh, FP64) and the neig most significant eigenvectors -- chi(0) is negative
    semidefinite, so the most negative eigenvalues -- are the columns of C_s [N_G, neig].
    Returns (C_s, eigenvalues ascending)."""
    w, v = np.linalg.eigh(np.asarray(chi_w0, np.complex128))
    return np.ascontiguousarray(v[:, :neig]), w[:neig].copy()


def chi0_subspace(M, dl, basis) -> np.ndarray:
    """Eq. chi_mat_sub: chi_BB' = sum_vc conj(M^B_vc) Delta_vc M^B'_vc with
    M^B_vc = sum_G M_vc(G) C_s[G][B] (the projection written out as a matrix product)."""
    return chi0(np.asarray(M, np.complex128) @ np.asarray(basis, np.complex128), dl)


def epsilon_inverse(chi, vcoul) -> np.ndarray:
    """Eq. epsilon_mat: eps^-1 = [I - v chi]^-1 with v the diagonal Coulomb matrix (numpy inv,
    FP64, as a library step)."""
    chi = np.asarray(chi, np.complex128)
    v = np.asarray(vcoul, np.float64)
    return np.linalg.inv(np.eye(chi.shape[0]) - v[:, None] * chi)


def delta_real(ev, ec, omega: float, eta: float) -> np.ndarray:
    """Delta_vc(w) = 2/(x - w - i eta) + 2/(x + w + i eta), x = E_v - E_c, in complex arithmetic
    (the imaginary-axis factor with i w -> w + i eta), pairs p = v * nc + c."""
    x = (np.asarray(ev, np.float64)[:, None] - np.asarray(ec, np.float64)[None, :]).ravel()
    z = complex(omega, eta)
    return 2.0 / (x - z) + 2.0 / (x + z)


def chi0_real(M, dc) -> np.ndarray:
    """chi = sum_p conj(M[p,G]) Delta_p M[p,G'] with complex Delta: the two Hermitian
    contractions with Re Delta and Im Delta (each by ``chi0``), chi_R + i chi_I."""
    dc = np.asarray(dc, np.complex128)
    return chi0(M, dc.real) + 1j * chi0(M, dc.imag)


def jvp(gpsi, cv, ev, cc, ec, gchi, dcv, dcc, dev, dec, omega: float) -> np.ndarray:
    """d chi0 along (dcv, dcc, dev, dec): M and dM = M(d psi_v, psi_c) + M(psi_v, d psi_c) by the
    G-space convolution, dDelta = d/dx [2/(x - iw) + 2/(x + iw)] (dE_v - dE_c), and
    dchi = dM^H Delta M + M^H Delta dM + M^H dDelta M (matrix products as library steps)."""
    M = m_conv(gpsi, cv, gpsi, cc, gchi)
    dM = m_conv(gpsi, dcv, gpsi, cc, gchi) + m_conv(gpsi, cv, gpsi, dcc, gchi)
    x = (np.asarray(ev, np.float64)[:, None] - np.asarray(ec, np.float64)[None, :]).ravel()
    dx = (np.asarray(dev, np.float64)[:, None] - np.asarray(dec, np.float64)[None, :]).ravel()
    dl = delta(ev, ec, omega)
    ddl = (-2.0 / (x - 1j * omega) ** 2 - 2.0 / (x + 1j * omega) ** 2).real * dx
    return (dM.conj().T * dl) @ M + (M.conj().T * dl) @ dM + (M.conj().T * ddl) @ M



def gpp_pole_matrix(omega2, wtilde, vcoul, d: float, occupied: bool) -> np.ndarray:
    """P^n_GG'(E) of the prep. step for one band n at one energy, d = E - E_n: the correlation
    part of the plasmon-pole self-energy (Hybertsen-Louie model, cited by the paper for the
    frequency dependence).  With B_GG' = v_G' Omega2_GG' / (2 wt_GG'), the residue of the
    screened interaction's pole, P = B / (d + wt) for an occupied band and B / (d - wt) for an
    empty one."""
    s = -1.0 if occupied else 1.0
    wt = np.asarray(wtilde, np.complex128)
    return np.asarray(vcoul, np.float64)[None, :] * np.asarray(omega2, np.complex128) / (2.0 * wt * (d - s * wt))


def sigma_gpp(M, En, nocc: int, omega2, wtilde, vcoul, E) -> np.ndarray:
    """Full self-energy matrix on an energy grid (section on the off-diagonal GPP kernel;
    the two products counted by Eq. flop_count_fullmat):
    Sigma_lm(E_e) = sum_n sum_GG' conj(M_n[l][G]) P^n_GG'(E_e) M_n[m][G'],
    for every (n, E_e) first X = conj(M_n) P (N_Sigma x N_G x N_G), then X M_n^T
    (N_Sigma x N_G x N_Sigma).  Returns [ne][nsig][nsig] complex128."""
    M = np.asarray(M, np.complex128)
    nb, nsig, _ = M.shape
    E = np.asarray(E, np.float64)
    out = np.zeros((len(E), nsig, nsig), np.complex128)
    for e, Ee in enumerate(E):
        for n in range(nb):
            P = gpp_pole_matrix(omega2, wtilde, vcoul, Ee - float(En[n]), n < nocc)
            out[e] += (M[n].conj() @ P) @ M[n].T
    return out
