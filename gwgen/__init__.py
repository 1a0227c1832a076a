"""Seeded synthetic inputs for the chi0 path (shared by the oracle tests and the CUDA path).

This module only *draws* inputs: G-vector lists, orthonormal random plane-wave
coefficients, band energies, imaginary frequencies and Hermitian test matrices.
It holds none of the method's arithmetic (no pair products, no transforms, no
energy factor, no contraction), so the oracle and the CUDA path can both take
their inputs from here without sharing any computation.

Readings of the paper used here (the paper gives no input recipe; its systems
are real crystals whose wavefunctions are not available):

* cubic cell, reciprocal lattice vectors = identity in Miller-index units;
* a sphere of n G-vectors = the first n integer triples ordered by |q+G|^2,
  ties broken lexicographically on (Gx, Gy, Gz); the dielectric sphere at q=0
  omits the head G=0 ("G=0 head excluded");
* band coefficients: Re and Im i.i.d. N(0,1) drawn with numpy's default_rng,
  then orthonormalised jointly over all N_v + N_c bands in band order (valence
  first).  Gram-Schmidt in that order equals the QR factorisation whose R has a
  positive real diagonal, which is how it is computed here;
* energies: valence uniform in [-10, -1] eV, conduction uniform in [1, 30] eV,
  drawn independently (not sorted);
* imaginary frequencies: n-point Gauss-Legendre nodes on [-1, 1] mapped
  linearly onto [lo, hi] eV.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

BASE_SEED = 20250923


def gsphere(n: int, q: Sequence[float] = (0.0, 0.0, 0.0), exclude_zero: bool = False) -> np.ndarray:
    """First ``n`` integer G ordered by (|q+G|^2, Gx, Gy, Gz); int32 [n, 3]."""
    if n <= 0:
        return np.zeros((0, 3), np.int32)
    q = np.asarray(q, np.float64)
    r = int(math.ceil((3.0 * n / (4.0 * math.pi)) ** (1.0 / 3.0))) + 3
    while True:
        ax = np.arange(-r, r + 1)
        g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
        if exclude_zero:
            g = g[np.any(g != 0, axis=1)]
        k2 = ((g + q) ** 2).sum(1)
        order = np.lexsort((g[:, 2], g[:, 1], g[:, 0], k2))
        g = g[order]
        k2 = k2[order]
        # the shell at radius r-1 is complete inside the cube, so the first n are exact
        if len(g) >= n and k2[n - 1] < (r - 1 - np.abs(q).max()) ** 2:
            return np.ascontiguousarray(g[:n].astype(np.int32))
        r += 2


def orthonormal_bands(rng: np.random.Generator, nb: int, ngpsi: int) -> np.ndarray:
    """nb orthonormal complex128 coefficient rows of length ngpsi (Gram-Schmidt order)."""
    if nb > ngpsi:
        raise ValueError("more bands than plane waves")
    raw = rng.standard_normal((nb, ngpsi, 2))
    a = raw[..., 0] + 1j * raw[..., 1]
    q, r = np.linalg.qr(a.T)  # a.T = q r, columns of q orthonormal
    d = np.diag(r)
    ph = d / np.abs(d)  # make diag(r) real positive: the Gram-Schmidt factorisation
    q = q * ph[None, :]
    return np.ascontiguousarray(q.T.astype(np.complex128))


def band_energies(rng: np.random.Generator, nv: int, nc: int):
    ev = rng.uniform(-10.0, -1.0, nv)
    ec = rng.uniform(1.0, 30.0, nc)
    return ev.astype(np.float64), ec.astype(np.float64)


def gl_freqs(n: int = 16, lo: float = 0.0, hi: float = 100.0) -> np.ndarray:
    x, _ = np.polynomial.legendre.leggauss(n)
    return (lo + (hi - lo) * 0.5 * (x + 1.0)).astype(np.float64)


def hermitian(rng: np.random.Generator, n: int) -> np.ndarray:
    raw = rng.standard_normal((n, n, 2))
    a = raw[..., 0] + 1j * raw[..., 1]
    return np.ascontiguousarray(0.5 * (a + a.conj().T))


def qgrid(m: int = 4) -> np.ndarray:
    """Uniform m x m x m grid of q in reciprocal units, q_i in {0, 1/m, ..., (m-1)/m}."""
    ax = np.arange(m) / m
    return np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)


@dataclasses.dataclass(frozen=True)
class Config:
    name: str
    grid: tuple
    nv: int
    nc: int
    ngpsi: int
    ng: int
    nw: int = 1
    nq: int = 1
    pair_chunk: int = 8192
    index: int = 0

    @property
    def npairs(self) -> int:
        return self.nv * self.nc


# Workloads shaped like the ones the paper's chi0 path runs (sizes stated in the bench docs).
CONFIGS = {
    "c1_24cube": Config("c1_24cube", (24, 24, 24), 16, 64, 600, 200, index=0),
    "c2_48cube": Config("c2_48cube", (48, 48, 48), 128, 1024, 6000, 2000, index=1),
    "c3_72cube": Config("c3_72cube", (72, 72, 72), 256, 2048, 20000, 6000, index=2),
    "c4_batch": Config("c4_batch", (40, 40, 40), 64, 512, 8000, 3000, nw=16, nq=64, index=3),
    "c5_adjoint": Config("c5_adjoint", (40, 40, 40), 96, 768, 4500, 1500, index=4),
    # one 8192-pair chunk of the 48^3 workload: the small case kernel profiles are taken on
    "p1_48cube_onechunk": Config("p1_48cube_onechunk", (48, 48, 48), 8, 1024, 6000, 2000, index=1),
    # one 8192-pair chunk of the 48^3 workload as the tensor-core stage (a) forms it (all 128
    # valence bands x 64 conduction bands): the small case its kernel profiles are taken on
    "p2_48cube_chunk": Config("p2_48cube_chunk", (48, 48, 48), 128, 64, 6000, 2000, index=1),
    # one 8192-pair chunk of the 72^3 workload (slice-count sweep)
    "p3_72cube_onechunk": Config("p3_72cube_onechunk", (72, 72, 72), 4, 2048, 20000, 6000, index=2),
}


@dataclasses.dataclass
class Problem:
    grid: tuple
    gpsi: np.ndarray      # [ngpsi, 3] int32, shared by valence and conduction
    cv: np.ndarray        # [nv, ngpsi] complex128
    cc: np.ndarray        # [nc, ngpsi] complex128
    ev: np.ndarray        # [nv] float64, eV
    ec: np.ndarray        # [nc] float64, eV
    gchi: np.ndarray      # [ng, 3] int32
    omega: np.ndarray     # [nw] float64, imaginary-axis magnitudes in eV
    q: tuple = (0.0, 0.0, 0.0)


def make_problem(grid, nv, nc, ngpsi, ng, seed, omega=(0.0,), q=(0.0, 0.0, 0.0),
                 exclude_head: Optional[bool] = None) -> Problem:
    """One q-point: orthonormal valence+conduction bands, energies and the chi sphere."""
    rng = np.random.default_rng(seed)
    gpsi = gsphere(ngpsi)
    bands = orthonormal_bands(rng, nv + nc, ngpsi)
    ev, ec = band_energies(rng, nv, nc)
    if exclude_head is None:
        exclude_head = not np.any(np.asarray(q) != 0)
    gchi = gsphere(ng, q=q, exclude_zero=exclude_head)
    return Problem(tuple(grid), gpsi, np.ascontiguousarray(bands[:nv]), np.ascontiguousarray(bands[nv:]),
                   ev, ec, gchi, np.asarray(omega, np.float64), tuple(q))


def config_problem(cfg: Config, seed: Optional[int] = None, omega=None) -> Problem:
    seed = BASE_SEED + cfg.index if seed is None else seed
    if omega is None:
        omega = gl_freqs(cfg.nw) if cfg.nw > 1 else (0.0,)
    return make_problem(cfg.grid, cfg.nv, cfg.nc, cfg.ngpsi, cfg.ng, seed, omega=omega)


@dataclasses.dataclass
class BatchProblem:
    """Many q-points: conduction bands at k shared, one valence set per q (bands at k+q)."""
    grid: tuple
    gpsi: np.ndarray
    cc: np.ndarray
    ec: np.ndarray
    qs: np.ndarray          # [nq, 3]
    cv: list                # nq x [nv, ngpsi]
    ev: list                # nq x [nv]
    gchi: list              # nq x [ng_q, 3]
    omega: np.ndarray


def make_batch(grid, nv, nc, ngpsi, ng_lo, ng_hi, nq_side, nw, seed) -> BatchProblem:
    rng = np.random.default_rng(seed)
    gpsi = gsphere(ngpsi)
    qs = qgrid(nq_side)
    cond = orthonormal_bands(rng, nc, ngpsi)
    ec = rng.uniform(1.0, 30.0, nc)
    ngs = rng.integers(ng_lo, ng_hi + 1, len(qs))
    cvs, evs, gch = [], [], []
    for iq, q in enumerate(qs):
        r = np.random.default_rng([seed, iq])
        # valence at k+q: orthonormal among themselves; orthogonality to the
        # conduction set at k is not required at q != 0
        cvs.append(orthonormal_bands(r, nv, ngpsi))
        evs.append(r.uniform(-10.0, -1.0, nv))
        gch.append(gsphere(int(ngs[iq]), q=q, exclude_zero=not np.any(q != 0)))
    return BatchProblem(tuple(grid), gpsi, cond, ec, qs, cvs, evs, gch, gl_freqs(nw))


def coulomb(gchi, q=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Synthetic Coulomb diagonal v_G = 4 pi / |q + G|^2 (reciprocal-lattice index units) for the
    dielectric-matrix inputs; G = 0 at q = 0 must not be in the sphere."""
    k = np.asarray(gchi, np.float64) + np.asarray(q, np.float64)
    return 4.0 * np.pi / np.einsum("ij,ij->i", k, k)



@dataclasses.dataclass
class GppProblem:
    """Inputs of the off-diagonal plasmon-pole self-energy: matrix elements between the summed
    bands n and the self-energy bands l, band energies, plasmon-pole parameters, the Coulomb
    diagonal and the energy grid."""
    M: np.ndarray           # [nb, nsig, ng] complex128, M[n][l][G]
    En: np.ndarray          # [nb] float64, eV
    nocc: int               # bands n < nocc are occupied
    omega2: np.ndarray      # [ng, ng] complex128, Omega^2_GG' (eV^2)
    wtilde: np.ndarray      # [ng, ng] complex128, mode energies (eV)
    vcoul: np.ndarray       # [ng] float64
    E: np.ndarray           # [ne] float64, eV
    gchi: np.ndarray        # [ng, 3] int32


def make_gpp(nb: int, nocc: int, nsig: int, ng: int, ne: int, seed: int, wp: float = 16.6, eta: float = 0.25,
             ewin=(-6.0, 6.0), q=(0.0, 0.0, 0.0)) -> GppProblem:
    """Synthetic plasmon-pole inputs with the structure of the Hybertsen-Louie model:

    * M: Re and Im i.i.d. N(0, 1/(2 ng)) (matrix elements of unit-norm band products);
    * E_n: occupied uniform in [-10, -1] eV, empty uniform in [1, 30] eV (bands n < nocc occupied);
    * Omega^2_GG' = wp^2 exp(-|G - G'|^2 / 8) e^{i(t_G - t_G')}: wp^2 on the diagonal (the
      plasma frequency, 16.6 eV for silicon), decaying with |G - G'| like the charge density
      rho(G - G') the model scales it by, Hermitian (t_G uniform phases);
    * wtilde_GG' = wp (1 + (u_G + u_G') / 2) - i eta: mode energies between wp and 2 wp, symmetric,
      with a damping eta so that no energy of the grid sits on a pole;
    * v_G = 4 pi / |q + G|^2 on the sphere (G = 0 left out at q = 0);
    * E: ne points spaced evenly over the window ``ewin`` (the energy range of the self-energy
      bands, where the full-matrix solution of Dyson's equation needs Sigma)."""
    rng = np.random.default_rng(seed)
    gchi = gsphere(ng, q=q, exclude_zero=not np.any(np.asarray(q) != 0))
    scale = 1.0 / math.sqrt(2.0 * ng)
    M = (rng.standard_normal((nb, nsig, ng)) + 1j * rng.standard_normal((nb, nsig, ng))) * scale
    En = np.concatenate([rng.uniform(-10.0, -1.0, nocc), rng.uniform(1.0, 30.0, nb - nocc)])
    g = gchi.astype(np.float64) + np.asarray(q, np.float64)
    g2 = np.einsum("ij,ij->i", g, g)
    d2 = g2[:, None] + g2[None, :] - 2.0 * (g @ g.T)
    t = rng.uniform(0.0, 2.0 * math.pi, ng)
    omega2 = (wp * wp) * np.exp(-d2 / 8.0) * np.exp(1j * (t[:, None] - t[None, :]))
    u = rng.uniform(0.0, 1.0, ng)
    wtilde = wp * (1.0 + 0.5 * (u[:, None] + u[None, :])) - 1j * eta
    E = np.linspace(ewin[0], ewin[1], ne) if ne > 1 else np.full(ne, 0.5 * (ewin[0] + ewin[1]))
    return GppProblem(np.ascontiguousarray(M), En, int(nocc), np.ascontiguousarray(omega2),
                      np.ascontiguousarray(wtilde), coulomb(gchi, q), E, gchi)
