/*
 * gw_oracle.c -- plain, slow FP64 CPU oracle for the chi0 path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * What it computes (SC'25 BerkeleyGW paper, "Overview of the Problem"):
 *   - plane-wave matrix elements  M_mn^G = \int psi_m^*(r) e^{iG.r} psi_n(r) dr
 *     (definition given inline after Eq. ff-ch), with psi_n(r) = sum_K c_n(K) e^{iK.r}
 *     and the integral normalised by the cell volume;
 *   - the polarizability of Eq. chi_mat,
 *     chi_GG'(w) = sum_vc conj(M_vc^G) Delta_vc(w) M_vc^G',
 *     with Delta_vc(iw) = 2/(x - iw) + 2/(x + iw), x = E_v - E_c (the paper leaves
 *     Delta open; this is the form the hot path is specified with, imaginary w);
 *   - the adjoint of L = Re Tr(W chi) with respect to the energies and the
 *     plane-wave coefficients (motivated by the GWPT derivative, Eq. gwpt).
 *
 * Two independent routes to M are provided:
 *   oracle_m_conv : G-space convolution  M_vc(G) = sum_K conj(c_v(K)) c_c(K - G)
 *   oracle_m_dft  : psi on the real-space grid by a direct (triple) sum, the
 *                   pair product, then M(G) = (1/N_r) sum_r rho(r) e^{+iG.r} by a
 *                   direct sum (tiny grids only).
 * Sums over pairs use Neumaier compensation so the oracle's own rounding stays
 * far below the 1e-11 parity bar.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846264338327950288

/* ---------------------------------------------------------------- helpers */

typedef struct {
    int lo[3], ext[3];
    int32_t *idx; /* -1 where no G of the list sits */
} gbox;

static int gbox_build(gbox *b, int n, const int32_t *g)
{
    int hi[3];
    for (int a = 0; a < 3; ++a) { b->lo[a] = 0; hi[a] = 0; }
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            if (i == 0 || g[3 * i + a] < b->lo[a]) b->lo[a] = g[3 * i + a];
            if (i == 0 || g[3 * i + a] > hi[a]) hi[a] = g[3 * i + a];
        }
    size_t tot = 1;
    for (int a = 0; a < 3; ++a) { b->ext[a] = hi[a] - b->lo[a] + 1; tot *= (size_t)b->ext[a]; }
    b->idx = (int32_t *)malloc(tot * sizeof(int32_t));
    if (!b->idx) return -1;
    for (size_t t = 0; t < tot; ++t) b->idx[t] = -1;
    for (int i = 0; i < n; ++i) {
        size_t o = ((size_t)(g[3 * i] - b->lo[0]) * b->ext[1] + (g[3 * i + 1] - b->lo[1])) * b->ext[2] +
                   (g[3 * i + 2] - b->lo[2]);
        b->idx[o] = i;
    }
    return 0;
}

static int gbox_find(const gbox *b, int g0, int g1, int g2)
{
    int d0 = g0 - b->lo[0], d1 = g1 - b->lo[1], d2 = g2 - b->lo[2];
    if (d0 < 0 || d1 < 0 || d2 < 0 || d0 >= b->ext[0] || d1 >= b->ext[1] || d2 >= b->ext[2]) return -1;
    return b->idx[((size_t)d0 * b->ext[1] + d1) * b->ext[2] + d2];
}

/* Neumaier-compensated accumulator */
typedef struct { double s, c; } nsum;
static inline void nadd(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static inline double nval(const nsum *a) { return a->s + a->c; }

/* e^{2 pi i (k r mod n)/n}: the integer product is reduced before the angle is formed */
static inline void phase(long long kr, int n, double *re, double *im)
{
    long long m = kr % n;
    if (m < 0) m += n;
    double ang = 2.0 * PI * (double)m / (double)n;
    *re = cos(ang);
    *im = sin(ang);
}

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------ M, G-space convolution */
/*
 * M_vc(G) = sum_{K in sphere_v} conj(c_v(K)) c_c(K - G); c_c = 0 outside its sphere.
 * Complex arrays are interleaved (re, im) doubles.
 *   cv [nv][ngv], cc [nc][ngc], M [nv*nc][ng], pair index p = v*nc + c.
 * Returns 0, or -1 when memory runs out.
 */
int oracle_m_conv(int nv, int ngv, const int32_t *gv, const double *cv,
                  int nc, int ngc, const int32_t *gc, const double *cc,
                  int ng, const int32_t *gchi, double *M)
{
    gbox bc;
    if (gbox_build(&bc, ngc, gc)) return -1;
    int err = 0;
#pragma omp parallel
    {
        int *kk = (int *)malloc(sizeof(int) * (size_t)ngv);
        int *jj = (int *)malloc(sizeof(int) * (size_t)ngv);
        if (!kk || !jj) {
#pragma omp atomic write
            err = -1;
        } else {
#pragma omp for schedule(dynamic)
            for (int g = 0; g < ng; ++g) {
                /* pairs (K, K-G) that both lie in their spheres */
                int nk = 0;
                for (int k = 0; k < ngv; ++k) {
                    int j = gbox_find(&bc, gv[3 * k] - gchi[3 * g], gv[3 * k + 1] - gchi[3 * g + 1],
                                      gv[3 * k + 2] - gchi[3 * g + 2]);
                    if (j >= 0) { kk[nk] = k; jj[nk] = j; ++nk; }
                }
                for (int v = 0; v < nv; ++v)
                    for (int c = 0; c < nc; ++c) {
                        const double *a = cv + 2 * (size_t)v * ngv;
                        const double *b = cc + 2 * (size_t)c * ngc;
                        nsum sr = {0, 0}, si = {0, 0};
                        for (int t = 0; t < nk; ++t) {
                            double ar = a[2 * kk[t]], ai = a[2 * kk[t] + 1];
                            double br = b[2 * jj[t]], bi = b[2 * jj[t] + 1];
                            /* conj(a) * b */
                            nadd(&sr, ar * br + ai * bi);
                            nadd(&si, ar * bi - ai * br);
                        }
                        size_t o = 2 * (((size_t)v * nc + c) * ng + g);
                        M[o] = nval(&sr);
                        M[o + 1] = nval(&si);
                    }
            }
        }
        free(kk);
        free(jj);
    }
    free(bc.idx);
    return err;
}

/* ------------------------------------------------ psi on the grid, direct sum */
/* psi_n(r) = sum_K c_n(K) e^{+2 pi i (K0 r0/n0 + K1 r1/n1 + K2 r2/n2)};  psi [nb][n0][n1][n2] */
void oracle_psi_dft(int n0, int n1, int n2, int nb, int ngk, const int32_t *gk, const double *coef, double *psi)
{
    long long nr = (long long)n0 * n1 * n2;
#pragma omp parallel for schedule(static)
    for (long long r = 0; r < nr; ++r) {
        int r0 = (int)(r / ((long long)n1 * n2)), r1 = (int)((r / n2) % n1), r2 = (int)(r % n2);
        for (int b = 0; b < nb; ++b) {
            nsum sr = {0, 0}, si = {0, 0};
            for (int k = 0; k < ngk; ++k) {
                double p0r, p0i, p1r, p1i, p2r, p2i;
                phase((long long)gk[3 * k] * r0, n0, &p0r, &p0i);
                phase((long long)gk[3 * k + 1] * r1, n1, &p1r, &p1i);
                phase((long long)gk[3 * k + 2] * r2, n2, &p2r, &p2i);
                double tr = p0r * p1r - p0i * p1i, ti = p0r * p1i + p0i * p1r;
                double er = tr * p2r - ti * p2i, ei = tr * p2i + ti * p2r;
                double cr = coef[2 * ((size_t)b * ngk + k)], ci = coef[2 * ((size_t)b * ngk + k) + 1];
                nadd(&sr, cr * er - ci * ei);
                nadd(&si, cr * ei + ci * er);
            }
            psi[2 * ((size_t)b * nr + r)] = nval(&sr);
            psi[2 * ((size_t)b * nr + r) + 1] = nval(&si);
        }
    }
}

/* ------------------------------------------------ M, real-space route */
/*
 * rho_vc(r) = conj(psi_v(r)) psi_c(r);  M_vc(G) = (1/N_r) sum_r rho_vc(r) e^{+iG.r}.
 * psi_v [nv][N_r], psi_c [nc][N_r] as produced by oracle_psi_dft.
 */
void oracle_m_from_psi(int n0, int n1, int n2, int nv, const double *psiv, int nc, const double *psic,
                       int ng, const int32_t *gchi, double *M)
{
    long long nr = (long long)n0 * n1 * n2;
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int v = 0; v < nv; ++v)
        for (int c = 0; c < nc; ++c)
            for (int g = 0; g < ng; ++g) {
                nsum sr = {0, 0}, si = {0, 0};
                for (long long r = 0; r < nr; ++r) {
                    int r0 = (int)(r / ((long long)n1 * n2)), r1 = (int)((r / n2) % n1), r2 = (int)(r % n2);
                    double ar = psiv[2 * ((size_t)v * nr + r)], ai = psiv[2 * ((size_t)v * nr + r) + 1];
                    double br = psic[2 * ((size_t)c * nr + r)], bi = psic[2 * ((size_t)c * nr + r) + 1];
                    double rr = ar * br + ai * bi, ri = ar * bi - ai * br; /* conj(psi_v) psi_c */
                    double p0r, p0i, p1r, p1i, p2r, p2i;
                    phase((long long)gchi[3 * g] * r0, n0, &p0r, &p0i);
                    phase((long long)gchi[3 * g + 1] * r1, n1, &p1r, &p1i);
                    phase((long long)gchi[3 * g + 2] * r2, n2, &p2r, &p2i);
                    double tr = p0r * p1r - p0i * p1i, ti = p0r * p1i + p0i * p1r;
                    double er = tr * p2r - ti * p2i, ei = tr * p2i + ti * p2r;
                    nadd(&sr, rr * er - ri * ei);
                    nadd(&si, rr * ei + ri * er);
                }
                size_t o = 2 * (((size_t)v * nc + c) * ng + g);
                M[o] = nval(&sr) / (double)nr;
                M[o + 1] = nval(&si) / (double)nr;
            }
}

/* ------------------------------------------------ energy factor */
/*
 * Delta_vc(iw) = 2/(x - iw) + 2/(x + iw), x = E_v - E_c, evaluated in complex
 * arithmetic exactly as written; the imaginary parts cancel and only the real
 * part is returned (the largest |Im| seen goes to *imag_resid).
 */
void oracle_delta(int nv, const double *ev, int nc, const double *ec, double omega, double *delta,
                  double *imag_resid)
{
    double worst = 0.0;
    for (int v = 0; v < nv; ++v)
        for (int c = 0; c < nc; ++c) {
            double x = ev[v] - ec[c];
            /* 2/(x - i w) = 2 (x + i w)/(x^2 + w^2) */
            double d1 = x * x + omega * omega;
            double ar = 2.0 * x / d1, ai = 2.0 * omega / d1;
            /* 2/(x + i w) = 2 (x - i w)/(x^2 + w^2) */
            double br = 2.0 * x / d1, bi = -2.0 * omega / d1;
            delta[(size_t)v * nc + c] = ar + br;
            if (fabs(ai + bi) > worst) worst = fabs(ai + bi);
        }
    if (imag_resid) *imag_resid = worst;
}

/* d Delta / dx of the same form: -2/(x - iw)^2 - 2/(x + iw)^2 (real part) */
static double delta_dx(double x, double w)
{
    /* 1/(x - iw)^2 = (x + iw)^2 / (x^2 + w^2)^2 */
    double d = (x * x + w * w) * (x * x + w * w);
    double re1 = (x * x - w * w) / d;  /* Re (x+iw)^2 / d */
    double re2 = (x * x - w * w) / d;  /* Re (x-iw)^2 / d */
    return -2.0 * re1 - 2.0 * re2;
}

/* ------------------------------------------------ chi0 (Eq. chi_mat) */
/*
 * chi[G][G'] = sum_p conj(M[p][G]) delta[p] M[p][G'];  M [P][ng], chi [ng][ng].
 * Every entry (both triangles) is summed on its own, compensated over p.
 */
void oracle_chi0(long long P, int ng, const double *M, const double *delta, double *chi)
{
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int g = 0; g < ng; ++g)
        for (int h = 0; h < ng; ++h) {
            nsum sr = {0, 0}, si = {0, 0};
            for (long long p = 0; p < P; ++p) {
                double ar = M[2 * ((size_t)p * ng + g)], ai = M[2 * ((size_t)p * ng + g) + 1];
                double br = M[2 * ((size_t)p * ng + h)], bi = M[2 * ((size_t)p * ng + h) + 1];
                double d = delta[p];
                nadd(&sr, d * (ar * br + ai * bi));
                nadd(&si, d * (ar * bi - ai * br));
            }
            chi[2 * ((size_t)g * ng + h)] = nval(&sr);
            chi[2 * ((size_t)g * ng + h) + 1] = nval(&si);
        }
}

/* ------------------------------------------------ adjoint of L = Re Tr(W chi) */
/*
 * W [ng][ng] Hermitian.  With m_p = M[p][:] (a row), L = sum_p Delta_p q_p,
 * q_p = sum_{G,G'} m_p(G) W[G][G'] conj(m_p(G')) (real for Hermitian W).
 * Wirtinger: g_p(G') = dL/dconj(m_p(G')) = Delta_p (m_p W)(G').
 *   dL/dconj(c_c(J)) = sum_{v,G} g_vc(G) c_v(J + G)
 *   dL/dconj(c_v(J)) = sum_{c,G} conj(g_vc(G)) c_c(J - G)
 * Outputs follow the convention grad = dL/dRe + i dL/dIm = 2 dL/dconj.
 *   dL/dE_v = sum_c q_vc dDelta/dx,  dL/dE_c = -sum_v q_vc dDelta/dx,  x = E_v - E_c.
 * Returns 0 or -1 (out of memory).
 */
int oracle_adjoint(int nv, int ngv, const int32_t *gv, const double *cv, const double *ev,
                   int nc, int ngc, const int32_t *gc, const double *cc, const double *ec,
                   int ng, const int32_t *gchi, const double *W, double omega,
                   double *L_out, double *dEv, double *dEc, double *dcv, double *dcc)
{
    long long P = (long long)nv * nc;
    double *M = (double *)malloc(sizeof(double) * 2 * (size_t)P * ng);
    double *Y = (double *)malloc(sizeof(double) * 2 * (size_t)P * ng);
    double *q = (double *)malloc(sizeof(double) * (size_t)P);
    double *dl = (double *)malloc(sizeof(double) * (size_t)P);
    gbox bv, bc;
    bv.idx = NULL;
    bc.idx = NULL;
    int err = 0;
    if (!M || !Y || !q || !dl) { err = -1; goto done; }
    if (oracle_m_conv(nv, ngv, gv, cv, nc, ngc, gc, cc, ng, gchi, M)) { err = -1; goto done; }
    oracle_delta(nv, ev, nc, ec, omega, dl, NULL);

    /* Y = M W and q_p = Re sum_G Y_p(G) conj(m_p(G)) */
#pragma omp parallel for schedule(dynamic)
    for (long long p = 0; p < P; ++p) {
        for (int h = 0; h < ng; ++h) {
            nsum sr = {0, 0}, si = {0, 0};
            for (int g = 0; g < ng; ++g) {
                double mr = M[2 * ((size_t)p * ng + g)], mi = M[2 * ((size_t)p * ng + g) + 1];
                double wr = W[2 * ((size_t)g * ng + h)], wi = W[2 * ((size_t)g * ng + h) + 1];
                nadd(&sr, mr * wr - mi * wi);
                nadd(&si, mr * wi + mi * wr);
            }
            Y[2 * ((size_t)p * ng + h)] = nval(&sr);
            Y[2 * ((size_t)p * ng + h) + 1] = nval(&si);
        }
        nsum qs = {0, 0};
        for (int h = 0; h < ng; ++h) {
            double yr = Y[2 * ((size_t)p * ng + h)], yi = Y[2 * ((size_t)p * ng + h) + 1];
            double mr = M[2 * ((size_t)p * ng + h)], mi = M[2 * ((size_t)p * ng + h) + 1];
            nadd(&qs, yr * mr + yi * mi);
        }
        q[p] = nval(&qs);
    }
    {
        nsum ls = {0, 0};
        for (long long p = 0; p < P; ++p) nadd(&ls, dl[p] * q[p]);
        if (L_out) *L_out = nval(&ls);
    }
    for (int v = 0; v < nv; ++v) {
        nsum s = {0, 0};
        for (int c = 0; c < nc; ++c) nadd(&s, q[(size_t)v * nc + c] * delta_dx(ev[v] - ec[c], omega));
        dEv[v] = nval(&s);
    }
    for (int c = 0; c < nc; ++c) {
        nsum s = {0, 0};
        for (int v = 0; v < nv; ++v) nadd(&s, q[(size_t)v * nc + c] * delta_dx(ev[v] - ec[c], omega));
        dEc[c] = -nval(&s);
    }
    if (gbox_build(&bv, ngv, gv) || gbox_build(&bc, ngc, gc)) { err = -1; goto done; }

    /* conduction: 2 sum_{v,G} g_vc(G) c_v(J + G) */
#pragma omp parallel for schedule(dynamic)
    for (int c = 0; c < nc; ++c)
        for (int j = 0; j < ngc; ++j) {
            nsum sr = {0, 0}, si = {0, 0};
            for (int g = 0; g < ng; ++g) {
                int k = gbox_find(&bv, gc[3 * j] + gchi[3 * g], gc[3 * j + 1] + gchi[3 * g + 1],
                                  gc[3 * j + 2] + gchi[3 * g + 2]);
                if (k < 0) continue;
                for (int v = 0; v < nv; ++v) {
                    size_t p = (size_t)v * nc + c;
                    double gr = dl[p] * Y[2 * (p * ng + g)], gi = dl[p] * Y[2 * (p * ng + g) + 1];
                    double ar = cv[2 * ((size_t)v * ngv + k)], ai = cv[2 * ((size_t)v * ngv + k) + 1];
                    nadd(&sr, gr * ar - gi * ai);
                    nadd(&si, gr * ai + gi * ar);
                }
            }
            dcc[2 * ((size_t)c * ngc + j)] = 2.0 * nval(&sr);
            dcc[2 * ((size_t)c * ngc + j) + 1] = 2.0 * nval(&si);
        }
    /* valence: 2 sum_{c,G} conj(g_vc(G)) c_c(J - G) */
#pragma omp parallel for schedule(dynamic)
    for (int v = 0; v < nv; ++v)
        for (int j = 0; j < ngv; ++j) {
            nsum sr = {0, 0}, si = {0, 0};
            for (int g = 0; g < ng; ++g) {
                int k = gbox_find(&bc, gv[3 * j] - gchi[3 * g], gv[3 * j + 1] - gchi[3 * g + 1],
                                  gv[3 * j + 2] - gchi[3 * g + 2]);
                if (k < 0) continue;
                for (int c = 0; c < nc; ++c) {
                    size_t p = (size_t)v * nc + c;
                    double gr = dl[p] * Y[2 * (p * ng + g)], gi = -dl[p] * Y[2 * (p * ng + g) + 1];
                    double br = cc[2 * ((size_t)c * ngc + k)], bi = cc[2 * ((size_t)c * ngc + k) + 1];
                    nadd(&sr, gr * br - gi * bi);
                    nadd(&si, gr * bi + gi * br);
                }
            }
            dcv[2 * ((size_t)v * ngv + j)] = 2.0 * nval(&sr);
            dcv[2 * ((size_t)v * ngv + j) + 1] = 2.0 * nval(&si);
        }
done:
    free(M); free(Y); free(q); free(dl); free(bv.idx); free(bc.idx);
    return err;
}
