// Full-matrix (off-diagonal) plasmon-pole self-energy on an energy grid, the Sigma-module kernel
// of the section on the off-diagonal GPP kernel:
//     Sigma_lm(E) = sum_n sum_GG' conj(M_n[l][G]) P^n_GG'(E) M_n[m][G'],
// with the prep. step forming P^n(E) per (n, E) and the two products the paper counts in Eq.
// flop_count_fullmat, X = conj(M_n) P (N_Sigma x N_G x N_G) and Sigma += X M_n^T
// (N_Sigma x N_G x N_Sigma).
//
// Split precision (the handle's split mode) runs the transposed products, so that the large
// operand P enters as a row-split A operand (one slice row per complex row, half the bytes of
// the column-split layout): X_E^T = P^T conj(M_n)^T, then Sigma^T += M_n X^T.  conj(M_n)^T is split
// by columns and M_n by rows once per band n; for a batch of energies the prep. kernel writes
// the row slices of every P^n(E)^T straight from the pole parameters (two-float arithmetic on
// the FP32 pipes), one persistent tensor-core launch forms every X_E^T of the batch side by side,
// X^T is split by columns and one more launch adds M_n X^T into Sigma^T for the whole batch;
// Sigma is transposed back once at the end.  FP64 mode stores P and runs both products on
// DMMA.
#include "api_internal.h"

using namespace gwapi;

namespace {

enum { kA, kW, kP, kX, kZA, kZB, kZP, kZX, kE, kNBuf };
static_assert(kNBuf == sizeof(((gw_chi0 *)nullptr)->gpp) / sizeof(gw_chi0::Buf), "buffer table");

gw_status gbuf(gw_chi0 *h, int i, size_t bytes, const char *what)
{
    return grow(h, &h->gpp[i].p, &h->gpp[i].cap, std::max<size_t>(bytes, 256), what);
}

// Energies per batch.  X^T (and its slices) for up to 16 energies, so that the second product
// runs on 16 N_Sigma columns at once; P^T slices (28 ng^2 bytes each at s = 7) for as many of
// them as 32 GiB (a quarter of the handle's memory budget, when one is set) holds: one prep.
// launch and one first-product launch per batch, so the pole parameters are read once per
// batch and the product's tiles fill the last wave.
constexpr int kGppBatch = 16;
static_assert(kGppBatch <= gw::kGppMaxE, "one prep. launch per energy batch");

int x_batch(int ne) { return std::max(1, std::min(kGppBatch, ne)); }

int p_batch(const gw_chi0 *h, int ebx, int ng, int s, int64_t kpad)
{
    const double per = (double)s * ng * kpad * 2;
    const double budget = h->d.mem_budget_bytes ? 0.25 * (double)h->d.mem_budget_bytes : 32.0 * 1073741824.0;
    const int eb = (int)std::min<double>(ebx, std::floor(budget / per));
    return std::max(1, eb);
}

gw_status gen_job(gw_chi0 *h, gw::OzJob &j, void *ZA, int rows_a, void *ZB, int nout, int64_t kpad, const int *EA,
                  const int *EB, double2 *out, int64_t ldo, int bn)
{
    std::memset(&j, 0, sizeof j);
    const int s = h->d.nslices;
    gw_status st;
    if ((st = make_tmap_z(h, &j.tmA, ZA, kpad, rows_a, s, gw::oz_box_rows_a())) ||
        (st = make_tmap_z(h, &j.tmB, ZB, kpad, 2 * nout, s, bn)))
        return st;
    j.E = EA;
    j.E2 = EB;
    j.out = (double *)out;
    j.ldo = 2 * ldo;
    j.rows_a = rows_a;
    j.rows_b = 2 * nout;
    j.nk = (int)(kpad / gw::oz_box_k());
    j.s = s;
    j.ntiles = ((rows_a + gw::oz_box_rows_a() - 1) / gw::oz_box_rows_a()) * ((2 * nout + bn - 1) / bn);
    return GW_OK;
}

gw_status run_gen_jobs(gw_chi0 *h, std::vector<gw::OzJob> &jobs, int bn, const char *name)
{
    int items = 0;
    for (auto &j : jobs) {
        j.item_start = items;
        items += j.ntiles;
    }
    const void *dj;
    gw_status st = upload_jobs(h, jobs.data(), sizeof(gw::OzJob) * jobs.size(), &dj);
    if (st) return st;
    Scope sc(h, name);
    CK(h, gw::launch_oz_gemm_general(bn, (const gw::OzJob *)dj, (int)jobs.size(), items, std::min(items, num_sms()),
                                     h->status, h->st),
       name);
    return GW_OK;
}

// One first-product launch: energies [p0, p0 + cp) of the energy batch starting at e0, band n.
struct PItem {
    int n, e0, cx, p0, cp;
};

gw_status sigma_split(gw_chi0 *h, int nb, int nocc, int nsig, int ng, const double2 *M, const double *En,
                      const double2 *omega2, const double2 *wtilde, const double *vcoul, int ne, const double *E,
                      double2 *sigma)
{
    const int s = h->d.nslices;
    const int64_t kpad = oz_kpad(ng);
    const int ebx = x_batch(ne), ebp = p_batch(h, ebx, ng, s, kpad);
    const size_t nn = (size_t)ng * ng;
    const size_t zp1 = (size_t)s * ng * kpad;       // bf16 per P^T
    const int64_t ldx = (int64_t)ebx * nsig;        // X^T row length (complex)
    gw_status st;
    if ((st = gbuf(h, kA, sizeof(float4) * nn, "pole residues")) ||
        (st = gbuf(h, kW, sizeof(float4) * nn, "mode energies")) ||
        (st = gbuf(h, kX, sizeof(double2) * (size_t)ng * ldx, "X^T")) ||
        (st = gbuf(h, kP, sizeof(double2) * (size_t)nsig * ne * nsig, "Sigma^T")) ||
        (st = gbuf(h, kZA, 2 * (size_t)s * nsig * kpad, "M_n slices")) ||
        (st = gbuf(h, kZB, 2 * (size_t)s * 2 * nsig * kpad, "conj(M_n)^T slices")) ||
        (st = gbuf(h, kZP, 2 * zp1 * ebp, "P^T slices")) ||
        (st = gbuf(h, kZX, 2 * (size_t)s * 2 * ldx * kpad, "X^T slices")) ||
        (st = gbuf(h, kE, sizeof(int) * ((size_t)2 * nsig + (size_t)ebp * ng + (size_t)ldx), "exponents")))
        return st;
    float4 *At = (float4 *)h->gpp[kA].p, *Wt = (float4 *)h->gpp[kW].p;
    double2 *XT = (double2 *)h->gpp[kX].p, *ST = (double2 *)h->gpp[kP].p;
    char *ZA = (char *)h->gpp[kZA].p, *ZB = (char *)h->gpp[kZB].p, *ZP = (char *)h->gpp[kZP].p,
         *ZX = (char *)h->gpp[kZX].p;
    int *EA = (int *)h->gpp[kE].p, *EB = EA + nsig, *EP = EB + nsig, *EX = EP + (size_t)ebp * ng;
    {
        Scope sc(h, "gpp_setup");
        CK(h, gw::launch_gpp_setup_tf(omega2, wtilde, vcoul, ng, At, Wt, h->st), "pole setup");
    }
    CK(h, cudaMemsetAsync(ST, 0, sizeof(double2) * (size_t)nsig * ne * nsig, h->st), "zero Sigma^T");
    std::vector<PItem> items;
    for (int n = 0; n < nb; ++n)
        for (int e0 = 0; e0 < ne; e0 += ebx) {
            const int cx = std::min(ebx, ne - e0);
            for (int p0 = 0; p0 < cx; p0 += ebp) items.push_back({n, e0, cx, p0, std::min(ebp, cx - p0)});
        }
    const int bn1 = 2 * nsig >= 256 ? 256 : 128;
    std::vector<gw::OzJob> jobs;
    for (const PItem &it : items) {
        if (it.e0 == 0 && it.p0 == 0) {
            const double2 *Mn = M + (size_t)it.n * nsig * ng;
            Scope sc(h, "oz_split_m");
            CK(h, gw::launch_oz_split_rows(Mn, nsig, ng, s, kpad, ZA, EA, h->st), "M_n slices");
            CK(h, gw::launch_oz_split_cols(Mn, ng, nsig, 1, ng, true, s, kpad, ZB, EB, h->st), "conj(M_n)^T slices");
        }
        if (it.p0 == 0) CK(h, cudaMemsetAsync(XT, 0, sizeof(double2) * (size_t)ng * ldx, h->st), "zero X^T");
        {
            double d[gw::kGppMaxE];
            for (int j = 0; j < it.cp; ++j) d[j] = E[it.e0 + it.p0 + j] - En[it.n];
            Scope sc(h, "gpp_prep_split");
            CK(h, gw::launch_gpp_prep_split(At, Wt, ng, d, it.cp, it.n < nocc ? -1.0f : 1.0f, s, kpad, (int64_t)zp1,
                                            ZP, EP, h->st),
               "prep. step");
        }
        // X^T[c][(e, l)] = sum_g P[g][c] conj(M_n[l][g])
        jobs.assign(it.cp, gw::OzJob{});
        for (int j = 0; j < it.cp; ++j)
            if ((st = gen_job(h, jobs[j], ZP + 2 * zp1 * j, ng, ZB, nsig, kpad, EP + (size_t)j * ng, EB,
                              XT + (size_t)(it.p0 + j) * nsig, ldx, bn1)))
                return st;
        if ((st = run_gen_jobs(h, jobs, bn1, "gpp_gemm_x"))) return st;
        if (it.p0 + it.cp == it.cx) {
            {
                Scope sc(h, "oz_split_x");
                CK(h, gw::launch_oz_split_cols(XT, ng, it.cx * nsig, ldx, 1, false, s, kpad, ZX, EX, h->st),
                   "X^T slices");
            }
            // Sigma^T[m][(e, l)] += sum_c M_n[m][c] X^T[c][(e, l)]
            const int bn2 = 2 * it.cx * nsig >= 256 ? 256 : 128;
            jobs.assign(1, gw::OzJob{});
            if ((st = gen_job(h, jobs[0], ZA, nsig, ZX, it.cx * nsig, kpad, EA, EX, ST + (size_t)it.e0 * nsig,
                              (int64_t)ne * nsig, bn2)))
                return st;
            if ((st = run_gen_jobs(h, jobs, bn2, "gpp_gemm_sigma"))) return st;
        }
    }
    Scope sc(h, "gpp_untranspose");
    CK(h, gw::launch_gpp_untranspose(ST, ne, nsig, sigma, h->st), "Sigma");
    return GW_OK;
}

gw_status sigma_f64(gw_chi0 *h, int nb, int nocc, int nsig, int ng, const double2 *M, const double *En,
                    const double2 *omega2, const double2 *wtilde, const double *vcoul, int ne, const double *E,
                    double2 *sigma)
{
    const size_t nn = (size_t)ng * ng;
    gw_status st;
    if ((st = gbuf(h, kA, sizeof(double2) * nn, "pole residues")) ||
        (st = gbuf(h, kP, sizeof(double2) * nn, "P")) ||
        (st = gbuf(h, kX, sizeof(double2) * (size_t)nsig * ng, "X = conj(M) P")))
        return st;
    double2 *A = (double2 *)h->gpp[kA].p, *P = (double2 *)h->gpp[kP].p, *X = (double2 *)h->gpp[kX].p;
    {
        Scope sc(h, "gpp_setup");
        CK(h, gw::launch_gpp_setup(omega2, wtilde, vcoul, ng, A, h->st), "pole setup");
    }
    for (int n = 0; n < nb; ++n) {
        const double2 *Mn = M + (size_t)n * nsig * ng;
        const double sgn = n < nocc ? -1.0 : 1.0;
        for (int e = 0; e < ne; ++e) {
            {
                Scope sc(h, "gpp_prep_f64");
                CK(h, gw::launch_gpp_prep_f64(A, wtilde, ng, E[e] - En[n], sgn, P, h->st), "prep. step");
            }
            Scope sc(h, "gpp_zgemm");
            CK(h, gw::launch_zgemm_ex(Mn, P, X, nsig, ng, ng, true, false, false, h->st), "X = conj(M_n) P");
            CK(h, gw::launch_zgemm_ex(X, Mn, sigma + (size_t)e * nsig * nsig, nsig, ng, nsig, false, true, true, h->st),
               "Sigma += X M_n^T");
        }
    }
    return GW_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

} // namespace

gw_status gw_chi0_sigma_gpp(gw_chi0 *h, int nb, int nocc, int nsig, int ng, const double *M, const double *En,
                            const double *omega2, const double *wtilde, const double *vcoul, int ne, const double *E,
                            double *sigma)
{
    if (!h) return GW_ERR_ARG;
    if (nb < 0 || nocc < 0 || nocc > nb || nsig < 1 || ng < 1 || ne < 0)
        return fail(h, GW_ERR_ARG, "bad sizes (nb %d, nocc %d, nsig %d, ng %d, ne %d)", nb, nocc, nsig, ng, ne);
    if (ne == 0) return GW_OK;
    if (!sigma || !E || (nb > 0 && (!M || !En || !omega2 || !wtilde || !vcoul)))
        return fail(h, GW_ERR_ARG, "null pointer");
    if (!aligned16(sigma) || (nb > 0 && (!aligned16(M) || !aligned16(omega2) || !aligned16(wtilde))))
        return fail(h, GW_ERR_ARG, "complex arrays must be 16-byte aligned");
    if ((int64_t)ng * 2 > (int64_t)1 << 30 || (int64_t)nsig * ne > (int64_t)1 << 30 || ne > 65535)
        return fail(h, GW_ERR_ARG, "sizes out of range");
    for (int e = 0; e < ne; ++e)
        if (!std::isfinite(E[e])) return fail(h, GW_ERR_ARG, "E[%d] not finite", e);
    for (int n = 0; n < nb; ++n)
        if (!std::isfinite(En[n])) return fail(h, GW_ERR_ARG, "En[%d] not finite", n);
    CK(h, cudaMemsetAsync(sigma, 0, sizeof(double2) * (size_t)ne * nsig * nsig, h->st), "zero Sigma");
    if (nb == 0) return GW_OK;
    if (h->d.prec == GW_PREC_OZAKI_BF16)
        return sigma_split(h, nb, nocc, nsig, ng, (const double2 *)M, En, (const double2 *)omega2,
                           (const double2 *)wtilde, vcoul, ne, E, (double2 *)sigma);
    return sigma_f64(h, nb, nocc, nsig, ng, (const double2 *)M, En, (const double2 *)omega2, (const double2 *)wtilde,
                     vcoul, ne, E, (double2 *)sigma);
}
