// Entry points beyond chi0 itself: the adjoint of L = Re Tr(W chi0), the static subspace,
// the inverse dielectric matrix, chi0 on the real axis and the forward derivative.
#include "api_internal.h"

using namespace gwapi;

gw_status gw_chi0_adjoint(gw_chi0 *h, int iq, double omega, const double *W, double *L, double *dE_v, double *dE_c,
                          double *dcoeff_v, double *dcoeff_c)
{
    if (!h) return GW_ERR_ARG;
    gw_status s = check_slot(h, iq);
    if (s) return s;
    if (!W || !dE_v || !dE_c || !dcoeff_v || !dcoeff_c) return fail(h, GW_ERR_ARG, "null pointer");
    if (!(omega >= 0.0) || !std::isfinite(omega)) return fail(h, GW_ERR_ARG, "omega must be finite and >= 0");
    const BandSet &v = h->val[iq];
    const BandSet &c = h->cond;
    const Sphere &sp = h->sph[iq];
    const int nv = v.nb, nc = c.nb, ng = sp.ng;
    const int64_t nr = h->nr;
    const bool tf = h->d.mtxel_prec == GW_MTXEL_TWOFLOAT;
    // valence bands per chunk: bounded by the pair chunk and by 2 GiB of back-projected grids
    int64_t vch = std::max<int64_t>(1, h->d.pair_chunk / nc);
    vch = std::min<int64_t>(vch, std::max<int64_t>(1, (int64_t(2) << 30) / ((int64_t)nc * nr * 16)));
    vch = std::min<int64_t>(vch, nv);
    const int64_t cmax = vch * nc;
    // work buffers, held only for this call
    double2 *Mb = nullptr, *Yb = nullptr, *Hb = nullptr, *pbv = nullptr, *pbc = nullptr, *Wh = nullptr;
    double *Lacc = nullptr;
    int *cs = nullptr, *cg = nullptr;
    const int ncell = (int)sp.cstart.size() - 1;
    size_t szM = sizeof(double2) * cmax * ng, szH = sizeof(double2) * cmax * nr;
    size_t szV = sizeof(double2) * (size_t)nv * nr, szC = sizeof(double2) * (size_t)nc * nr;
    const size_t szW = sizeof(double2) * (size_t)ng * ng;
    auto cleanup = [&]() {
        cudaStreamSynchronize(h->st);
        dfree(h, Wh, szW);
        dfree(h, Mb, szM);
        dfree(h, Yb, szM);
        dfree(h, Hb, szH);
        dfree(h, pbv, szV);
        dfree(h, pbc, szC);
        dfree(h, Lacc, sizeof(double));
        dfree(h, cs, sizeof(int) * (ncell + 1));
        dfree(h, cg, sizeof(int) * ng);
    };
#define ACK(x, what)                       \
    do {                                   \
        cudaError_t e_ = (x);              \
        if (e_ != cudaSuccess) {           \
            gw_status r_ = cuda_fail(h, e_, what); \
            cleanup();                     \
            return r_;                     \
        }                                  \
    } while (0)
    if ((s = dalloc(h, (void **)&Mb, szM, "adjoint M")) || (s = dalloc(h, (void **)&Yb, szM, "adjoint Y")) ||
        (s = dalloc(h, (void **)&Hb, szH, "adjoint grids")) || (s = dalloc(h, (void **)&pbv, szV, "valence adjoint")) ||
        (s = dalloc(h, (void **)&pbc, szC, "conduction adjoint")) ||
        (s = dalloc(h, (void **)&Lacc, sizeof(double), "L")) ||
        (s = dalloc(h, (void **)&cs, sizeof(int) * (ncell + 1), "cells")) ||
        (s = dalloc(h, (void **)&cg, sizeof(int) * ng, "cells")) ||
        (s = dalloc(h, (void **)&Wh, szW, "Hermitian part of W"))) {
        cleanup();
        return s;
    }
    // L sees W only through its Hermitian part (chi is Hermitian)
    ACK(gw::launch_herm_part((const double2 *)W, ng, Wh, h->st), "Hermitian part of W");
    ACK(cudaMemcpyAsync(cs, sp.cstart.data(), sizeof(int) * (ncell + 1), cudaMemcpyHostToDevice, h->st), "cells");
    ACK(cudaMemcpyAsync(cg, sp.cg.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, h->st), "cells");
    ACK(cudaMemsetAsync(Lacc, 0, sizeof(double), h->st), "zero");
    ACK(cudaMemsetAsync(dE_v, 0, sizeof(double) * nv, h->st), "zero");
    ACK(cudaMemsetAsync(dE_c, 0, sizeof(double) * nc, h->st), "zero");
    ACK(cudaMemsetAsync(pbv, 0, szV, h->st), "zero");
    ACK(cudaMemsetAsync(pbc, 0, szC, h->st), "zero");
    gw::PairPlan pp = pair_plan(h, sp);
    // split precision: Y = M W as a split product, W's slices once per call
    const bool split = h->d.prec == GW_PREC_OZAKI_BF16;
    if (split && (s = oz_prepare_b(h, Wh, ng, ng))) {
        cleanup();
        return s;
    }
    for (int v0 = 0; v0 < nv; v0 += (int)vch) {
        const int nvc = (int)std::min<int64_t>(vch, nv - v0);
        const int64_t p0 = (int64_t)v0 * nc, cnt = (int64_t)nvc * nc;
        {
            Scope sc(h, "pair_mtxel");
            ACK(run_pair(h, v.psi, c.psi, nc, p0, cnt, pp, Mb), "pair kernel");
        }
        {
            Scope sc(h, "adj_zgemm");
            if (split) {
                if ((s = oz_product(h, Mb, cnt, ng, ng, Yb))) {
                    cleanup();
                    return s;
                }
            } else {
                ACK(gw::launch_zgemm(Mb, Wh, Yb, cnt, ng, ng, h->st), "Y = M W");
            }
        }
        {
            Scope sc(h, "adj_rows");
            ACK(gw::launch_adj_rows(Mb, Yb, cnt, ng, nc, p0, v.energy, c.energy, omega, Lacc, dE_v, dE_c, h->st),
                "row reductions");
        }
        {
            Scope sc(h, "adj_pair");
            ACK(gw::launch_adj_pair(Yb, cnt, pp, cs, cg, ncell, Hb, tf, h->st), "back-projection");
        }
        {
            Scope sc(h, "adj_products");
            ACK(gw::launch_adj_products(v.psi, c.psi, v0, nvc, nc, Hb, nr, tf, pbv, pbc, h->st), "products");
        }
    }
    {
        Scope sc(h, "adj_band");
        if (tf) {
            ACK(gw::launch_tf_to_f64(pbv, (int64_t)nv * nr, h->st), "valence adjoint to FP64");
            ACK(gw::launch_tf_to_f64(pbc, (int64_t)nc * nr, h->st), "conduction adjoint to FP64");
        }
        ACK(gw::launch_band_adjoint(pbv, nv, h->d.n, h->ax, v.gofs, v.ngpsi, (double2 *)dcoeff_v, h->st),
            "valence band adjoint");
        ACK(gw::launch_band_adjoint(pbc, nc, h->d.n, h->ax, c.gofs, c.ngpsi, (double2 *)dcoeff_c, h->st),
            "conduction band adjoint");
    }
    if (L) ACK(cudaMemcpyAsync(L, Lacc, sizeof(double), cudaMemcpyDeviceToHost, h->st), "L");
#undef ACK
    cleanup(); // synchronises: L is valid on return
    return GW_OK;
}

// ------------------------------------------------------------------ static subspace
namespace {
gw_status load_solver(gw_chi0 *h)
{
    if (h->sol.hdl) return GW_OK;
    const char *names[] = {"libcusolver.so.12", "libcusolver.so.11", "libcusolver.so",
                           "/usr/local/cuda/lib64/libcusolver.so.12", "/usr/local/cuda/lib64/libcusolver.so"};
    for (const char *n : names)
        if ((h->sol.lib = dlopen(n, RTLD_NOW | RTLD_LOCAL))) break;
    if (!h->sol.lib) return fail(h, GW_ERR_UNSUPPORTED, "the dense eigensolver (libcusolver) was not found");
    h->sol.create = (decltype(h->sol.create))dlsym(h->sol.lib, "cusolverDnCreate");
    h->sol.destroy = (decltype(h->sol.destroy))dlsym(h->sol.lib, "cusolverDnDestroy");
    h->sol.set_stream = (decltype(h->sol.set_stream))dlsym(h->sol.lib, "cusolverDnSetStream");
    h->sol.buffer_size = (decltype(h->sol.buffer_size))dlsym(h->sol.lib, "cusolverDnZheevdx_bufferSize");
    h->sol.heevdx = (decltype(h->sol.heevdx))dlsym(h->sol.lib, "cusolverDnZheevdx");
    if (!h->sol.create || !h->sol.destroy || !h->sol.set_stream || !h->sol.buffer_size || !h->sol.heevdx)
        return fail(h, GW_ERR_UNSUPPORTED, "libcusolver lacks the Hermitian eigensolver entry points");
    if (h->sol.create(&h->sol.hdl) != CUSOLVER_STATUS_SUCCESS) {
        h->sol.hdl = nullptr;
        return fail(h, GW_ERR_CUDA, "cusolverDnCreate failed");
    }
    return GW_OK;
}
} // namespace

gw_status gw_chi0_subspace_basis(gw_chi0 *h, int ng, const double *chi0, int neig, double *basis, double *evals)
{
    if (!h) return GW_ERR_ARG;
    if (ng < 1 || neig < 1 || neig > ng) return fail(h, GW_ERR_ARG, "need 1 <= neig <= ng");
    if (!chi0 || !basis) return fail(h, GW_ERR_ARG, "null pointer");
    gw_status st = load_solver(h);
    if (st) return st;
    const size_t nn = (size_t)ng * ng;
    if ((st = grow(h, (void **)&h->eigA, &h->eigA_cap, sizeof(double2) * nn, "eigensolver matrix")) ||
        (st = grow(h, (void **)&h->eigW, &h->eigW_cap, sizeof(double) * (size_t)ng, "eigenvalues")) ||
        (st = grow(h, (void **)&h->eigInfo, &h->eigInfo_cap, sizeof(int), "eigensolver status")))
        return st;
    // The row-major Hermitian chi0 read column-major is its transpose, conj(chi0): the solver
    // returns the conjugated eigenvectors, which the transposing copy conjugates back.
    CK(h, cudaMemcpyAsync(h->eigA, chi0, sizeof(double2) * nn, cudaMemcpyDeviceToDevice, h->st), "copy chi0");
    if (h->sol.set_stream(h->sol.hdl, h->st) != CUSOLVER_STATUS_SUCCESS) return fail(h, GW_ERR_CUDA, "solver stream");
    int meig = 0, lwork = 0;
    if (h->sol.buffer_size(h->sol.hdl, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_LOWER, ng,
                           (const cuDoubleComplex *)h->eigA, ng, 0.0, 0.0, 1, neig, &meig, h->eigW,
                           &lwork) != CUSOLVER_STATUS_SUCCESS)
        return fail(h, GW_ERR_CUDA, "eigensolver workspace query failed");
    if ((st = grow(h, (void **)&h->eigWork, &h->eigWork_cap, sizeof(double2) * (size_t)std::max(lwork, 1),
                   "eigensolver workspace")))
        return st;
    {
        Scope sc(h, "subspace_eig");
        if (h->sol.heevdx(h->sol.hdl, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_LOWER, ng,
                          (cuDoubleComplex *)h->eigA, ng, 0.0, 0.0, 1, neig, &meig, h->eigW,
                          (cuDoubleComplex *)h->eigWork, lwork, h->eigInfo) != CUSOLVER_STATUS_SUCCESS)
            return fail(h, GW_ERR_CUDA, "eigensolver failed");
        CK(h, gw::launch_conj_transpose(h->eigA, ng, neig, (double2 *)basis, h->st), "basis");
    }
    if (evals)
        CK(h, cudaMemcpyAsync(evals, h->eigW, sizeof(double) * neig, cudaMemcpyDeviceToDevice, h->st), "eigenvalues");
    int info = 0;
    CK(h, cudaMemcpyAsync(&info, h->eigInfo, sizeof(int), cudaMemcpyDeviceToHost, h->st), "solver status");
    CK(h, cudaStreamSynchronize(h->st), "subspace basis sync");
    if (info != 0) return fail(h, GW_ERR_CUDA, "eigensolver reported %d", info);
    if (meig != neig) return fail(h, GW_ERR_CUDA, "eigensolver returned %d of %d vectors", meig, neig);
    return GW_OK;
}

gw_status gw_chi0_compute_subspace(gw_chi0 *h, int iq, int neig, const double *basis, int nw, const double *omega,
                                   double *chi_sub)
{
    if (!h) return GW_ERR_ARG;
    if (nw < 1 || nw > gw::kMaxOmega || !omega || !basis || !chi_sub)
        return fail(h, GW_ERR_ARG, "bad arguments (1 <= nw <= %d, non-null pointers)", gw::kMaxOmega);
    gw::OmegaList om;
    om.nw = nw;
    for (int i = 0; i < nw; ++i) {
        if (!(omega[i] >= 0.0) || !std::isfinite(omega[i])) return fail(h, GW_ERR_ARG, "omega must be finite and >= 0");
        om.w[i] = omega[i];
    }
    gw_status s = check_slot(h, iq);
    if (s) return s;
    const Sphere &sp = h->sph[iq];
    const BandSet &v = h->val[iq];
    const int ng = sp.ng;
    if (neig < 1 || neig > ng) return fail(h, GW_ERR_ARG, "need 1 <= neig <= ng");
    const int64_t P = (int64_t)v.nb * h->cond.nb;
    const int64_t chunk = std::min<int64_t>(h->d.pair_chunk, P);
    CK(h, cudaMemsetAsync(chi_sub, 0, sizeof(double2) * (size_t)nw * neig * neig, h->st), "zero chi");
    if ((s = ensure_work(h, (size_t)chunk * ng, (size_t)chunk * nw)) ||
        (s = grow(h, (void **)&h->MBbuf, &h->MBcap, sizeof(double2) * (size_t)chunk * neig, "projected M")))
        return s;
    const bool split = h->d.prec == GW_PREC_OZAKI_BF16;
    if (split && (s = oz_prepare_b(h, (const double2 *)basis, ng, neig))) return s;
    gw::PairPlan pp = pair_plan(h, sp);
    const double2 *Mres = resident_for(h, iq); // kept by the last gw_chi0_compute of this slot
    for (int64_t p0 = 0; p0 < P; p0 += chunk) {
        const int64_t cnt = std::min(chunk, P - p0);
        const double2 *Mc = Mres ? Mres + p0 * ng : h->Mbuf;
        if (!Mres) {
            Scope sc(h, "pair_mtxel");
            CK(h, run_pair(h, v.psi, h->cond.psi, h->cond.nb, p0, cnt, pp, h->Mbuf), "pair kernel");
        }
        {
            Scope sc(h, "subspace_projection");
            if (split) {
                if ((s = oz_product(h, Mc, cnt, ng, neig, h->MBbuf))) return s;
            } else {
                CK(h, gw::launch_zgemm(Mc, (const double2 *)basis, h->MBbuf, cnt, ng, neig, h->st), "projection");
            }
        }
        {
            Scope sc(h, "delta");
            CK(h, gw::launch_delta(v.energy, h->cond.energy, h->cond.nb, p0, cnt, om, h->dbuf, h->st), "delta");
        }
        if ((s = contract_chunk(h, h->MBbuf, cnt, neig, h->dbuf, cnt, nw, (double2 *)chi_sub))) return s;
    }
    Scope sc(h, "symmetrize");
    CK(h, gw::launch_symmetrize((double2 *)chi_sub, neig, nw, h->st), "symmetrize");
    return GW_OK;
}

// ------------------------------------------------------------------ dielectric matrix inverse
// Dense product C = A B of two [n][n] complex matrices in the handle's precision mode.
static gw_status square_product(gw_chi0 *h, const double2 *A, const double2 *B, int n, double2 *C, int nslices = 0)
{
    if (h->d.prec == GW_PREC_OZAKI_BF16) {
        gw_status st = oz_prepare_b(h, B, n, n, nslices);
        if (st) return st;
        return oz_product(h, A, n, n, n, C, nslices);
    }
    CK(h, gw::launch_zgemm(A, B, C, n, n, n, h->st), "product");
    return GW_OK;
}

// Slices of the split products of the last Newton-Schulz steps (the most the digit step takes).
constexpr int kEpsFinalSlices = 8;

gw_status gw_chi0_epsilon_inverse(gw_chi0 *h, int ng, int nw, const double *chi, const double *vcoul,
                                  double *epsinv)
{
    if (!h) return GW_ERR_ARG;
    if (ng < 1 || nw < 1 || !chi || !vcoul || !epsinv) return fail(h, GW_ERR_ARG, "bad arguments");
    {
        std::vector<double> v(ng);
        CK(h, cudaMemcpyAsync(v.data(), vcoul, sizeof(double) * ng, cudaMemcpyDeviceToHost, h->st), "read v");
        CK(h, cudaStreamSynchronize(h->st), "read v");
        for (int i = 0; i < ng; ++i)
            if (!(v[i] > 0.0) || !std::isfinite(v[i])) return fail(h, GW_ERR_ARG, "v[%d] must be finite and > 0", i);
    }
    const size_t nn = (size_t)ng * ng;
    gw_status st = grow(h, &h->epsbuf, &h->epscap, sizeof(double2) * 4 * nn + sizeof(double) * ng + 64,
                        "dielectric work");
    if (st) return st;
    double2 *A = (double2 *)h->epsbuf, *X = A + nn, *T = X + nn, *Pm = T + nn;
    double *sv = (double *)(Pm + nn);
    unsigned long long *bmax = (unsigned long long *)(((uintptr_t)(sv + ng) + 15) & ~(uintptr_t)15);
    CK(h, gw::launch_eps_sqrt(vcoul, ng, sv, h->st), "sqrt v");
    for (int w = 0; w < nw; ++w) {
        Scope sc(h, "epsilon_inverse");
        CK(h, gw::launch_eps_sym((const double2 *)chi + (int64_t)w * nn, sv, ng, A, bmax, h->st), "I - s chi s");
        unsigned long long bits = 0;
        CK(h, cudaMemcpyAsync(&bits, bmax, sizeof bits, cudaMemcpyDeviceToHost, h->st), "bound");
        CK(h, cudaStreamSynchronize(h->st), "bound");
        double b;
        std::memcpy(&b, &bits, sizeof b);
        if (!(b >= 1.0) || !std::isfinite(b)) return fail(h, GW_ERR_ARG, "I - v chi is not positive (bound %g)", b);
        // steps for (b - 1)/(b + 1) squared repeatedly to reach 1e-17, plus one for rounding
        const double r = (b - 1.0) / (b + 1.0);
        int steps = 1;
        if (r > 0.0) steps = (int)std::ceil(std::log2(std::log(1e-17) / std::log(r))) + 1;
        steps = std::max(steps, 1);
        CK(h, gw::launch_eps_init(X, ng, bmax, h->st), "X0");
        // The error of the converged iterate is the rounding of the last steps' products (earlier
        // errors are squared away), so in split precision the last two steps take the most slices.
        for (int k = 0; k < steps; ++k) {
            Scope sp(h, "eps_products"); // two N_G^3 products per step: the launch count gives the steps
            const int s = (h->d.prec == GW_PREC_OZAKI_BF16 && k >= steps - 2) ? kEpsFinalSlices : 0;
            if ((st = square_product(h, A, X, ng, T, s)) || (st = square_product(h, X, T, ng, Pm, s))) return st;
            CK(h, gw::launch_eps_step(X, Pm, (int64_t)nn, h->st), "Newton-Schulz step");
        }
        CK(h, gw::launch_eps_unsym(X, sv, ng, (double2 *)epsinv + (int64_t)w * nn, h->st), "s X s^-1");
    }
    return GW_OK;
}

// ------------------------------------------------------------------ real frequencies
gw_status gw_chi0_compute_real(gw_chi0 *h, int iq, int nw, const double *omega, double eta, double *chi)
{
    if (!h) return GW_ERR_ARG;
    if (nw < 1 || 3 * nw > gw::kMaxOmega || !omega || !chi)
        return fail(h, GW_ERR_ARG, "bad arguments (1 <= nw <= %d, non-null pointers)", gw::kMaxOmega / 3);
    if (!(eta > 0.0) || !std::isfinite(eta)) return fail(h, GW_ERR_ARG, "eta must be finite and > 0");
    gw::OmegaList om;
    om.nw = nw;
    for (int i = 0; i < nw; ++i) {
        if (!(omega[i] >= 0.0) || !std::isfinite(omega[i])) return fail(h, GW_ERR_ARG, "omega must be finite and >= 0");
        om.w[i] = omega[i];
    }
    gw_status s = check_slot(h, iq);
    if (s) return s;
    const Sphere &sp = h->sph[iq];
    const BandSet &v = h->val[iq];
    const int ng = sp.ng;
    const int64_t nn = (int64_t)ng * ng;
    const int64_t P = (int64_t)v.nb * h->cond.nb;
    const int64_t chunk = std::min<int64_t>(h->d.pair_chunk, P);
    if ((s = grow(h, (void **)&h->realbuf, &h->realcap, sizeof(double2) * 3 * nw * nn, "real-axis parts")) ||
        (s = ensure_work(h, (size_t)chunk * ng, (size_t)chunk * 3 * nw)))
        return s;
    CK(h, cudaMemsetAsync(h->realbuf, 0, sizeof(double2) * 3 * nw * nn, h->st), "zero parts");
    gw::PairPlan pp = pair_plan(h, sp);
    const double2 *Mres = resident_for(h, iq); // kept by the last gw_chi0_compute of this slot
    for (int64_t p0 = 0; p0 < P; p0 += chunk) {
        const int64_t cnt = std::min(chunk, P - p0);
        const double2 *Mc = Mres ? Mres + p0 * ng : h->Mbuf;
        if (!Mres) {
            Scope sc(h, "pair_mtxel");
            CK(h, run_pair(h, v.psi, h->cond.psi, h->cond.nb, p0, cnt, pp, h->Mbuf), "pair kernel");
        }
        {
            Scope sc(h, "delta");
            CK(h, gw::launch_delta_real(v.energy, h->cond.energy, h->cond.nb, p0, cnt, om, eta, h->dbuf, h->st),
               "real-axis delta");
        }
        if ((s = contract_chunk(h, Mc, cnt, ng, h->dbuf, cnt, 3 * nw, h->realbuf))) return s;
    }
    Scope sc(h, "symmetrize");
    CK(h, gw::launch_symmetrize(h->realbuf, ng, 3 * nw, h->st), "symmetrize");
    CK(h, gw::launch_combine_real(h->realbuf, nn, nw, (double2 *)chi, h->st), "combine");
    return GW_OK;
}

// ------------------------------------------------------------------ forward derivative (JVP)
// Real-space grids of caller coefficients on a stored band set's plane waves (the band
// setup of gw_chi0_set_bands, into psi).
static gw_status band_grids(gw_chi0 *h, const BandSet &b, const double *coeff, void *psi)
{
    CK(h, cudaMemsetAsync(psi, 0, sizeof(double2) * (size_t)b.nb * h->nr, h->st), "zero grids");
    if (h->d.mtxel_prec == GW_MTXEL_TWOFLOAT) {
        Scope sc(h, "band_setup_tf");
        CK(h, gw::launch_band_setup_tf((const double2 *)coeff, b.gofs, b.nb, b.ngpsi, psi, h->d.n, h->ax, b.maxabs,
                                       h->st),
           "tangent band setup (two-float)");
    } else {
        CK(h, gw::launch_scatter((const double2 *)coeff, b.gofs, b.nb, b.ngpsi, h->nr, (double2 *)psi, h->st),
           "tangent scatter");
        CK(h, gw::launch_band_fft((double2 *)psi, b.nb, h->d.n, h->ax, h->st), "tangent band fft");
    }
    return GW_OK;
}

gw_status gw_chi0_jvp(gw_chi0 *h, int iq, int nw, const double *omega, const double *dcoeff_v,
                      const double *dcoeff_c, const double *dE_v, const double *dE_c, double *dchi)
{
    if (!h) return GW_ERR_ARG;
    if (nw < 1 || 2 * nw > gw::kMaxOmega || !omega || !dcoeff_v || !dcoeff_c || !dE_v || !dE_c || !dchi)
        return fail(h, GW_ERR_ARG, "bad arguments (1 <= nw <= %d, non-null pointers)", gw::kMaxOmega / 2);
    gw::OmegaList om;
    om.nw = nw;
    for (int i = 0; i < nw; ++i) {
        if (!(omega[i] >= 0.0) || !std::isfinite(omega[i])) return fail(h, GW_ERR_ARG, "omega must be finite and >= 0");
        om.w[i] = omega[i];
    }
    gw_status s = check_slot(h, iq);
    if (s) return s;
    const BandSet &v = h->val[iq];
    const BandSet &c = h->cond;
    const Sphere &sp = h->sph[iq];
    const int ng = sp.ng, nc = c.nb;
    const int64_t nn = (int64_t)ng * ng;
    const int64_t P = (int64_t)v.nb * nc;
    const int64_t chunk = std::min<int64_t>(h->d.pair_chunk, P);
    // work held only for this call
    void *gv = nullptr, *gc = nullptr;
    double2 *X1 = nullptr, *X2 = nullptr, *T = nullptr;
    double *wb = nullptr;
    const size_t szv = sizeof(double2) * (size_t)v.nb * h->nr, szc = sizeof(double2) * (size_t)nc * h->nr;
    const size_t szx = sizeof(double2) * (size_t)chunk * ng, szt = sizeof(double2) * 4 * nw * nn;
    const size_t szw = sizeof(double) * 2 * nw * (size_t)chunk;
    auto cleanup = [&]() {
        cudaStreamSynchronize(h->st);
        dfree(h, gv, szv);
        dfree(h, gc, szc);
        dfree(h, X1, szx);
        dfree(h, X2, szx);
        dfree(h, T, szt);
        dfree(h, wb, szw);
    };
    if ((s = dalloc(h, &gv, szv, "tangent valence grids")) || (s = dalloc(h, &gc, szc, "tangent conduction grids")) ||
        (s = dalloc(h, (void **)&X1, szx, "tangent pairs")) || (s = dalloc(h, (void **)&X2, szx, "tangent pairs")) ||
        (s = dalloc(h, (void **)&T, szt, "tangent parts")) || (s = dalloc(h, (void **)&wb, szw, "tangent weights")) ||
        (s = ensure_work(h, (size_t)chunk * ng, (size_t)chunk * 2 * nw)) || (s = band_grids(h, v, dcoeff_v, gv)) ||
        (s = band_grids(h, c, dcoeff_c, gc))) {
        cleanup();
        return s;
    }
#define JCK(x, what)                            \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) {                \
            gw_status r_ = cuda_fail(h, e_, what); \
            cleanup();                          \
            return r_;                          \
        }                                       \
    } while (0)
    JCK(cudaMemsetAsync(T, 0, szt, h->st), "zero parts");
    double2 *Tp = T, *Tm = T + (int64_t)nw * nn, *Tw = T + 2 * (int64_t)nw * nn;
    gw::PairPlan pp = pair_plan(h, sp);
    const double2 *Mres = resident_for(h, iq); // kept by the last gw_chi0_compute of this slot
    for (int64_t p0 = 0; p0 < P; p0 += chunk) {
        const int64_t cnt = std::min(chunk, P - p0);
        const double2 *Mc = Mres ? Mres + p0 * ng : h->Mbuf;
        {
            Scope sc(h, "pair_mtxel");
            if (!Mres) JCK(run_pair(h, v.psi, c.psi, nc, p0, cnt, pp, h->Mbuf), "pair kernel");
            JCK(run_pair(h, gv, c.psi, nc, p0, cnt, pp, X1), "pair kernel (tangent valence)");
            JCK(run_pair(h, v.psi, gc, nc, p0, cnt, pp, X2), "pair kernel (tangent conduction)");
            JCK(gw::launch_jvp_mix(Mc, X1, X2, cnt * ng, h->st), "M +- dM");
        }
        {
            Scope sc(h, "delta");
            JCK(gw::launch_delta(v.energy, c.energy, nc, p0, cnt, om, h->dbuf, h->st), "delta");
            JCK(gw::launch_delta_jvp(v.energy, c.energy, dE_v, dE_c, nc, p0, cnt, om, wb, h->st), "delta derivative");
        }
        // d chi = [chi(M + dM) - chi(M - dM)] / 2 + sum_p conj(M) dDelta M
        if ((s = contract_chunk(h, X1, cnt, ng, h->dbuf, cnt, nw, Tp)) ||
            (s = contract_chunk(h, X2, cnt, ng, h->dbuf, cnt, nw, Tm)) ||
            (s = contract_chunk(h, Mc, cnt, ng, wb, cnt, 2 * nw, Tw))) {
            cleanup();
            return s;
        }
    }
    {
        Scope sc(h, "symmetrize");
        JCK(gw::launch_symmetrize(T, ng, 4 * nw, h->st), "symmetrize");
        JCK(gw::launch_combine_jvp(Tp, Tm, Tw, nn, nw, (double2 *)dchi, h->st), "combine");
    }
#undef JCK
    cleanup();
    return GW_OK;
}

