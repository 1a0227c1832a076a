// Host side of the C ABI declared in include/gw_chi0.h: handle state, validation,
// library-owned device memory, per-chunk orchestration and optional per-kernel timing.
#include "api_internal.h"

namespace gwapi {
gw_status fail(gw_chi0 *h, gw_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    return s;
}

gw_status cuda_fail(gw_chi0 *h, cudaError_t e, const char *what)
{
    return fail(h, e == cudaErrorMemoryAllocation ? GW_ERR_OOM : GW_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}



gw_status dalloc(gw_chi0 *h, void **p, size_t n, const char *what)
{
    if (n == 0) n = 16;
    if (h->d.mem_budget_bytes && h->bytes + n > h->d.mem_budget_bytes)
        return fail(h, GW_ERR_OOM, "%s: %zu bytes would exceed the memory budget (%zu held, budget %zu)", what, n,
                    h->bytes, h->d.mem_budget_bytes);
    cudaError_t e = cudaMalloc(p, n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, GW_ERR_OOM, "%s: cudaMalloc(%zu) failed: %s", what, n, cudaGetErrorString(e));
    }
    h->bytes += n;
    return GW_OK;
}

void dfree(gw_chi0 *h, void *p, size_t n)
{
    if (!p) return;
    cudaFree(p);
    h->bytes -= (n == 0 ? 16 : n);
}

// Radices for an n-point line transform: as many 4s as possible, 3s and 5s, a leftover 2
// merged with a 4 into an 8.  Odd radices run first: the first Stockham stage stores with
// a stride of R elements, and a stride of 3 or 5 16-byte elements is free of shared-memory
// bank conflicts where 4 and 8 are not.
bool factor(int n, FftAxis &a)
{
    a.n = n;
    a.nst = 0;
    int m = n, n4 = 0, n2 = 0, n3 = 0, n5 = 0;
    while (m % 4 == 0) { ++n4; m /= 4; }
    while (m % 2 == 0) { ++n2; m /= 2; }
    while (m % 3 == 0) { ++n3; m /= 3; }
    while (m % 5 == 0) { ++n5; m /= 5; }
    if (m != 1) return false;
    int n8 = 0;
    if (n2 && n4) { n2 = 0; --n4; n8 = 1; }
    if (n3 + n5 + n4 + n8 + n2 > gw::kMaxStages) return false;
    for (int i = 0; i < n3; ++i) a.rad[a.nst++] = 3;
    for (int i = 0; i < n5; ++i) a.rad[a.nst++] = 5;
    for (int i = 0; i < n4; ++i) a.rad[a.nst++] = 4;
    for (int i = 0; i < n8; ++i) a.rad[a.nst++] = 8;
    for (int i = 0; i < n2; ++i) a.rad[a.nst++] = 2;
    return true;
}

int mod(int a, int n) { return ((a % n) + n) % n; }

// Host-side fault injection for tests: GW_CHI0_FAULT_AT_CHUNK=k makes the streamed compute
// fail before enqueueing chunk k (nothing faults on the device).
int64_t fault_chunk()
{
    const char *e = std::getenv("GW_CHI0_FAULT_AT_CHUNK");
    return e ? std::atoll(e) : -1;
}

// ------------------------------------------------------------------ timing helpers
cudaEvent_t ev_get(gw_chi0 *h)
{
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}



void drain_timing(gw_chi0 *h)
{
    if (h->pending.empty()) return;
    cudaStreamSynchronize(h->st);
    for (auto &r : h->pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto &x = h->acc[r.name];
        x.first += ms;
        x.second += 1;
        h->pool.push_back(r.a);
        h->pool.push_back(r.b);
    }
    h->pending.clear();
}

// ------------------------------------------------------------------ buffers
gw_status ensure_work(gw_chi0 *h, size_t m_elems, size_t d_elems)
{
    if (m_elems > h->Mcap) {
        dfree(h, h->Mbuf, h->Mcap * sizeof(double2));
        h->Mbuf = nullptr;
        h->Mcap = 0;
        gw_status s = dalloc(h, (void **)&h->Mbuf, m_elems * sizeof(double2), "M chunk buffer");
        if (s) return s;
        h->Mcap = m_elems;
    }
    if (d_elems > h->dcap) {
        dfree(h, h->dbuf, h->dcap * sizeof(double));
        h->dbuf = nullptr;
        h->dcap = 0;
        gw_status s = dalloc(h, (void **)&h->dbuf, d_elems * sizeof(double), "Delta buffer");
        if (s) return s;
        h->dcap = d_elems;
    }
    return GW_OK;
}

gw_status make_tmap(gw_chi0 *h, CUtensorMap *map, const void *M, int64_t P, int ng, int bt)
{
    if (((uintptr_t)M & 15) != 0) return fail(h, GW_ERR_ARG, "M must be 16-byte aligned");
    cuuint64_t dims[2] = {(cuuint64_t)2 * ng, (cuuint64_t)P};
    cuuint64_t strides[1] = {(cuuint64_t)2 * ng * sizeof(double)};
    cuuint32_t box[2] = {(cuuint32_t)(2 * bt), (cuuint32_t)gw::contract_f64_bk()};
    cuuint32_t es[2] = {1, 1};
    CUresult r = h->encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void *>(M), dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, GW_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return GW_OK;
}

int num_sms()
{
    int sms = 152, dev;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// Captured graphs hold raw device pointers: drop them whenever a buffer they may use is
// reallocated or the bands or spheres change (they are recaptured on the next call).
void drop_graphs(gw_chi0 *h)
{
    if (h->graphs.empty()) return;
    cudaStreamSynchronize(h->st); // a replay may still be running
    for (auto &g : h->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        dfree(h, g.jobs, g.jobs_bytes);
    }
    h->graphs.clear();
}

gw_status grow(gw_chi0 *h, void **p, size_t *cap, size_t bytes, const char *what)
{
    if (bytes <= *cap) return GW_OK;
    if (*p) drop_graphs(h);
    dfree(h, *p, *cap);
    *p = nullptr;
    *cap = 0;
    gw_status s = dalloc(h, p, bytes, what);
    if (s) return s;
    *cap = bytes;
    return GW_OK;
}

// Copy a job table into the handle's job buffer, in stream order (the copy runs after every
// kernel already enqueued, so rewriting the buffer never races a kernel that reads it).
gw_status upload_jobs(gw_chi0 *h, const void *src, size_t bytes, const void **dev)
{
    gw_status s = grow(h, &h->jobbuf, &h->jobcap, bytes, "job table");
    if (s) return s;
    CK(h, cudaMemcpyAsync(h->jobbuf, src, bytes, cudaMemcpyHostToDevice, h->st), "job table upload");
    *dev = h->jobbuf;
    return GW_OK;
}

// FP64 jobs for one M block and nw frequencies; item_start and ksplit filled in by the caller.
gw_status f64_jobs(gw_chi0 *h, std::vector<gw::F64Job> &jobs, const double2 *M, int64_t P, int ng,
                   const double *delta, int64_t dstride, int nw, double2 *chi, int bt)
{
    CUtensorMap map;
    gw_status s = make_tmap(h, &map, M, P, ng, bt);
    if (s) return s;
    for (int w = 0; w < nw; ++w) {
        gw::F64Job j;
        std::memset(&j, 0, sizeof j);
        j.tm = map;
        j.delta = delta + (int64_t)w * dstride;
        j.chi = (double *)(chi + (int64_t)w * ng * ng);
        j.P = P;
        j.ng = ng;
        j.ntile = (ng + bt - 1) / bt;
        jobs.push_back(j);
    }
    return GW_OK;
}

// Order jobs largest first, pick a uniform pair split for `waves` block waves, set item ranges.
int f64_schedule(std::vector<gw::F64Job> &jobs, int waves)
{
    std::stable_sort(jobs.begin(), jobs.end(), [](const gw::F64Job &a, const gw::F64Job &b) {
        return (double)a.ng * a.ng * a.P > (double)b.ng * b.ng * b.P;
    });
    int64_t tiles = 0;
    for (auto &j : jobs) tiles += (int64_t)j.ntile * (j.ntile + 1) / 2;
    const int64_t want = (int64_t)waves * 2 * num_sms();
    int64_t ks = std::max<int64_t>(1, (want + tiles - 1) / std::max<int64_t>(tiles, 1));
    int items = 0;
    for (auto &j : jobs) {
        int64_t kj = std::min<int64_t>(ks, std::max<int64_t>(1, (j.P + 255) / 256)); // >= 256 pairs per item
        j.ksplit = (int)kj;
        j.item_start = items;
        items += (int)(kj * j.ntile * (j.ntile + 1) / 2);
    }
    return items;
}

gw_status launch_f64_jobs(gw_chi0 *h, std::vector<gw::F64Job> &jobs, int bt, int waves)
{
    const int nitems = f64_schedule(jobs, waves);
    const void *dj;
    gw_status s = upload_jobs(h, jobs.data(), sizeof(gw::F64Job) * jobs.size(), &dj);
    if (s) return s;
    const int grid = std::max(1, std::min(nitems, 2 * num_sms()));
    Scope sc(h, "contract_f64");
    CK(h, gw::launch_contract_f64_jobs(bt, (const gw::F64Job *)dj, (int)jobs.size(), nitems, grid, h->status, h->st),
       "contract_f64");
    return GW_OK;
}

gw_status make_tmap_z(gw_chi0 *h, CUtensorMap *map, void *Z, int64_t kpad, int nrows, int s, int box_rows)
{
    cuuint64_t dims[3] = {(cuuint64_t)kpad, (cuuint64_t)nrows, (cuuint64_t)s};
    cuuint64_t strides[2] = {(cuuint64_t)kpad * 2, (cuuint64_t)kpad * 2 * nrows};
    cuuint32_t box[3] = {(cuuint32_t)gw::oz_box_k(), (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = h->encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, Z, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, GW_ERR_CUDA, "cuTensorMapEncodeTiled (slices) failed (%d)", (int)r);
    return GW_OK;
}

// GW_CHI0_SPLIT_TILE=128|240|256, read at every contraction, forces the width (the result does not
// depend on it: every entry sums the same slice products in the same K order)
int contraction_bn(const gw_chi0 *h, int ng)
{
    if (const char *e = getenv("GW_CHI0_SPLIT_TILE")) {
        const int v = atoi(e);
        if (v == 128 || v == 240 || v == 256) return v;
    }
    return h->bn_tuned ? h->tuned_bn : gw::oz_pick_bn(ng, num_sms());
}

gw_status oz_job(gw_chi0 *h, gw::OzJob &j, void *Z, int64_t kpad, int ng, const int *E, double2 *chi, int bn)
{
    std::memset(&j, 0, sizeof j);
    gw_status st;
    if ((st = make_tmap_z(h, &j.tmA, Z, kpad, 2 * ng, h->d.nslices, gw::oz_box_rows_a())) ||
        (st = make_tmap_z(h, &j.tmB, Z, kpad, 2 * ng, h->d.nslices, bn)))
        return st;
    j.E = E;
    j.chi = (double *)chi;
    j.ng = ng;
    j.nk = (int)(kpad / gw::oz_box_k());
    j.s = h->d.nslices;
    j.ntiles = gw::oz_tiles(ng, bn);
    return GW_OK;
}

int oz_schedule(std::vector<gw::OzJob> &jobs)
{
    std::stable_sort(jobs.begin(), jobs.end(), [](const gw::OzJob &a, const gw::OzJob &b) {
        return (double)a.ng * a.ng * a.nk > (double)b.ng * b.ng * b.nk;
    });
    int items = 0;
    for (auto &j : jobs) {
        j.item_start = items;
        items += j.ntiles;
    }
    return items;
}

gw_status launch_oz_jobs(gw_chi0 *h, std::vector<gw::OzJob> &jobs, int bn)
{
    const int nitems = oz_schedule(jobs);
    const void *dj;
    gw_status s = upload_jobs(h, jobs.data(), sizeof(gw::OzJob) * jobs.size(), &dj);
    if (s) return s;
    const int grid = std::max(1, std::min(nitems, num_sms()));
    Scope sc(h, "ozaki_gemm");
    CK(h, gw::launch_oz_gemm_jobs(bn, (const gw::OzJob *)dj, (int)jobs.size(), nitems, grid, h->status, h->st),
       "oz gemm");
    return GW_OK;
}

// Split-precision contraction of one chunk for each frequency (chi blocks [nw][ng][ng]).
gw_status contract_chunk_ozaki(gw_chi0 *h, const double2 *M, int64_t P, int ng, const double *delta, int64_t dstride,
                               int nw, double2 *chi)
{
    const int s = h->d.nslices;
    const int64_t kpad = (P + 63) / 64 * 64;
    const size_t zper = (size_t)s * 2 * ng * kpad; // bf16 slices of one frequency
    // several frequencies: slice a group at once (M read once per pass for the group), the group's
    // slices within 4 GiB
    const int wg = nw == 1 ? 1 : std::max(1, std::min({nw, gw::oz_group_w(), (int)(4294967296.0 / (2.0 * zper))}));
    gw_status st;
    if ((st = grow(h, &h->Zbuf, &h->Zcap, zper * 2 * wg, "slice buffer")) ||
        (st = grow(h, (void **)&h->spbuf, &h->spcap, sizeof(double) * (size_t)nw * dstride, "scale buffer")) ||
        (st = grow(h, (void **)&h->Ebuf, &h->Ecap, sizeof(int) * (size_t)ng * wg, "exponent buffer")))
        return st;
    {
        Scope sc(h, "oz_split");
        CK(h, gw::launch_oz_sqrt(delta, (int64_t)nw * dstride, h->spbuf, h->st), "oz sqrt");
    }
    const int bn = contraction_bn(h, ng);
    for (int w0 = 0; w0 < nw; w0 += wg) {
        const int cnt = std::min(wg, nw - w0);
        const double *sp = h->spbuf + (int64_t)w0 * dstride;
        {
            Scope sc(h, "oz_split");
            if (cnt == 1) {
                CK(h, gw::launch_oz_colexp(M, P, ng, sp, h->Ebuf, h->st), "oz exponents");
                CK(h, gw::launch_oz_slice(M, P, ng, sp, h->Ebuf, s, kpad, h->Zbuf, h->st), "oz slices");
            } else {
                CK(h, gw::launch_oz_split_multi(M, P, ng, sp, dstride, cnt, h->Ebuf, s, kpad, h->Zbuf, (int64_t)zper,
                                                h->st),
                   "oz slices (frequency group)");
            }
        }
        for (int j = 0; j < cnt; ++j) {
            std::vector<gw::OzJob> jobs(1);
            if ((st = oz_job(h, jobs[0], (uint16_t *)h->Zbuf + zper * j, kpad, ng, h->Ebuf + (size_t)ng * j,
                             chi + (int64_t)(w0 + j) * ng * ng, bn)))
                return st;
            // few tiles (small N_G): split K over jobs so that about one wave of blocks runs,
            // at least 8 K-steps each; the atomic epilogue adds the parts
            const int nk = jobs[0].nk;
            const int ks = std::max(1, std::min(num_sms() / std::max(1, jobs[0].ntiles), nk / 8));
            if (ks > 1) {
                const gw::OzJob base = jobs[0];
                jobs.assign(ks, base);
                for (int i = 0; i < ks; ++i) {
                    jobs[i].kb0 = (int)((int64_t)nk * i / ks);
                    jobs[i].nk = (int)((int64_t)nk * (i + 1) / ks) - jobs[i].kb0;
                }
            }
            if ((st = launch_oz_jobs(h, jobs, bn))) return st;
        }
    }
    return GW_OK;
}

gw_status contract_chunk(gw_chi0 *h, const double2 *M, int64_t P, int ng, const double *delta, int64_t dstride,
                         int nw, double2 *chi)
{
    if (h->d.prec == GW_PREC_OZAKI_BF16) return contract_chunk_ozaki(h, M, P, ng, delta, dstride, nw, chi);
    std::vector<gw::F64Job> jobs;
    gw_status s = f64_jobs(h, jobs, M, P, ng, delta, dstride, nw, chi, h->tuned_bt);
    if (s) return s;
    return launch_f64_jobs(h, jobs, h->tuned_bt, h->tuned_waves);
}

// Real K extent of a general product with ka complex inner entries, padded for the TMA boxes.
int64_t oz_kpad(int ka) { return ((int64_t)2 * ka + 63) / 64 * 64; }

// B operand of a general split product: the columns of B [ka][nout] (complex, row-major)
// into the handle's ZB / EB buffers.
gw_status oz_prepare_b(gw_chi0 *h, const double2 *B, int ka, int nout, int nslices)
{
    const int s = nslices > 0 ? nslices : h->d.nslices;
    const int64_t kpad = oz_kpad(ka);
    gw_status st;
    if ((st = grow(h, &h->ZBbuf, &h->ZBcap, (size_t)s * 2 * nout * kpad * 2, "product operand slices")) ||
        (st = grow(h, (void **)&h->EBbuf, &h->EBcap, sizeof(int) * (size_t)nout, "product operand exponents")))
        return st;
    CK(h, gw::launch_oz_split_cols(B, ka, nout, nout, 1, false, s, kpad, h->ZBbuf, h->EBbuf, h->st),
       "oz column slices");
    return GW_OK;
}

// Y[rows][nout] = A[rows][ka] B[ka][nout] (complex, row-major) in split precision, B prepared
// by oz_prepare_b.  A's slices reuse the contraction's slice buffer (stream order separates
// the two uses).
gw_status oz_product(gw_chi0 *h, const double2 *A, int64_t rows, int ka, int nout, double2 *Y, int nslices)
{
    const int s = nslices > 0 ? nslices : h->d.nslices;
    const int64_t kpad = oz_kpad(ka);
    const int bn = 2 * nout >= 256 ? 256 : 128;
    gw_status st;
    if ((st = grow(h, &h->Zbuf, &h->Zcap, (size_t)s * rows * kpad * 2, "slice buffer")) ||
        (st = grow(h, (void **)&h->EAbuf, &h->EAcap, sizeof(int) * (size_t)rows, "product row exponents")))
        return st;
    CK(h, cudaMemsetAsync(Y, 0, sizeof(double2) * (size_t)rows * nout, h->st), "zero product");
    CK(h, gw::launch_oz_split_rows(A, rows, ka, s, kpad, h->Zbuf, h->EAbuf, h->st), "oz row slices");
    gw::OzJob j;
    std::memset(&j, 0, sizeof j);
    if ((st = make_tmap_z(h, &j.tmA, h->Zbuf, kpad, (int)rows, s, gw::oz_box_rows_a())) ||
        (st = make_tmap_z(h, &j.tmB, h->ZBbuf, kpad, 2 * nout, s, bn)))
        return st;
    j.E = h->EAbuf;
    j.E2 = h->EBbuf;
    j.out = (double *)Y;
    j.ldo = 2 * (int64_t)nout;
    j.rows_a = (int)rows;
    j.rows_b = 2 * nout;
    j.nk = (int)(kpad / gw::oz_box_k());
    j.s = s;
    j.ntiles = (int)((rows + gw::oz_box_rows_a() - 1) / gw::oz_box_rows_a()) * ((2 * nout + bn - 1) / bn);
    j.item_start = 0;
    const void *dj;
    if ((st = upload_jobs(h, &j, sizeof j, &dj))) return st;
    CK(h, gw::launch_oz_gemm_general(bn, (const gw::OzJob *)dj, 1, j.ntiles, std::min(j.ntiles, num_sms()), h->status,
                                     h->st),
       "oz general product");
    return GW_OK;
}

bool alias_free(const gw_chi0 *h, const BandSet &v, const BandSet &c, const Sphere &s, int *axis)
{
    for (int a = 0; a < 3; ++a)
        if (v.maxabs[a] + c.maxabs[a] + s.maxabs[a] >= h->d.n[a]) {
            *axis = a;
            return false;
        }
    return true;
}

gw_status check_slot(gw_chi0 *h, int iq)
{
    if (iq < 0 || iq >= h->d.nq) return fail(h, GW_ERR_ARG, "q slot %d out of range [0, %d)", iq, h->d.nq);
    const BandSet &v = h->val[iq];
    const Sphere &s = h->sph[iq];
    if (v.nb == 0) return fail(h, GW_ERR_STATE, "valence bands of slot %d not set", iq);
    if (h->cond.nb == 0) return fail(h, GW_ERR_STATE, "conduction bands not set");
    if (s.ng == 0) return fail(h, GW_ERR_STATE, "G-sphere of slot %d not set", iq);
    int ax;
    if (!alias_free(h, v, h->cond, s, &ax))
        return fail(h, GW_ERR_ARG, "slot %d: max|K_v| + max|K_c| + max|G| >= n on axis %d (aliasing)", iq, ax);
    double vmax = *std::max_element(v.e.begin(), v.e.end());
    double cmin = *std::min_element(h->cond.e.begin(), h->cond.e.end());
    if (!(vmax < cmin)) return fail(h, GW_ERR_ARG, "slot %d: a valence energy is not below every conduction energy", iq);
    return GW_OK;
}

cudaError_t run_pair(gw_chi0 *h, const void *psiv, const void *psic, int nc, int64_t p0, int64_t cnt,
                     const gw::PairPlan &pp, double2 *M)
{
    if (h->d.mtxel_prec == GW_MTXEL_TWOFLOAT) return gw::launch_pair_tf(psiv, psic, nc, p0, cnt, pp, M, h->st);
    return gw::launch_pair((const double2 *)psiv, (const double2 *)psic, nc, p0, cnt, pp, M, h->st);
}

gw::PairPlan pair_plan(gw_chi0 *h, const Sphere &s)
{
    gw::PairPlan pp;
    for (int a = 0; a < 3; ++a) {
        pp.n[a] = h->d.n[a];
        pp.ax[a] = h->ax[a];
    }
    pp.K2 = s.K2;
    pp.kz = s.kz;
    pp.ng = s.ng;
    pp.gpack = s.gpack;
    pp.K12 = s.K12;
    pp.cell = s.cell;
    pp.cstart = s.cstart_d;
    pp.cpts = s.cpts;
    pp.scr = h->pscr;
    pp.slot_flags = h->pflags;
    pp.nslots = s.nslots;
    pp.status = h->status;
    return pp;
}

void free_bands(gw_chi0 *h, BandSet &b)
{
    dfree(h, b.psi, sizeof(double2) * (size_t)b.nb * h->nr);
    dfree(h, b.energy, sizeof(double) * b.nb);
    dfree(h, b.gvec, sizeof(int32_t) * 3 * b.ngpsi);
    dfree(h, b.gofs, sizeof(int32_t) * b.ngpsi);
    b = BandSet();
}

void free_sphere(gw_chi0 *h, Sphere &s)
{
    dfree(h, s.kz, sizeof(int) * s.K2);
    dfree(h, s.gpack, sizeof(int32_t) * s.ng);
    dfree(h, s.gvec, sizeof(int32_t) * 3 * s.ng);
    dfree(h, s.cell, sizeof(int32_t) * s.K12);
    dfree(h, s.cstart_d, sizeof(int) * (s.K12 + 1));
    dfree(h, s.cpts, sizeof(int2) * s.ng);
    s = Sphere();
}
// The high-priority second stream and the events of the overlapped paths (created on first use).
gw_status ensure_overlap_stream(gw_chi0 *h)
{
    if (h->ov_st) return GW_OK;
    int lo = 0, hi = 0;
    CK(h, cudaDeviceGetStreamPriorityRange(&lo, &hi), "stream priorities");
    CK(h, cudaStreamCreateWithPriority(&h->ov_st, cudaStreamNonBlocking, hi), "contraction stream");
    for (int b = 0; b < 2; ++b) {
        CK(h, cudaEventCreateWithFlags(&h->ov_split[b], cudaEventDisableTiming), "event");
        CK(h, cudaEventCreateWithFlags(&h->ov_gemm[b], cudaEventDisableTiming), "event");
    }
    return GW_OK;
}

// ------------------------------------------------------------------ stage (a) on the tensor cores
// The last-axis transform of the pair products as a split product per grid line (zdft.cu) for
// two-float stage (a) on the 48^3 grid; chunks are all valence bands x a block of conduction
// bands, rows r = cl nv + v, on one stream (the last-axis product and the split contraction each
// need whole SMs' shared memory: running the contraction on a second stream beside the next
// chunk's FP32 stages measured slower, 163 against 142 ms per 48^3 q-point).
// GW_CHI0_STAGE_A=fft selects the FFT pair kernel instead.
bool zd_route(gw_chi0 *h, int iq, bool resident)
{
    static const bool fft_only = [] {
        const char *e = getenv("GW_CHI0_STAGE_A");
        return e && strcmp(e, "fft") == 0;
    }();
    if (fft_only || resident || h->d.mtxel_prec != GW_MTXEL_TWOFLOAT) return false;
    const Sphere &sp = h->sph[iq];
    const int n = h->d.n[0];
    if (h->d.n[1] != n || h->d.n[2] != n || sp.nslots <= 0 || !h->pscr) return false;
    return gw::zd_supported(n, sp.K2, h->val[iq].nb) && h->d.pair_chunk >= h->val[iq].nb;
}

int zd_chunk_bands(gw_chi0 *h, int iq)
{
    const int nv = h->val[iq].nb;
    return (int)std::max<int64_t>(1, std::min<int64_t>(h->cond.nb, h->d.pair_chunk / nv));
}

gw_status zd_prepare(gw_chi0 *h, int iq, CUtensorMap *tmA, CUtensorMap *tmC)
{
    const BandSet &v = h->val[iq];
    const Sphere &sp = h->sph[iq];
    const int n = h->d.n[0], nv = v.nb, cb = zd_chunk_bands(h, iq);
    const int64_t lines = (int64_t)n * n;
    const size_t abytes = (size_t)gw::kZdSlices * lines * nv * 2 * n * 2;
    const size_t fbytes = sizeof(float4) * (size_t)lines * nv * cb * sp.K2;
    gw_status s;
    if ((s = grow(h, &h->zdA, &h->zdAcap, abytes, "valence slices")) ||
        (s = grow(h, (void **)&h->zdF, &h->zdFcap, fbytes, "last-axis transform")))
        return s;
    {
        Scope sc(h, "zd_aslices");
        CK(h, gw::launch_zd_aslices(v.psi, nv, n, (uint16_t *)h->zdA, h->st), "valence slices");
    }
    cuuint64_t dims[4] = {(cuuint64_t)2 * n, (cuuint64_t)nv, (cuuint64_t)lines, (cuuint64_t)gw::kZdSlices};
    cuuint64_t strides[3] = {(cuuint64_t)2 * n * 2, (cuuint64_t)2 * n * 2 * nv, (cuuint64_t)2 * n * 2 * nv * lines};
    cuuint32_t box[4] = {32, 128, 1, (cuuint32_t)gw::kZdSlices};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = h->encode(tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, h->zdA, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, GW_ERR_CUDA, "cuTensorMapEncodeTiled (valence slices) failed (%d)", (int)r);
    // the conduction grids, line by line: box of one line of CT bands
    cuuint64_t cd[3] = {(cuuint64_t)4 * n, (cuuint64_t)lines, (cuuint64_t)h->cond.nb};
    cuuint64_t cst[2] = {(cuuint64_t)4 * n * 4, (cuuint64_t)16 * lines * n};
    cuuint32_t cbox[3] = {(cuuint32_t)(4 * n), 1, (cuuint32_t)gw::zd_conduction_per_tile(sp.K2)};
    cuuint32_t ces[3] = {1, 1, 1};
    r = h->encode(tmC, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, h->cond.psi, cd, cst, cbox, ces, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, GW_ERR_CUDA, "cuTensorMapEncodeTiled (conduction grids) failed (%d)", (int)r);
    return GW_OK;
}

gw_status zd_stage_a(gw_chi0 *h, int iq, const CUtensorMap &tmA, const CUtensorMap &tmC, int c0, int cb,
                     const gw::PairPlan &pp, double2 *M)
{
    const BandSet &v = h->val[iq];
    const Sphere &sp = h->sph[iq];
    const int n = h->d.n[0];
    {
        Scope sc(h, "zdft");
        CK(h, gw::launch_zd_gemm(tmA, tmC, h->cond.psi, sp.kz, pp.ax[2].twf, n, v.nb, c0, cb, sp.K2, h->zdF,
                                 h->status, h->st),
           "last-axis transform");
    }
    // F as [n^2 lines][R K2] two-float entries: the middle/first-axis kernel loads a slab pair's
    // 2n lines of one row (K2 entries each) with one TMA box
    const int64_t R = (int64_t)v.nb * cb;
    CUtensorMap tmF;
    cuuint64_t fd[2] = {(cuuint64_t)R * sp.K2 * 4, (cuuint64_t)n * n};
    cuuint64_t fst[1] = {(cuuint64_t)R * sp.K2 * 16};
    cuuint32_t fbox[2] = {(cuuint32_t)(sp.K2 * 4), (cuuint32_t)(2 * n)};
    cuuint32_t fes[2] = {1, 1};
    CUresult r = h->encode(&tmF, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h->zdF, fd, fst, fbox, fes,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, GW_ERR_CUDA, "cuTensorMapEncodeTiled (last-axis output) failed (%d)", (int)r);
    // the scratch slots as [nslots n rows][K12] entries: phase 2 loads batches of 2 K2 cells of
    // all n rows of its slot with one TMA box
    CUtensorMap tmS;
    cuuint64_t sd[2] = {(cuuint64_t)pp.K12 * 4, (cuuint64_t)pp.nslots * n};
    cuuint64_t sst[1] = {(cuuint64_t)pp.K12 * 16};
    cuuint32_t sbox[2] = {(cuuint32_t)(8 * sp.K2), (cuuint32_t)n};
    r = h->encode(&tmS, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, pp.scr, sd, sst, sbox, fes, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, GW_ERR_CUDA, "cuTensorMapEncodeTiled (pair scratch) failed (%d)", (int)r);
    Scope sc(h, "pair_from_f");
    CK(h, gw::launch_pair_tf_from_f(tmF, tmS, R, pp, M, h->st), "pair elements from F");
    return GW_OK;
}

// Split-precision streamed compute with the contraction of job j (chunk, frequency) on a
// high-priority second stream while the user stream forms the pair elements and slices of
// the jobs after it.  The split-precision contraction runs on the tensor cores and the pair
// kernel on the FP32 pipes, so the two share the SMs: the contraction uses a 2-deep TMA ring
// (99 KB of shared memory) to fit beside two pair-kernel blocks.  Slices, exponents and job
// tables alternate between two buffer sets; job j waits for the contraction of job j - 2.
// The overlapped path pays off when two pair-kernel blocks fit on an SM beside a contraction
// block (48^3: 180 vs 189 ms per q-point); with room for one (72^3, 112 KB pair blocks) the pair
// kernel, the critical path, runs at half its occupancy (5.9 vs 4.8 s per q-point).
bool overlap_enabled(gw_chi0 *h, const gw::PairPlan &pp)
{
    if (h->d.prec != GW_PREC_OZAKI_BF16 || h->d.single_stream || h->d.mtxel_prec != GW_MTXEL_TWOFLOAT) return false;
    const size_t ps = gw::pair_tf_ct_smem_bytes(pp);
    if (ps == 0) return false;
    int dev = 0, sm_bytes = 0, resv = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const size_t gs = std::max(gw::oz_smem_bytes(256, 2), gw::oz_smem_bytes(h->tuned_bn, 2));
    return 2 * (ps + (size_t)resv) + gs + (size_t)resv <= (size_t)sm_bytes;
}

gw_status resident_begin(gw_chi0 *h, int64_t P, int ng, bool *use)
{
    *use = false;
    h->Mres_iq = -1;
    if (!h->keep_m) return GW_OK;
    const size_t need = sizeof(double2) * (size_t)P * ng;
    if (h->d.mem_budget_bytes && h->bytes - h->Mres_cap + need > h->d.mem_budget_bytes) return GW_OK;
    size_t free_b = 0, total_b = 0;
    if (need > h->Mres_cap && (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess || need - h->Mres_cap > free_b / 2)) {
        cudaGetLastError();
        return GW_OK; // keep at most half of what is free: the elements are an optimisation, not a need
    }
    gw_status s = grow(h, (void **)&h->Mres, &h->Mres_cap, need, "resident pair elements");
    if (s) return s;
    *use = true;
    return GW_OK;
}

double2 *resident_for(gw_chi0 *h, int iq) { return h->keep_m && h->Mres_iq == iq ? h->Mres : nullptr; }

gw_status compute_overlap(gw_chi0 *h, int iq, const gw::OmegaList &om, double2 *cq, double *dq, double2 *Mres)
{
    const Sphere &sp = h->sph[iq];
    const BandSet &v = h->val[iq];
    const int ng = sp.ng, nw = om.nw, s = h->d.nslices;
    const int64_t P = (int64_t)v.nb * h->cond.nb;
    const int64_t chunk = std::min<int64_t>(h->d.pair_chunk, P);
    const int64_t kpad_max = (chunk + 63) / 64 * 64;
    gw_status st = ensure_work(h, (size_t)chunk * ng, (size_t)chunk * nw);
    if (st) return st;
    if ((st = grow(h, (void **)&h->spbuf, &h->spcap, sizeof(double) * (size_t)nw * chunk, "scale buffer"))) return st;
    for (int b = 0; b < 2; ++b)
        if ((st = grow(h, &h->ovZ[b], &h->ovZcap[b], (size_t)s * 2 * ng * kpad_max * 2, "slice buffer")) ||
            (st = grow(h, (void **)&h->ovE[b], &h->ovEcap[b], sizeof(int) * (size_t)ng, "exponent buffer")) ||
            (st = grow(h, &h->ovJ[b], &h->ovJcap[b], sizeof(gw::OzJob) * 256, "job table")))
            return st;
    if ((st = ensure_overlap_stream(h))) return st;
    const int bn = contraction_bn(h, ng);
    gw::PairPlan pp = pair_plan(h, sp);
    bool used[2] = {false, false};
    int64_t j = 0;
    for (int64_t p0 = 0; p0 < P; p0 += chunk) {
        const int64_t cnt = std::min(chunk, P - p0);
        const int64_t kpad = (cnt + 63) / 64 * 64;
        double2 *Mc = Mres ? Mres + p0 * ng : h->Mbuf;
        {
            Scope sc(h, "pair_mtxel");
            CK(h, run_pair(h, v.psi, h->cond.psi, h->cond.nb, p0, cnt, pp, Mc), "pair kernel");
        }
        {
            Scope sc(h, "delta");
            CK(h, gw::launch_delta(v.energy, h->cond.energy, h->cond.nb, p0, cnt, om, h->dbuf, h->st), "delta");
        }
        {
            Scope sc(h, "oz_split");
            CK(h, gw::launch_oz_sqrt(h->dbuf, (int64_t)nw * cnt, h->spbuf, h->st), "oz sqrt");
        }
        if (dq) {
            Scope sc(h, "diag");
            CK(h, gw::launch_diag(Mc, cnt, ng, h->dbuf, cnt, nw, dq, ng, h->st), "diag");
        }
        for (int w = 0; w < nw; ++w, ++j) {
            const int b = (int)(j & 1);
            if (used[b]) CK(h, cudaStreamWaitEvent(h->st, h->ov_gemm[b], 0), "wait contraction");
            {
                Scope sc(h, "oz_split");
                const double *spw = h->spbuf + (int64_t)w * cnt;
                CK(h, gw::launch_oz_colexp(Mc, cnt, ng, spw, h->ovE[b], h->st), "oz exponents");
                CK(h, gw::launch_oz_slice(Mc, cnt, ng, spw, h->ovE[b], s, kpad, h->ovZ[b], h->st), "oz slices");
            }
            std::vector<gw::OzJob> jobs(1);
            if ((st = oz_job(h, jobs[0], h->ovZ[b], kpad, ng, h->ovE[b], cq + (int64_t)w * ng * ng, bn))) return st;
            const int nitems = oz_schedule(jobs);
            CK(h, cudaMemcpyAsync(h->ovJ[b], jobs.data(), sizeof(gw::OzJob) * jobs.size(), cudaMemcpyHostToDevice,
                                  h->st),
               "job table");
            CK(h, cudaEventRecord(h->ov_split[b], h->st), "record");
            CK(h, cudaStreamWaitEvent(h->ov_st, h->ov_split[b], 0), "wait slices");
            {
                Scope sc(h, "ozaki_gemm", h->ov_st);
                CK(h, gw::launch_oz_gemm_jobs(bn, (const gw::OzJob *)h->ovJ[b], (int)jobs.size(), nitems,
                                              std::max(1, std::min(nitems, num_sms())), h->status, h->ov_st, 2),
                   "oz gemm");
            }
            CK(h, cudaEventRecord(h->ov_gemm[b], h->ov_st), "record");
            used[b] = true;
        }
    }
    for (int b = 0; b < 2; ++b)
        if (used[b]) CK(h, cudaStreamWaitEvent(h->st, h->ov_gemm[b], 0), "join");
    return GW_OK;
}
} // namespace gwapi

using namespace gwapi;
// =================================================================== C ABI
extern "C" {

gw_status gw_chi0_create(gw_chi0 **out, const gw_chi0_desc *d, void *stream)
{
    if (!out || !d) return GW_ERR_ARG;
    *out = nullptr;
    gw_chi0 *h = new (std::nothrow) gw_chi0();
    if (!h) return GW_ERR_OOM;
    h->d = *d;
    h->st = (cudaStream_t)stream;
    if (h->d.pair_chunk <= 0) h->d.pair_chunk = 8192;
    if (h->d.nq < 1) { delete h; return GW_ERR_ARG; }
    if (h->d.prec != GW_PREC_FP64 && h->d.prec != GW_PREC_OZAKI_BF16) { delete h; return GW_ERR_ARG; }
    if (h->d.prec == GW_PREC_OZAKI_BF16 && (h->d.nslices < 3 || h->d.nslices > 8)) { delete h; return GW_ERR_ARG; }
    if (h->d.mtxel_prec != GW_MTXEL_FP64 && h->d.mtxel_prec != GW_MTXEL_TWOFLOAT) { delete h; return GW_ERR_ARG; }
    if (h->d.single_stream != 0 && h->d.single_stream != 1) { delete h; return GW_ERR_ARG; }
    for (int a = 0; a < 3; ++a) {
        int n = h->d.n[a];
        if (n < 4 || n > 128 || !factor(n, h->ax[a])) { delete h; return GW_ERR_ARG; }
    }
    if (cudaSetDevice(h->d.device) != cudaSuccess) { cudaGetLastError(); delete h; return GW_ERR_CUDA; }
    h->nr = (int64_t)h->d.n[0] * h->d.n[1] * h->d.n[2];
    h->val.resize(h->d.nq);
    h->sph.resize(h->d.nq);

    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        delete h;
        return GW_ERR_CUDA;
    }
    h->encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;

    // twiddle tables e^{+2 pi i t/n}, computed in extended precision on the host
    int ntot = h->d.n[0] + h->d.n[1] + h->d.n[2];
    std::vector<double2> tw(ntot);
    int off = 0;
    for (int a = 0; a < 3; ++a) {
        int n = h->d.n[a];
        for (int t = 0; t < n; ++t) {
            long double ang = 2.0L * 3.141592653589793238462643383279502884L * (long double)t / (long double)n;
            tw[off + t] = make_double2((double)cosl(ang), (double)sinl(ang));
        }
        off += n;
    }
    std::vector<float4> twf(ntot);
    for (int t = 0; t < ntot; ++t) {
        float rh = (float)tw[t].x, ih = (float)tw[t].y;
        twf[t] = make_float4(rh, (float)(tw[t].x - (double)rh), ih, (float)(tw[t].y - (double)ih));
    }
    if (dalloc(h, (void **)&h->tw, sizeof(double2) * ntot, "twiddles") ||
        dalloc(h, (void **)&h->twf, sizeof(float4) * ntot, "twiddles (two-float)") ||
        dalloc(h, (void **)&h->status, sizeof(int), "status word")) {
        gw_chi0_destroy(h);
        return GW_ERR_OOM;
    }
    if (cudaMemcpy(h->tw, tw.data(), sizeof(double2) * ntot, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->twf, twf.data(), sizeof(float4) * ntot, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(h->status, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        gw_chi0_destroy(h);
        return GW_ERR_CUDA;
    }
    off = 0;
    for (int a = 0; a < 3; ++a) {
        h->ax[a].tw = h->tw + off;
        h->ax[a].twf = h->twf + off;
        off += h->d.n[a];
    }
    *out = h;
    return GW_OK;
}

int gw_chi0_streams(gw_chi0 *h, int iq)
{
    if (!h) return -(int)GW_ERR_ARG;
    gw_status s = check_slot(h, iq);
    if (s) return -(int)s;
    if (zd_route(h, iq, h->keep_m)) return 1; // the tensor-core stage (a) leaves no room beside it
    return overlap_enabled(h, pair_plan(h, h->sph[iq])) ? 2 : 1;
}

void gw_chi0_destroy(gw_chi0 *h)
{
    if (!h) return;
    cudaStreamSynchronize(h->st);
    free_bands(h, h->cond);
    for (auto &b : h->val) free_bands(h, b);
    for (auto &s : h->sph) free_sphere(h, s);
    dfree(h, h->Mbuf, h->Mcap * sizeof(double2));
    dfree(h, h->dbuf, h->dcap * sizeof(double));
    dfree(h, h->Zbuf, h->Zcap);
    dfree(h, h->spbuf, h->spcap);
    dfree(h, h->Ebuf, h->Ecap);
    dfree(h, h->jobbuf, h->jobcap);
    dfree(h, h->Mall, h->Mall_cap);
    dfree(h, h->pscr, h->pscr_cap);
    dfree(h, h->pflags, h->pflags_cap);
    dfree(h, h->EAbuf, h->EAcap);
    dfree(h, h->EBbuf, h->EBcap);
    dfree(h, h->ZBbuf, h->ZBcap);
    dfree(h, h->MBbuf, h->MBcap);
    dfree(h, h->zdA, h->zdAcap);
    dfree(h, h->zdF, h->zdFcap);
    for (int b = 0; b < 2; ++b) {
        dfree(h, h->ovZ[b], h->ovZcap[b]);
        dfree(h, h->ovE[b], h->ovEcap[b]);
        dfree(h, h->ovJ[b], h->ovJcap[b]);
        if (h->ov_split[b]) cudaEventDestroy(h->ov_split[b]);
        if (h->ov_gemm[b]) cudaEventDestroy(h->ov_gemm[b]);
    }
    if (h->ov_st) cudaStreamDestroy(h->ov_st);
    dfree(h, h->epsbuf, h->epscap);
    dfree(h, h->Mres, h->Mres_cap);
    for (auto &b : h->gpp) dfree(h, b.p, b.cap);
    dfree(h, h->realbuf, h->realcap);
    dfree(h, h->eigA, h->eigA_cap);
    dfree(h, h->eigWork, h->eigWork_cap);
    dfree(h, h->eigW, h->eigW_cap);
    dfree(h, h->eigInfo, h->eigInfo_cap);
    if (h->sol.hdl) h->sol.destroy(h->sol.hdl);
    if (h->sol.lib) dlclose(h->sol.lib);
    dfree(h, h->Dall, h->Dall_cap);
    dfree(h, h->SPall, h->SPall_cap);
    dfree(h, h->Zall, h->Zall_cap);
    dfree(h, h->Eall, h->Eall_cap);
    for (auto &g : h->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        dfree(h, g.jobs, g.jobs_bytes);
    }
    if (h->cap_st) cudaStreamDestroy(h->cap_st);
    {
        size_t ntw = (size_t)h->d.n[0] + h->d.n[1] + h->d.n[2];
        dfree(h, h->tw, sizeof(double2) * ntw);
        dfree(h, h->twf, sizeof(float4) * ntw);
    }
    dfree(h, h->status, sizeof(int));
    for (auto &r : h->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : h->pool) cudaEventDestroy(e);
    cudaGetLastError();
    delete h;
}

const char *gw_chi0_last_error(const gw_chi0 *h) { return h ? h->err.c_str() : "null handle"; }

gw_status gw_chi0_set_stream(gw_chi0 *h, void *stream)
{
    if (!h) return GW_ERR_ARG;
    h->st = (cudaStream_t)stream;
    return GW_OK;
}

gw_status gw_chi0_set_bands(gw_chi0 *h, int iq, int kind, int nb, int ngpsi, const int32_t *gvec, const double *coeff,
                            const double *energy)
{
    if (!h) return GW_ERR_ARG;
    if (kind != 0 && kind != 1) return fail(h, GW_ERR_ARG, "kind must be 0 (valence) or 1 (conduction)");
    if (kind == 0 && (iq < 0 || iq >= h->d.nq)) return fail(h, GW_ERR_ARG, "q slot %d out of range", iq);
    if (nb < 1 || ngpsi < 1) return fail(h, GW_ERR_ARG, "nb and ngpsi must be >= 1");
    if (!gvec || !coeff || !energy) return fail(h, GW_ERR_ARG, "null pointer");
    drop_graphs(h);
    BandSet nbs;
    nbs.nb = nb;
    nbs.ngpsi = ngpsi;
    nbs.g.resize((size_t)3 * ngpsi);
    nbs.e.resize(nb);
    CK(h, cudaMemcpyAsync(nbs.g.data(), gvec, sizeof(int32_t) * 3 * ngpsi, cudaMemcpyDeviceToHost, h->st), "copy gvec");
    CK(h, cudaMemcpyAsync(nbs.e.data(), energy, sizeof(double) * nb, cudaMemcpyDeviceToHost, h->st), "copy energy");
    CK(h, cudaStreamSynchronize(h->st), "set_bands sync");
    std::vector<int32_t> gofs(ngpsi);
    for (int k = 0; k < ngpsi; ++k) {
        int idx[3];
        for (int a = 0; a < 3; ++a) {
            int g = nbs.g[3 * k + a];
            if (2 * std::abs(g) >= h->d.n[a])
                return fail(h, GW_ERR_ARG, "plane wave %d: component %d outside (-n/2, n/2)", k, g);
            nbs.maxabs[a] = std::max(nbs.maxabs[a], std::abs(g));
            idx[a] = mod(g, h->d.n[a]);
        }
        gofs[k] = (idx[0] * h->d.n[1] + idx[1]) * h->d.n[2] + idx[2];
    }
    for (double e : nbs.e)
        if (!std::isfinite(e)) return fail(h, GW_ERR_ARG, "non-finite band energy");
    // energy ordering against the other set, when present
    const BandSet *other = nullptr;
    if (kind == 0 && h->cond.nb) other = &h->cond;
    if (other) {
        double vmax = *std::max_element(nbs.e.begin(), nbs.e.end());
        double cmin = *std::min_element(other->e.begin(), other->e.end());
        if (!(vmax < cmin)) return fail(h, GW_ERR_ARG, "a valence energy is not below every conduction energy");
    }
    if (kind == 1) {
        double cmin = *std::min_element(nbs.e.begin(), nbs.e.end());
        for (auto &v : h->val)
            if (v.nb && !(*std::max_element(v.e.begin(), v.e.end()) < cmin))
                return fail(h, GW_ERR_ARG, "a valence energy is not below every conduction energy");
    }
    if (kind == 1 || iq == h->Mres_iq) h->Mres_iq = -1; // resident pair elements no longer match
    BandSet &dst = kind == 0 ? h->val[iq] : h->cond;
    if (dst.nb == nb && dst.ngpsi == ngpsi) {
        // same shape: reuse the device buffers (no allocation on repeated setup)
        nbs.psi = dst.psi;
        nbs.energy = dst.energy;
        nbs.gvec = dst.gvec;
        nbs.gofs = dst.gofs;
        dst.psi = nullptr;
        dst.energy = nullptr;
        dst.gvec = nullptr;
        dst.gofs = nullptr;
        dst = BandSet();
    } else {
        free_bands(h, dst);
        gw_status s;
        if ((s = dalloc(h, (void **)&nbs.psi, sizeof(double2) * (size_t)nb * h->nr, "psi grids")) ||
            (s = dalloc(h, (void **)&nbs.energy, sizeof(double) * nb, "energies")) ||
            (s = dalloc(h, (void **)&nbs.gvec, sizeof(int32_t) * 3 * ngpsi, "gvec")) ||
            (s = dalloc(h, (void **)&nbs.gofs, sizeof(int32_t) * ngpsi, "grid offsets"))) {
            free_bands(h, nbs);
            return s;
        }
    }
    CK(h, cudaMemcpyAsync(nbs.energy, energy, sizeof(double) * nb, cudaMemcpyDeviceToDevice, h->st), "energies");
    CK(h, cudaMemcpyAsync(nbs.gvec, gvec, sizeof(int32_t) * 3 * ngpsi, cudaMemcpyDeviceToDevice, h->st), "gvec");
    CK(h, cudaMemcpyAsync(nbs.gofs, gofs.data(), sizeof(int32_t) * ngpsi, cudaMemcpyHostToDevice, h->st), "gofs");
    CK(h, cudaMemsetAsync(nbs.psi, 0, sizeof(double2) * (size_t)nb * h->nr, h->st), "zero psi");
    if (h->d.mtxel_prec == GW_MTXEL_TWOFLOAT) {
        Scope sc(h, "band_setup_tf");
        CK(h, gw::launch_band_setup_tf((const double2 *)coeff, nbs.gofs, nb, ngpsi, nbs.psi, h->d.n, h->ax,
                                       nbs.maxabs, h->st),
           "band setup (two-float)"); // three kernels
    } else {
        {
            Scope sc(h, "band_scatter");
            CK(h, gw::launch_scatter((const double2 *)coeff, nbs.gofs, nb, ngpsi, h->nr, nbs.psi, h->st), "scatter");
        }
        Scope sc(h, "band_fft");
        CK(h, gw::launch_band_fft(nbs.psi, nb, h->d.n, h->ax, h->st), "band fft"); // two kernels
    }
    CK(h, cudaStreamSynchronize(h->st), "set_bands sync"); // gofs host vector goes out of scope
    dst = std::move(nbs);
    return GW_OK;
}

gw_status gw_chi0_set_gsphere(gw_chi0 *h, int iq, int ng, const int32_t *gvec)
{
    if (!h) return GW_ERR_ARG;
    if (iq < 0 || iq >= h->d.nq) return fail(h, GW_ERR_ARG, "q slot %d out of range", iq);
    if (ng < 1) return fail(h, GW_ERR_ARG, "ng must be >= 1");
    if (ng > gw::pair_max_ng()) return fail(h, GW_ERR_UNSUPPORTED, "ng = %d exceeds %d", ng, gw::pair_max_ng());
    if (!gvec) return fail(h, GW_ERR_ARG, "null pointer");
    drop_graphs(h);
    Sphere s;
    s.ng = ng;
    s.g.resize((size_t)3 * ng);
    CK(h, cudaMemcpyAsync(s.g.data(), gvec, sizeof(int32_t) * 3 * ng, cudaMemcpyDeviceToHost, h->st), "copy sphere");
    CK(h, cudaStreamSynchronize(h->st), "set_gsphere sync");
    for (int i = 0; i < ng; ++i)
        for (int a = 0; a < 3; ++a) {
            int g = s.g[3 * i + a];
            if (2 * std::abs(g) >= h->d.n[a]) return fail(h, GW_ERR_ARG, "G %d: component %d outside (-n/2, n/2)", i, g);
            s.maxabs[a] = std::max(s.maxabs[a], std::abs(g));
        }
    gw::SpherePlanHost plan;
    gw::build_sphere_plan(h->d.n, ng, s.g.data(), plan);
    // alias check against whatever bands are already stored
    int ax;
    if (h->val[iq].nb && h->cond.nb && !alias_free(h, h->val[iq], h->cond, s, &ax))
        return fail(h, GW_ERR_ARG, "max|K_v| + max|K_c| + max|G| >= n on axis %d (aliasing)", ax);
    s.K2 = plan.K2;
    s.K12 = plan.K12;
    s.cstart = plan.cstart;
    s.cg = plan.cg;
    const std::vector<int> &kz = plan.kz;
    const std::vector<int32_t> &pack = plan.pack, &cell = plan.cell;
    std::vector<int2> cpts(ng);
    for (int m = 0; m < ng; ++m) cpts[m] = make_int2(plan.cpts[m].first, plan.cpts[m].second);
    gw_status st;
    if (iq == h->Mres_iq) h->Mres_iq = -1; // resident pair elements no longer match
    Sphere &old = h->sph[iq];
    if (old.ng == ng && old.K2 == s.K2 && old.K12 == s.K12) {
        s.kz = old.kz;
        s.gpack = old.gpack;
        s.gvec = old.gvec;
        s.cell = old.cell;
        s.cstart_d = old.cstart_d;
        s.cpts = old.cpts;
        old.kz = nullptr;
        old.gpack = nullptr;
        old.gvec = nullptr;
        old.cell = nullptr;
        old.cstart_d = nullptr;
        old.cpts = nullptr;
        old = Sphere();
    } else if ((st = dalloc(h, (void **)&s.kz, sizeof(int) * s.K2, "sphere kz")) ||
        (st = dalloc(h, (void **)&s.gpack, sizeof(int32_t) * ng, "sphere pack")) ||
        (st = dalloc(h, (void **)&s.gvec, sizeof(int32_t) * 3 * ng, "sphere gvec")) ||
        (st = dalloc(h, (void **)&s.cell, sizeof(int32_t) * s.K12, "sphere cells")) ||
        (st = dalloc(h, (void **)&s.cstart_d, sizeof(int) * (s.K12 + 1), "sphere cell starts")) ||
        (st = dalloc(h, (void **)&s.cpts, sizeof(int2) * ng, "sphere points by cell"))) {
        free_sphere(h, s);
        return st;
    }
    CK(h, cudaMemcpyAsync(s.kz, kz.data(), sizeof(int) * s.K2, cudaMemcpyHostToDevice, h->st), "kz");
    CK(h, cudaMemcpyAsync(s.gpack, pack.data(), sizeof(int32_t) * ng, cudaMemcpyHostToDevice, h->st), "pack");
    CK(h, cudaMemcpyAsync(s.cell, cell.data(), sizeof(int32_t) * s.K12, cudaMemcpyHostToDevice, h->st), "cells");
    CK(h, cudaMemcpyAsync(s.cstart_d, s.cstart.data(), sizeof(int) * (s.K12 + 1), cudaMemcpyHostToDevice, h->st),
       "cell starts");
    CK(h, cudaMemcpyAsync(s.cpts, cpts.data(), sizeof(int2) * ng, cudaMemcpyHostToDevice, h->st), "cell points");
    CK(h, cudaMemcpyAsync(s.gvec, gvec, sizeof(int32_t) * 3 * ng, cudaMemcpyDeviceToDevice, h->st), "gvec");
    if (h->d.mtxel_prec == GW_MTXEL_TWOFLOAT) {
        // scratch slots of the grid-specialised two-float pair kernel for this sphere
        size_t elems = 0;
        CK(h, gw::pair_tf_scratch(pair_plan(h, s), &s.nslots, &elems), "pair scratch size");
        if (s.nslots > 0) {
            if ((st = grow(h, (void **)&h->pscr, &h->pscr_cap, sizeof(float4) * elems * s.nslots, "pair scratch")) ||
                (st = grow(h, (void **)&h->pflags, &h->pflags_cap, sizeof(int) * s.nslots, "pair scratch flags"))) {
                free_sphere(h, s);
                return st;
            }
        }
    }
    CK(h, cudaStreamSynchronize(h->st), "set_gsphere sync");
    free_sphere(h, h->sph[iq]);
    h->sph[iq] = std::move(s);
    return GW_OK;
}

gw_status gw_chi0_pair_elements_block(gw_chi0 *h, int iq, int c0, int cb, double *M)
{
    if (!h) return GW_ERR_ARG;
    gw_status s = check_slot(h, iq);
    if (s) return s;
    if (c0 < 0 || cb < 0 || c0 + cb > h->cond.nb)
        return fail(h, GW_ERR_ARG, "conduction block [%d, %d) outside [0, %d)", c0, c0 + cb, h->cond.nb);
    if (cb && !M) return fail(h, GW_ERR_ARG, "null M");
    if (!zd_route(h, iq, h->keep_m)) return fail(h, GW_ERR_UNSUPPORTED, "slot %d does not take the tensor-core route", iq);
    if (cb == 0) return GW_OK;
    const int nv = h->val[iq].nb, cbmax = zd_chunk_bands(h, iq);
    CUtensorMap tmA, tmC;
    if ((s = zd_prepare(h, iq, &tmA, &tmC))) return s;
    const gw::PairPlan pp = pair_plan(h, h->sph[iq]);
    const int ng = h->sph[iq].ng;
    for (int b0 = 0; b0 < cb; b0 += cbmax) {
        const int n = std::min(cbmax, cb - b0);
        if ((s = zd_stage_a(h, iq, tmA, tmC, c0 + b0, n, pp, (double2 *)M + (int64_t)b0 * nv * ng))) return s;
    }
    return GW_OK;
}

gw_status gw_chi0_pair_elements(gw_chi0 *h, int iq, int64_t pair_begin, int64_t pair_count, double *M)
{
    if (!h) return GW_ERR_ARG;
    gw_status s = check_slot(h, iq);
    if (s) return s;
    const BandSet &v = h->val[iq];
    int64_t P = (int64_t)v.nb * h->cond.nb;
    if (pair_begin < 0 || pair_count < 0 || pair_begin + pair_count > P)
        return fail(h, GW_ERR_ARG, "pair range [%lld, %lld) outside [0, %lld)", (long long)pair_begin,
                    (long long)(pair_begin + pair_count), (long long)P);
    if (pair_count && !M) return fail(h, GW_ERR_ARG, "null M");
    Scope sc(h, "pair_mtxel");
    CK(h, run_pair(h, v.psi, h->cond.psi, h->cond.nb, pair_begin, pair_count, pair_plan(h, h->sph[iq]),
                   (double2 *)M),
       "pair kernel");
    return GW_OK;
}

gw_status gw_chi0_compute(gw_chi0 *h, int nq, const int *iq, int nw, const double *omega, double *chi, double *diag)
{
    if (!h) return GW_ERR_ARG;
    if (nq < 1 || !iq || nw < 1 || nw > gw::kMaxOmega || !omega || !chi)
        return fail(h, GW_ERR_ARG, "bad arguments (nq >= 1, 1 <= nw <= %d, non-null pointers)", gw::kMaxOmega);
    gw::OmegaList om;
    om.nw = nw;
    for (int i = 0; i < nw; ++i) {
        if (!(omega[i] >= 0.0) || !std::isfinite(omega[i])) return fail(h, GW_ERR_ARG, "omega must be finite and >= 0");
        om.w[i] = omega[i];
    }
    for (int i = 0; i < nq; ++i) {
        gw_status s = check_slot(h, iq[i]);
        if (s) return s;
    }
    size_t off = 0, doff = 0;
    for (int i = 0; i < nq; ++i) {
        const Sphere &sp = h->sph[iq[i]];
        const BandSet &v = h->val[iq[i]];
        const int ng = sp.ng;
        const int64_t P = (int64_t)v.nb * h->cond.nb;
        const int64_t chunk = std::min<int64_t>(h->d.pair_chunk, P);
        double2 *cq = (double2 *)chi + off;
        double *dq = diag ? diag + doff : nullptr;
        CK(h, cudaMemsetAsync(cq, 0, sizeof(double2) * (size_t)nw * ng * ng, h->st), "zero chi");
        if (dq) CK(h, cudaMemsetAsync(dq, 0, sizeof(double) * (size_t)nw * ng, h->st), "zero diag");
        gw::PairPlan pp = pair_plan(h, sp);
        bool keep = false;
        gw_status s = resident_begin(h, P, ng, &keep);
        if (s) return s;
        double2 *Mres = keep ? h->Mres : nullptr;
        // one frequency: a chunk's contraction is about as long as the next chunk's pair elements
        // and hides behind them; with more, the contractions (the shallow-ring variant) queue up
        // behind the two slice buffers and the single stream is faster
        if (nw == 1 && overlap_enabled(h, pp) && fault_chunk() < 0 && !zd_route(h, iq[i], keep)) {
            s = compute_overlap(h, iq[i], om, cq, dq, Mres);
            if (s) return s;
            Scope sc(h, "symmetrize");
            CK(h, gw::launch_symmetrize(cq, ng, nw, h->st), "symmetrize");
            off += (size_t)nw * ng * ng;
            doff += (size_t)nw * ng;
            if (keep) h->Mres_iq = iq[i];
            continue;
        }
        if (zd_route(h, iq[i], keep) && fault_chunk() < 0) {
            const int nv = v.nb, cb = zd_chunk_bands(h, iq[i]);
            s = ensure_work(h, (size_t)nv * cb * ng, (size_t)nv * cb * nw);
            if (s) return s;
            CUtensorMap tmA, tmC;
            if ((s = zd_prepare(h, iq[i], &tmA, &tmC))) return s;
            for (int c0 = 0; c0 < h->cond.nb; c0 += cb) {
                const int cbc = std::min(cb, h->cond.nb - c0);
                const int64_t cnt = (int64_t)nv * cbc;
                if ((s = zd_stage_a(h, iq[i], tmA, tmC, c0, cbc, pp, h->Mbuf))) return s;
                {
                    Scope sc(h, "delta");
                    CK(h, gw::launch_delta_block(v.energy, h->cond.energy, nv, c0, cbc, om, h->dbuf, h->st), "delta");
                }
                if ((s = contract_chunk(h, h->Mbuf, cnt, ng, h->dbuf, cnt, nw, cq))) return s;
                if (dq) {
                    Scope sc(h, "diag");
                    CK(h, gw::launch_diag(h->Mbuf, cnt, ng, h->dbuf, cnt, nw, dq, ng, h->st), "diag");
                }
            }
            Scope sc(h, "symmetrize");
            CK(h, gw::launch_symmetrize(cq, ng, nw, h->st), "symmetrize");
            off += (size_t)nw * ng * ng;
            doff += (size_t)nw * ng;
            continue;
        }
        s = ensure_work(h, (size_t)chunk * ng, (size_t)chunk * nw);
        if (s) return s;
        const int64_t fault_at = fault_chunk();
        for (int64_t p0 = 0, k = 0; p0 < P; p0 += chunk, ++k) {
            int64_t cnt = std::min(chunk, P - p0);
            if (k == fault_at) return fail(h, GW_ERR_CUDA, "injected host-side fault before chunk %lld", (long long)k);
            double2 *Mc = Mres ? Mres + p0 * ng : h->Mbuf;
            {
                Scope sc(h, "pair_mtxel");
                CK(h, run_pair(h, v.psi, h->cond.psi, h->cond.nb, p0, cnt, pp, Mc), "pair kernel");
            }
            {
                Scope sc(h, "delta");
                CK(h, gw::launch_delta(v.energy, h->cond.energy, h->cond.nb, p0, cnt, om, h->dbuf, h->st), "delta");
            }
            s = contract_chunk(h, Mc, cnt, ng, h->dbuf, cnt, nw, cq);
            if (s) return s;
            if (dq) {
                Scope sc(h, "diag");
                CK(h, gw::launch_diag(Mc, cnt, ng, h->dbuf, cnt, nw, dq, ng, h->st), "diag");
            }
        }
        {
            Scope sc(h, "symmetrize");
            CK(h, gw::launch_symmetrize(cq, ng, nw, h->st), "symmetrize");
        }
        off += (size_t)nw * ng * ng;
        doff += (size_t)nw * ng;
        if (keep) h->Mres_iq = iq[i];
    }
    return GW_OK;
}

gw_status gw_chi0_keep_pair_elements(gw_chi0 *h, int enable)
{
    if (!h) return GW_ERR_ARG;
    if (enable != 0 && enable != 1) return fail(h, GW_ERR_ARG, "enable must be 0 or 1");
    h->keep_m = enable == 1;
    h->Mres_iq = -1;
    if (!h->keep_m && h->Mres) {
        CK(h, cudaStreamSynchronize(h->st), "release resident pair elements");
        dfree(h, h->Mres, h->Mres_cap);
        h->Mres = nullptr;
        h->Mres_cap = 0;
    }
    return GW_OK;
}

gw_status gw_chi0_compute_batch(gw_chi0 *h, int nq, const int *iq, int nw, const double *omega, double *chi,
                                double *diag)
{
    if (!h) return GW_ERR_ARG;
    if (nq < 1 || !iq || nw < 1 || nw > gw::kMaxOmega || !omega || !chi)
        return fail(h, GW_ERR_ARG, "bad arguments (nq >= 1, 1 <= nw <= %d, non-null pointers)", gw::kMaxOmega);
    gw::OmegaList om;
    om.nw = nw;
    for (int i = 0; i < nw; ++i) {
        if (!(omega[i] >= 0.0) || !std::isfinite(omega[i])) return fail(h, GW_ERR_ARG, "omega must be finite and >= 0");
        om.w[i] = omega[i];
    }
    for (int i = 0; i < nq; ++i) {
        gw_status s = check_slot(h, iq[i]);
        if (s) return s;
        for (int j = 0; j < i; ++j)
            if (iq[j] == iq[i]) return fail(h, GW_ERR_ARG, "slot %d requested twice", iq[i]);
    }
    return compute_batch(h, nq, iq, nw, omega, om, chi, diag);
}

int gw_chi0_tuning(const gw_chi0 *h, int *tile_f64, int *waves_f64, int *tile_split)
{
    if (!h) return 0;
    if (tile_f64) *tile_f64 = h->tuned_bt;
    if (waves_f64) *waves_f64 = h->tuned_waves;
    if (tile_split) *tile_split = h->tuned_bn;
    return (int)h->tune_cache.size();
}

gw_status gw_chi0_contract(gw_chi0 *h, int nv, int nc, const double *ev, const double *ec, int ng, const double *M,
                           int nw, const double *omega, double *chi)
{
    if (!h) return GW_ERR_ARG;
    if (nv < 1 || nc < 1 || ng < 1 || nw < 1 || nw > gw::kMaxOmega || !ev || !ec || !M || !omega || !chi)
        return fail(h, GW_ERR_ARG, "bad arguments");
    gw::OmegaList om;
    om.nw = nw;
    for (int i = 0; i < nw; ++i) {
        if (!(omega[i] >= 0.0) || !std::isfinite(omega[i])) return fail(h, GW_ERR_ARG, "omega must be finite and >= 0");
        om.w[i] = omega[i];
    }
    const int64_t P = (int64_t)nv * nc;
    {
        std::vector<double> hv(nv), hc(nc);
        CK(h, cudaMemcpyAsync(hv.data(), ev, sizeof(double) * nv, cudaMemcpyDeviceToHost, h->st), "copy ev");
        CK(h, cudaMemcpyAsync(hc.data(), ec, sizeof(double) * nc, cudaMemcpyDeviceToHost, h->st), "copy ec");
        CK(h, cudaStreamSynchronize(h->st), "contract sync");
        if (!(*std::max_element(hv.begin(), hv.end()) < *std::min_element(hc.begin(), hc.end())))
            return fail(h, GW_ERR_ARG, "a valence energy is not below every conduction energy");
    }
    const int64_t chunk = std::min<int64_t>(h->d.pair_chunk, P);
    gw_status s = ensure_work(h, 0, (size_t)chunk * nw);
    if (s) return s;
    CK(h, cudaMemsetAsync(chi, 0, sizeof(double2) * (size_t)nw * ng * ng, h->st), "zero chi");
    for (int64_t p0 = 0; p0 < P; p0 += chunk) {
        const int64_t cnt = std::min(chunk, P - p0);
        {
            Scope sc(h, "delta");
            CK(h, gw::launch_delta(ev, ec, nc, p0, cnt, om, h->dbuf, h->st), "delta");
        }
        s = contract_chunk(h, (const double2 *)M + p0 * ng, cnt, ng, h->dbuf, cnt, nw, (double2 *)chi);
        if (s) return s;
    }
    Scope sc(h, "symmetrize");
    CK(h, gw::launch_symmetrize((double2 *)chi, ng, nw, h->st), "symmetrize");
    return GW_OK;
}

gw_status gw_chi0_sync(gw_chi0 *h)
{
    if (!h) return GW_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->st), "sync");
    int st = 0;
    CK(h, cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost), "status");
    CK(h, cudaMemset(h->status, 0, sizeof(int)), "status reset");
    if (st & gw::kStatusTimeout) return fail(h, GW_ERR_TIMEOUT, "a bounded device-side wait gave up");
    if (st & gw::kStatusNoSlot) return fail(h, GW_ERR_CUDA, "a pair block found no free scratch slot");
    if (st & gw::kStatusBounds) return fail(h, GW_ERR_CUDA, "an index outside its buffer (bounds-checked build)");
    return GW_OK;
}

gw_status gw_chi0_check_watchdog(gw_chi0 *h, long long iterations)
{
    if (!h) return GW_ERR_ARG;
    if (iterations < 1) return fail(h, GW_ERR_ARG, "iterations must be >= 1");
    CK(h, gw::launch_watchdog(iterations, h->status, h->st), "watchdog");
    return GW_OK;
}

gw_status gw_chi0_set_timing(gw_chi0 *h, int enable)
{
    if (!h) return GW_ERR_ARG;
    h->timing = enable != 0;
    return GW_OK;
}

int gw_chi0_timing(gw_chi0 *h, int n, char (*names)[32], double *ms, int64_t *launches, int reset)
{
    if (!h) return 0;
    drain_timing(h);
    int i = 0;
    for (auto &kv : h->acc) {
        if (i < n) {
            if (names) {
                std::strncpy(names[i], kv.first.c_str(), 31);
                names[i][31] = 0;
            }
            if (ms) ms[i] = kv.second.first;
            if (launches) launches[i] = kv.second.second;
        }
        ++i;
    }
    if (reset) h->acc.clear();
    return i;
}

size_t gw_chi0_device_bytes(const gw_chi0 *h) { return h ? h->bytes : 0; }

} // extern "C"

