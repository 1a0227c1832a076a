// Host side of the C ABI declared in include/gw_chi0.h: handle state, validation,
// library-owned device memory, per-chunk orchestration and optional per-kernel timing.
#include "../../include/gw_chi0.h"
#include "internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cusolverDn.h>
#include <dlfcn.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <array>
#include <map>
#include <string>
#include <vector>

using gw::FftAxis;

namespace {

struct BandSet {
    int nb = 0, ngpsi = 0;
    double2 *psi = nullptr;     // [nb][N_r]
    double *energy = nullptr;   // [nb] device copy
    int32_t *gvec = nullptr;    // [ngpsi][3] device copy (adjoint)
    int32_t *gofs = nullptr;    // [ngpsi] grid offsets
    std::vector<int32_t> g;     // host copy
    std::vector<double> e;      // host copy
    int maxabs[3] = {0, 0, 0};
};

struct Sphere {
    int ng = 0;
    std::vector<int32_t> g;
    int maxabs[3] = {0, 0, 0};
    int K2 = 0;
    int *kz = nullptr;          // device [K2]
    int32_t *gpack = nullptr;   // device [ng]
    int32_t *gvec = nullptr;    // device [ng][3]
    std::vector<int> cstart, cg; // (k1, k2) cells of the sphere, CSR (adjoint back-projection)
    int K12 = 0;                // number of cells
    int32_t *cell = nullptr;    // device [K12]  k2index << 8 | k1
    int *cstart_d = nullptr;    // device [K12 + 1] (cstart)
    int2 *cpts = nullptr;       // device [ng]   (point, k0 | cell << 8) in cell order
    int nslots = 0;             // scratch slots the two-float pair kernel needs (0: none)
};

struct TimerRec {
    std::string name;
    cudaEvent_t a, b;
};

} // namespace

struct gw_chi0 {
    gw_chi0_desc d{};
    cudaStream_t st = nullptr;
    std::string err;
    int64_t nr = 0;
    FftAxis ax[3]{};
    double2 *tw = nullptr;
    float4 *twf = nullptr;
    BandSet cond;
    std::vector<BandSet> val;
    std::vector<Sphere> sph;
    double2 *Mbuf = nullptr;
    size_t Mcap = 0; // elements
    double *dbuf = nullptr;
    size_t dcap = 0;
    // split-precision work buffers
    void *Zbuf = nullptr;      // bf16 slices [s][2 ng][kpad]
    size_t Zcap = 0;           // bytes
    double *spbuf = nullptr;   // sqrt(-Delta) [nw][chunk]
    size_t spcap = 0;
    int *Ebuf = nullptr;       // column exponents [ng]
    size_t Ecap = 0;
    void *jobbuf = nullptr;    // job tables of the batched contraction kernels
    size_t jobcap = 0;
    // contraction launch shapes (set by the autotuner; these are the defaults)
    int tuned_bt = 64, tuned_waves = 4, tuned_bn = 256;
    std::map<std::string, std::array<int, 3>> tune_cache; // signature -> (bt, waves, bn)
    // batched path: every slot's M resident, one graph per call signature
    double2 *Mall = nullptr;
    size_t Mall_cap = 0;
    double *Dall = nullptr, *SPall = nullptr;
    size_t Dall_cap = 0, SPall_cap = 0;
    void *Zall = nullptr;
    size_t Zall_cap = 0;
    int *Eall = nullptr;
    size_t Eall_cap = 0;
    cudaStream_t cap_st = nullptr;
    struct Graph {
        std::string key;
        cudaGraphExec_t exec = nullptr;
        void *jobs = nullptr;
        size_t jobs_bytes = 0;
    };
    std::vector<Graph> graphs;
    int *status = nullptr;
    // split-precision general products (subspace projection, adjoint Y = M W)
    int *EAbuf = nullptr, *EBbuf = nullptr;
    size_t EAcap = 0, EBcap = 0;
    void *ZBbuf = nullptr;      // B operand slices [s][2 nout][kpad]
    size_t ZBcap = 0;
    double2 *MBbuf = nullptr;   // projected pair elements of a chunk [chunk][neig]
    size_t MBcap = 0;
    void *epsbuf = nullptr;     // dielectric inverse: A, X, T, P [ng][ng], sqrt(v) [ng], bound
    size_t epscap = 0;
    double2 *realbuf = nullptr; // real-axis chi: the three Hermitian parts per frequency
    size_t realcap = 0;
    // dense eigensolver (cuSOLVER, loaded on first use) for the subspace basis
    struct {
        void *lib = nullptr;
        cusolverDnHandle_t hdl = nullptr;
        decltype(&cusolverDnCreate) create = nullptr;
        decltype(&cusolverDnDestroy) destroy = nullptr;
        decltype(&cusolverDnSetStream) set_stream = nullptr;
        decltype(&cusolverDnZheevdx_bufferSize) buffer_size = nullptr;
        decltype(&cusolverDnZheevdx) heevdx = nullptr;
    } sol;
    double2 *eigA = nullptr, *eigWork = nullptr;
    double *eigW = nullptr;
    int *eigInfo = nullptr;
    size_t eigA_cap = 0, eigWork_cap = 0, eigW_cap = 0, eigInfo_cap = 0;
    // scratch slots of the two-float pair kernel (sized in set_gsphere, outside any capture)
    float4 *pscr = nullptr;
    size_t pscr_cap = 0; // bytes
    int *pflags = nullptr;
    size_t pflags_cap = 0; // bytes
    size_t bytes = 0;
    PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    // timing
    bool timing = false;
    std::vector<TimerRec> pending;
    std::vector<cudaEvent_t> pool;
    std::map<std::string, std::pair<double, int64_t>> acc;
};

namespace {

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

#define CK(h, x, what)                                   \
    do {                                                 \
        cudaError_t e_ = (x);                            \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    } while (0)

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

struct Scope {
    gw_chi0 *h;
    const char *name;
    cudaEvent_t a = nullptr;
    Scope(gw_chi0 *h_, const char *n) : h(h_), name(n)
    {
        if (h->timing) {
            a = ev_get(h);
            cudaEventRecord(a, h->st);
        }
    }
    ~Scope()
    {
        if (h->timing) {
            cudaEvent_t b = ev_get(h);
            cudaEventRecord(b, h->st);
            h->pending.push_back({name, a, b});
        }
    }
};

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
    gw_status st;
    if ((st = grow(h, &h->Zbuf, &h->Zcap, (size_t)s * 2 * ng * kpad * 2, "slice buffer")) ||
        (st = grow(h, (void **)&h->spbuf, &h->spcap, sizeof(double) * (size_t)nw * dstride, "scale buffer")) ||
        (st = grow(h, (void **)&h->Ebuf, &h->Ecap, sizeof(int) * (size_t)ng, "exponent buffer")))
        return st;
    {
        Scope sc(h, "oz_split");
        CK(h, gw::launch_oz_sqrt(delta, (int64_t)nw * dstride, h->spbuf, h->st), "oz sqrt");
    }
    const int bn = h->tuned_bn;
    for (int w = 0; w < nw; ++w) {
        const double *sp = h->spbuf + (int64_t)w * dstride;
        {
            Scope sc(h, "oz_split");
            CK(h, gw::launch_oz_colexp(M, P, ng, sp, h->Ebuf, h->st), "oz exponents");
            CK(h, gw::launch_oz_slice(M, P, ng, sp, h->Ebuf, s, kpad, h->Zbuf, h->st), "oz slices");
        }
        std::vector<gw::OzJob> jobs(1);
        if ((st = oz_job(h, jobs[0], h->Zbuf, kpad, ng, h->Ebuf, chi + (int64_t)w * ng * ng, bn))) return st;
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
gw_status oz_prepare_b(gw_chi0 *h, const double2 *B, int ka, int nout)
{
    const int s = h->d.nslices;
    const int64_t kpad = oz_kpad(ka);
    gw_status st;
    if ((st = grow(h, &h->ZBbuf, &h->ZBcap, (size_t)s * 2 * nout * kpad * 2, "product operand slices")) ||
        (st = grow(h, (void **)&h->EBbuf, &h->EBcap, sizeof(int) * (size_t)nout, "product operand exponents")))
        return st;
    CK(h, gw::launch_oz_split_cols(B, ka, nout, s, kpad, h->ZBbuf, h->EBbuf, h->st), "oz column slices");
    return GW_OK;
}

// Y[rows][nout] = A[rows][ka] B[ka][nout] (complex, row-major) in split precision, B prepared
// by oz_prepare_b.  A's slices reuse the contraction's slice buffer (stream order separates
// the two uses).
gw_status oz_product(gw_chi0 *h, const double2 *A, int64_t rows, int ka, int nout, double2 *Y)
{
    const int s = h->d.nslices;
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


// ------------------------------------------------------------------ batched path (many q, many w)
// Every requested slot's M is produced once and kept resident; the contraction of all
// (q, w) blocks then runs as one persistent launch (FP64) or one persistent launch per
// frequency over all slots (split precision).  The whole sequence is captured once per
// call signature into a CUDA graph and replayed.  Launch shapes come from a small
// autotuner that times the candidates on the first call of a signature.
struct BatchLayout {
    std::vector<int64_t> P, moff, doff, coff, dgoff;
    std::vector<int> ng;
    // split precision: pair segments of at most pair_chunk pairs, each with its own
    // column exponents and slices (the exactness bound of the slice sums is per segment)
    struct Seg {
        int q;
        int64_t p0, cnt, kpad, zoff, eoff;
    };
    std::vector<Seg> seg;
    size_t Mtot = 0, Dtot = 0, Ztot = 0, Etot = 0;
};

BatchLayout batch_layout(gw_chi0 *h, int nq, const int *iq, int nw)
{
    BatchLayout L;
    size_t coff = 0, dgoff = 0;
    const int64_t kseg = h->d.pair_chunk;
    for (int i = 0; i < nq; ++i) {
        const int ng = h->sph[iq[i]].ng;
        const int64_t P = (int64_t)h->val[iq[i]].nb * h->cond.nb;
        L.ng.push_back(ng);
        L.P.push_back(P);
        L.moff.push_back((int64_t)L.Mtot);
        L.doff.push_back((int64_t)L.Dtot);
        L.coff.push_back((int64_t)coff);
        L.dgoff.push_back((int64_t)dgoff);
        L.Mtot += (size_t)P * ng;
        L.Dtot += (size_t)nw * P;
        coff += (size_t)nw * ng * ng;
        dgoff += (size_t)nw * ng;
        for (int64_t p0 = 0; p0 < P; p0 += kseg) {
            BatchLayout::Seg sg;
            sg.q = i;
            sg.p0 = p0;
            sg.cnt = std::min(kseg, P - p0);
            sg.kpad = (sg.cnt + 63) / 64 * 64;
            sg.zoff = (int64_t)L.Ztot;
            sg.eoff = (int64_t)L.Etot;
            L.Ztot += (size_t)h->d.nslices * 2 * ng * sg.kpad;
            L.Etot += (size_t)ng;
            L.seg.push_back(sg);
        }
    }
    return L;
}

std::string batch_key(gw_chi0 *h, int nq, const int *iq, int nw, const double *omega, const void *chi,
                      const void *diag)
{
    std::string k = "p" + std::to_string(h->d.prec) + "s" + std::to_string(h->d.nslices) + "m" +
                    std::to_string(h->d.mtxel_prec) + "|";
    char buf[64];
    for (int i = 0; i < nq; ++i) k += std::to_string(iq[i]) + ":" + std::to_string(h->sph[iq[i]].ng) + ",";
    k += "|";
    for (int i = 0; i < nw; ++i) {
        snprintf(buf, sizeof buf, "%a,", omega[i]);
        k += buf;
    }
    snprintf(buf, sizeof buf, "|%p|%p", chi, diag);
    return k + buf;
}

std::string tune_key(gw_chi0 *h, const BatchLayout &L, int nw)
{
    std::string k = "p" + std::to_string(h->d.prec) + "s" + std::to_string(h->d.nslices) + "w" + std::to_string(nw);
    for (size_t i = 0; i < L.ng.size(); ++i) k += "," + std::to_string(L.ng[i]) + "x" + std::to_string(L.P[i]);
    return k;
}

// Enqueue the producer stages: pair elements of every slot, Delta, and (split precision)
// the square roots.  The slices depend on the frequency and are enqueued per frequency.
gw_status batch_stage_a(gw_chi0 *h, int nq, const int *iq, const gw::OmegaList &om, const BatchLayout &L)
{
    for (int i = 0; i < nq; ++i) {
        const BandSet &v = h->val[iq[i]];
        gw::PairPlan pp = pair_plan(h, h->sph[iq[i]]);
        {
            Scope sc(h, "pair_mtxel");
            CK(h, run_pair(h, v.psi, h->cond.psi, h->cond.nb, 0, L.P[i], pp, h->Mall + L.moff[i]), "pair kernel");
        }
        Scope sc(h, "delta");
        CK(h, gw::launch_delta(v.energy, h->cond.energy, h->cond.nb, 0, L.P[i], om, h->Dall + L.doff[i], h->st),
           "delta");
    }
    if (h->d.prec == GW_PREC_OZAKI_BF16) {
        Scope sc(h, "oz_split");
        CK(h, gw::launch_oz_sqrt(h->Dall, (int64_t)L.Dtot, h->SPall, h->st), "oz sqrt");
    }
    return GW_OK;
}

gw_status batch_oz_split(gw_chi0 *h, int nq, int w, const BatchLayout &L)
{
    (void)nq;
    Scope sc(h, "oz_split");
    for (const auto &sg : L.seg) {
        const int ng = L.ng[sg.q];
        const double *sp = h->SPall + L.doff[sg.q] + (int64_t)w * L.P[sg.q] + sg.p0;
        const double2 *M = h->Mall + L.moff[sg.q] + sg.p0 * ng;
        CK(h, gw::launch_oz_colexp(M, sg.cnt, ng, sp, h->Eall + sg.eoff, h->st), "oz exponents");
        CK(h, gw::launch_oz_slice(M, sg.cnt, ng, sp, h->Eall + sg.eoff, h->d.nslices, sg.kpad,
                                  (uint16_t *)h->Zall + sg.zoff, h->st),
           "oz slices");
    }
    return GW_OK;
}

gw_status batch_f64_jobs(gw_chi0 *h, int nq, int nw, const BatchLayout &L, double2 *chi, int bt,
                         std::vector<gw::F64Job> &jobs)
{
    jobs.clear();
    for (int i = 0; i < nq; ++i) {
        gw_status s = f64_jobs(h, jobs, h->Mall + L.moff[i], L.P[i], L.ng[i], h->Dall + L.doff[i], L.P[i], nw,
                               chi + L.coff[i], bt);
        if (s) return s;
    }
    return GW_OK;
}

gw_status batch_oz_jobs(gw_chi0 *h, int nq, int w, const BatchLayout &L, double2 *chi, int bn,
                        std::vector<gw::OzJob> &jobs)
{
    (void)nq;
    jobs.clear();
    for (const auto &sg : L.seg) {
        const int ng = L.ng[sg.q];
        gw::OzJob j;
        gw_status s = oz_job(h, j, (uint16_t *)h->Zall + sg.zoff, sg.kpad, ng, h->Eall + sg.eoff,
                             chi + L.coff[sg.q] + (int64_t)w * ng * ng, bn);
        if (s) return s;
        jobs.push_back(j);
    }
    return GW_OK;
}

// Time each launch-shape candidate of the contraction on the real data (into chi, which
// is cleared afterwards by the real run) and keep the fastest.
gw_status batch_autotune(gw_chi0 *h, int nq, const int *iq, int nw, const gw::OmegaList &om, const BatchLayout &L,
                         double2 *chi)
{
    const std::string key = tune_key(h, L, nw);
    auto it = h->tune_cache.find(key);
    if (it != h->tune_cache.end()) {
        h->tuned_bt = it->second[0];
        h->tuned_waves = it->second[1];
        h->tuned_bn = it->second[2];
        return GW_OK;
    }
    gw_status s = batch_stage_a(h, nq, iq, om, L);
    if (s) return s;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    std::array<int, 3> pick = {h->tuned_bt, h->tuned_waves, h->tuned_bn};
    const bool saved_timing = h->timing;
    h->timing = false;
    if (h->d.prec == GW_PREC_FP64) {
        for (int bt : {64, 32})
            for (int waves : {2, 4, 8}) {
                std::vector<gw::F64Job> jobs;
                if ((s = batch_f64_jobs(h, nq, nw, L, chi, bt, jobs))) break;
                cudaEventRecord(e0, h->st);
                if ((s = launch_f64_jobs(h, jobs, bt, waves))) break;
                cudaEventRecord(e1, h->st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    pick = {bt, waves, h->tuned_bn};
                }
            }
    } else if (!(s = batch_oz_split(h, nq, 0, L))) {
        for (int bn : {256, 128}) {
            std::vector<gw::OzJob> jobs;
            if ((s = batch_oz_jobs(h, nq, 0, L, chi, bn, jobs))) break;
            cudaEventRecord(e0, h->st);
            if ((s = launch_oz_jobs(h, jobs, bn))) break;
            cudaEventRecord(e1, h->st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                pick = {h->tuned_bt, h->tuned_waves, bn};
            }
        }
    }
    h->timing = saved_timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s) return s;
    h->tune_cache[key] = pick;
    h->tuned_bt = pick[0];
    h->tuned_waves = pick[1];
    h->tuned_bn = pick[2];
    return GW_OK;
}

gw_status compute_batch(gw_chi0 *h, int nq, const int *iq, int nw, const double *omega, const gw::OmegaList &om,
                        double *chi, double *diag)
{
    const BatchLayout L = batch_layout(h, nq, iq, nw);
    gw_status s;
    if ((s = grow(h, (void **)&h->Mall, &h->Mall_cap, sizeof(double2) * L.Mtot, "resident M")) ||
        (s = grow(h, (void **)&h->Dall, &h->Dall_cap, sizeof(double) * L.Dtot, "resident Delta")))
        return s;
    if (h->d.prec == GW_PREC_OZAKI_BF16 &&
        ((s = grow(h, (void **)&h->SPall, &h->SPall_cap, sizeof(double) * L.Dtot, "resident scales")) ||
         (s = grow(h, &h->Zall, &h->Zall_cap, sizeof(uint16_t) * L.Ztot, "resident slices")) ||
         (s = grow(h, (void **)&h->Eall, &h->Eall_cap, sizeof(int) * L.Etot, "resident exponents"))))
        return s;
    if (!h->cap_st) CK(h, cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking), "capture stream");
    if ((s = batch_autotune(h, nq, iq, nw, om, L, (double2 *)chi))) return s;

    const std::string key = batch_key(h, nq, iq, nw, omega, chi, diag) + "|" + std::to_string(h->tuned_bt) + "," +
                            std::to_string(h->tuned_waves) + "," + std::to_string(h->tuned_bn);
    gw_chi0::Graph *g = nullptr;
    for (auto &x : h->graphs)
        if (x.key == key) g = &x;
    if (!g) {
        // job tables first (outside the capture), in a buffer owned by the graph
        std::vector<gw::F64Job> fj;
        std::vector<std::vector<gw::OzJob>> oj(nw);
        std::vector<unsigned char> blob;
        std::vector<size_t> offs;
        if (h->d.prec == GW_PREC_FP64) {
            if ((s = batch_f64_jobs(h, nq, nw, L, (double2 *)chi, h->tuned_bt, fj))) return s;
            f64_schedule(fj, h->tuned_waves);
            offs.push_back(0);
            blob.resize(sizeof(gw::F64Job) * fj.size());
            std::memcpy(blob.data(), fj.data(), blob.size());
        } else {
            for (int w = 0; w < nw; ++w) {
                if ((s = batch_oz_jobs(h, nq, w, L, (double2 *)chi, h->tuned_bn, oj[w]))) return s;
                oz_schedule(oj[w]);
                offs.push_back(blob.size());
                blob.resize(blob.size() + sizeof(gw::OzJob) * oj[w].size());
                std::memcpy(blob.data() + offs.back(), oj[w].data(), sizeof(gw::OzJob) * oj[w].size());
            }
        }
        gw_chi0::Graph ng;
        ng.key = key;
        ng.jobs_bytes = blob.size();
        if ((s = dalloc(h, &ng.jobs, ng.jobs_bytes, "graph job tables"))) return s;
        CK(h, cudaMemcpy(ng.jobs, blob.data(), blob.size(), cudaMemcpyHostToDevice), "graph job tables");

        cudaStream_t user = h->st;
        const bool saved_timing = h->timing;
        h->timing = false;
        h->st = h->cap_st;
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed);
        gw_status body = GW_OK;
        if (ce == cudaSuccess) {
            for (int i = 0; i < nq && !body; ++i) {
                if (cudaMemsetAsync((double2 *)chi + L.coff[i], 0, sizeof(double2) * (size_t)nw * L.ng[i] * L.ng[i],
                                    h->st) != cudaSuccess ||
                    (diag && cudaMemsetAsync(diag + L.dgoff[i], 0, sizeof(double) * (size_t)nw * L.ng[i], h->st) !=
                                 cudaSuccess))
                    body = fail(h, GW_ERR_CUDA, "capture: memset");
            }
            if (!body) body = batch_stage_a(h, nq, iq, om, L);
            if (!body && h->d.prec == GW_PREC_FP64) {
                int nitems = 0;
                for (auto &j : fj) nitems = std::max(nitems, j.item_start + (int)((int64_t)j.ksplit * j.ntile *
                                                                                   (j.ntile + 1) / 2));
                const int grid = std::max(1, std::min(nitems, 2 * num_sms()));
                if (gw::launch_contract_f64_jobs(h->tuned_bt, (const gw::F64Job *)ng.jobs, (int)fj.size(), nitems,
                                                 grid, h->status, h->st) != cudaSuccess)
                    body = fail(h, GW_ERR_CUDA, "capture: contraction");
            } else if (!body) {
                for (int w = 0; w < nw && !body; ++w) {
                    body = batch_oz_split(h, nq, w, L);
                    if (body) break;
                    int nitems = 0;
                    for (auto &j : oj[w]) nitems = std::max(nitems, j.item_start + j.ntiles);
                    const int grid = std::max(1, std::min(nitems, num_sms()));
                    if (gw::launch_oz_gemm_jobs(h->tuned_bn, (const gw::OzJob *)((char *)ng.jobs + offs[w]),
                                                (int)oj[w].size(), nitems, grid, h->status, h->st) != cudaSuccess)
                        body = fail(h, GW_ERR_CUDA, "capture: split contraction");
                }
            }
            for (int i = 0; i < nq && !body; ++i) {
                const double2 *M = h->Mall + L.moff[i];
                if (diag && gw::launch_diag(M, L.P[i], L.ng[i], h->Dall + L.doff[i], L.P[i], nw,
                                            diag + L.dgoff[i], L.ng[i], h->st) != cudaSuccess)
                    body = fail(h, GW_ERR_CUDA, "capture: diag");
                if (!body && gw::launch_symmetrize((double2 *)chi + L.coff[i], L.ng[i], nw, h->st) != cudaSuccess)
                    body = fail(h, GW_ERR_CUDA, "capture: symmetrize");
            }
            ce = cudaStreamEndCapture(h->st, &graph);
        }
        h->st = user;
        h->timing = saved_timing;
        if (body) {
            if (graph) cudaGraphDestroy(graph);
            dfree(h, ng.jobs, ng.jobs_bytes);
            return body;
        }
        if (ce != cudaSuccess) {
            dfree(h, ng.jobs, ng.jobs_bytes);
            return cuda_fail(h, ce, "stream capture");
        }
        ce = cudaGraphInstantiate(&ng.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            dfree(h, ng.jobs, ng.jobs_bytes);
            return cuda_fail(h, ce, "graph instantiate");
        }
        h->graphs.push_back(ng);
        g = &h->graphs.back();
    }
    Scope sc(h, "batch_graph");
    CK(h, cudaGraphLaunch(g->exec, h->st), "graph launch");
    return GW_OK;
}

} // namespace

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
    dfree(h, h->epsbuf, h->epscap);
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
    std::vector<int> present(h->d.n[2], 0);
    for (int i = 0; i < ng; ++i)
        for (int a = 0; a < 3; ++a) {
            int g = s.g[3 * i + a];
            if (2 * std::abs(g) >= h->d.n[a]) return fail(h, GW_ERR_ARG, "G %d: component %d outside (-n/2, n/2)", i, g);
            s.maxabs[a] = std::max(s.maxabs[a], std::abs(g));
        }
    for (int i = 0; i < ng; ++i) present[mod(s.g[3 * i + 2], h->d.n[2])] = 1;
    std::vector<int> kz, pos(h->d.n[2], -1);
    for (int k = 0; k < h->d.n[2]; ++k)
        if (present[k]) {
            pos[k] = (int)kz.size();
            kz.push_back(k);
        }
    std::vector<int32_t> pack(ng);
    for (int i = 0; i < ng; ++i) {
        int k0 = mod(s.g[3 * i], h->d.n[0]), k1 = mod(s.g[3 * i + 1], h->d.n[1]);
        int k2 = pos[mod(s.g[3 * i + 2], h->d.n[2])];
        pack[i] = k0 | (k1 << 8) | (k2 << 16);
    }
    // alias check against whatever bands are already stored
    int ax;
    if (h->val[iq].nb && h->cond.nb && !alias_free(h, h->val[iq], h->cond, s, &ax))
        return fail(h, GW_ERR_ARG, "max|K_v| + max|K_c| + max|G| >= n on axis %d (aliasing)", ax);
    s.K2 = (int)kz.size();
    {
        // group sphere points by their (k2 column, k1) cell
        std::vector<std::pair<int, int>> key(ng);
        for (int i = 0; i < ng; ++i) key[i] = {(pack[i] >> 16) * h->d.n[1] + ((pack[i] >> 8) & 255), i};
        std::sort(key.begin(), key.end());
        s.cg.resize(ng);
        for (int i = 0; i < ng; ++i) {
            if (i == 0 || key[i].first != key[i - 1].first) s.cstart.push_back(i);
            s.cg[i] = key[i].second;
        }
        s.cstart.push_back(ng);
    }
    // cell table of the pruned i1 stage and the sphere points grouped by cell
    s.K12 = (int)s.cstart.size() - 1;
    std::vector<int32_t> cell(s.K12);
    std::vector<int2> cpts(ng);
    for (int d = 0; d < s.K12; ++d) {
        const int i = s.cg[s.cstart[d]];
        cell[d] = (pack[i] >> 16) << 8 | ((pack[i] >> 8) & 255);
        for (int m = s.cstart[d]; m < s.cstart[d + 1]; ++m) cpts[m] = make_int2(s.cg[m], (pack[s.cg[m]] & 255) | d << 8);
    }
    gw_status st;
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
        gw_status s = ensure_work(h, (size_t)chunk * ng, (size_t)chunk * nw);
        if (s) return s;
        gw::PairPlan pp = pair_plan(h, sp);
        const int64_t fault_at = fault_chunk();
        for (int64_t p0 = 0, k = 0; p0 < P; p0 += chunk, ++k) {
            int64_t cnt = std::min(chunk, P - p0);
            if (k == fault_at) return fail(h, GW_ERR_CUDA, "injected host-side fault before chunk %lld", (long long)k);
            {
                Scope sc(h, "pair_mtxel");
                CK(h, run_pair(h, v.psi, h->cond.psi, h->cond.nb, p0, cnt, pp, h->Mbuf), "pair kernel");
            }
            {
                Scope sc(h, "delta");
                CK(h, gw::launch_delta(v.energy, h->cond.energy, h->cond.nb, p0, cnt, om, h->dbuf, h->st), "delta");
            }
            s = contract_chunk(h, h->Mbuf, cnt, ng, h->dbuf, cnt, nw, cq);
            if (s) return s;
            if (dq) {
                Scope sc(h, "diag");
                CK(h, gw::launch_diag(h->Mbuf, cnt, ng, h->dbuf, cnt, nw, dq, ng, h->st), "diag");
            }
        }
        {
            Scope sc(h, "symmetrize");
            CK(h, gw::launch_symmetrize(cq, ng, nw, h->st), "symmetrize");
        }
        off += (size_t)nw * ng * ng;
        doff += (size_t)nw * ng;
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
    double2 *Mb = nullptr, *Yb = nullptr, *Hb = nullptr, *pbv = nullptr, *pbc = nullptr;
    double *Lacc = nullptr;
    int *cs = nullptr, *cg = nullptr;
    const int ncell = (int)sp.cstart.size() - 1;
    size_t szM = sizeof(double2) * cmax * ng, szH = sizeof(double2) * cmax * nr;
    size_t szV = sizeof(double2) * (size_t)nv * nr, szC = sizeof(double2) * (size_t)nc * nr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(h->st);
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
        (s = dalloc(h, (void **)&cg, sizeof(int) * ng, "cells"))) {
        cleanup();
        return s;
    }
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
    if (split && (s = oz_prepare_b(h, (const double2 *)W, ng, ng))) {
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
                ACK(gw::launch_zgemm(Mb, (const double2 *)W, Yb, cnt, ng, ng, h->st), "Y = M W");
            }
        }
        {
            Scope sc(h, "adj_rows");
            ACK(gw::launch_adj_rows(Mb, Yb, cnt, ng, nc, p0, v.energy, c.energy, omega, Lacc, dE_v, dE_c, h->st),
                "row reductions");
        }
        {
            Scope sc(h, "adj_pair");
            ACK(gw::launch_adj_pair(Yb, cnt, pp, cs, cg, ncell, Hb, h->st), "back-projection");
        }
        {
            Scope sc(h, "adj_products");
            ACK(gw::launch_adj_products(v.psi, c.psi, v0, nvc, nc, Hb, nr, tf, pbv, pbc, h->st), "products");
        }
    }
    {
        Scope sc(h, "adj_band");
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

gw_status gw_chi0_sync(gw_chi0 *h)
{
    if (!h) return GW_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->st), "sync");
    int st = 0;
    CK(h, cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost), "status");
    CK(h, cudaMemset(h->status, 0, sizeof(int)), "status reset");
    if (st & gw::kStatusTimeout) return fail(h, GW_ERR_TIMEOUT, "a bounded device-side wait gave up");
    if (st & gw::kStatusNoSlot) return fail(h, GW_ERR_CUDA, "a pair block found no free scratch slot");
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
    for (int64_t p0 = 0; p0 < P; p0 += chunk) {
        const int64_t cnt = std::min(chunk, P - p0);
        {
            Scope sc(h, "pair_mtxel");
            CK(h, run_pair(h, v.psi, h->cond.psi, h->cond.nb, p0, cnt, pp, h->Mbuf), "pair kernel");
        }
        {
            Scope sc(h, "subspace_projection");
            if (split) {
                if ((s = oz_product(h, h->Mbuf, cnt, ng, neig, h->MBbuf))) return s;
            } else {
                CK(h, gw::launch_zgemm(h->Mbuf, (const double2 *)basis, h->MBbuf, cnt, ng, neig, h->st), "projection");
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
static gw_status square_product(gw_chi0 *h, const double2 *A, const double2 *B, int n, double2 *C)
{
    if (h->d.prec == GW_PREC_OZAKI_BF16) {
        gw_status st = oz_prepare_b(h, B, n, n);
        if (st) return st;
        return oz_product(h, A, n, n, n, C);
    }
    CK(h, gw::launch_zgemm(A, B, C, n, n, n, h->st), "product");
    return GW_OK;
}

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
        for (int k = 0; k < steps; ++k) {
            if ((st = square_product(h, A, X, ng, T)) || (st = square_product(h, X, T, ng, Pm))) return st;
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
    for (int64_t p0 = 0; p0 < P; p0 += chunk) {
        const int64_t cnt = std::min(chunk, P - p0);
        {
            Scope sc(h, "pair_mtxel");
            CK(h, run_pair(h, v.psi, h->cond.psi, h->cond.nb, p0, cnt, pp, h->Mbuf), "pair kernel");
        }
        {
            Scope sc(h, "delta");
            CK(h, gw::launch_delta_real(v.energy, h->cond.energy, h->cond.nb, p0, cnt, om, eta, h->dbuf, h->st),
               "real-axis delta");
        }
        if ((s = contract_chunk(h, h->Mbuf, cnt, ng, h->dbuf, cnt, 3 * nw, h->realbuf))) return s;
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
    for (int64_t p0 = 0; p0 < P; p0 += chunk) {
        const int64_t cnt = std::min(chunk, P - p0);
        {
            Scope sc(h, "pair_mtxel");
            JCK(run_pair(h, v.psi, c.psi, nc, p0, cnt, pp, h->Mbuf), "pair kernel");
            JCK(run_pair(h, gv, c.psi, nc, p0, cnt, pp, X1), "pair kernel (tangent valence)");
            JCK(run_pair(h, v.psi, gc, nc, p0, cnt, pp, X2), "pair kernel (tangent conduction)");
            JCK(gw::launch_jvp_mix(h->Mbuf, X1, X2, cnt * ng, h->st), "M +- dM");
        }
        {
            Scope sc(h, "delta");
            JCK(gw::launch_delta(v.energy, c.energy, nc, p0, cnt, om, h->dbuf, h->st), "delta");
            JCK(gw::launch_delta_jvp(v.energy, c.energy, dE_v, dE_c, nc, p0, cnt, om, wb, h->st), "delta derivative");
        }
        // d chi = [chi(M + dM) - chi(M - dM)] / 2 + sum_p conj(M) dDelta M
        if ((s = contract_chunk(h, X1, cnt, ng, h->dbuf, cnt, nw, Tp)) ||
            (s = contract_chunk(h, X2, cnt, ng, h->dbuf, cnt, nw, Tm)) ||
            (s = contract_chunk(h, h->Mbuf, cnt, ng, wb, cnt, 2 * nw, Tw))) {
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

