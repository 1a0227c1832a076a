// Host side of the C ABI declared in include/gw_chi0.h: the handle, its band sets and
// spheres, and the helpers shared by api.cu (handle, setup, streamed path, status and
// timing), api_batch.cu (the batched graph path) and api_ext.cu (adjoint, static subspace,
// dielectric inverse, real axis, forward derivative).  Not part of the public interface.
#pragma once
#include "../../include/gw_chi0.h"
#include "internal.h"
#include "sphere_plan.h"

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

namespace gwapi {
using gw::FftAxis;
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
} // namespace gwapi

using gwapi::BandSet;
using gwapi::Sphere;
using gwapi::TimerRec;

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
    bool bn_tuned = false; // tuned_bn set by the autotuner (else the width follows the wave count)
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
    // overlapped streamed path: contractions on a high-priority second stream, buffers by parity
    cudaStream_t ov_st = nullptr;
    cudaEvent_t ov_split[2] = {nullptr, nullptr}, ov_gemm[2] = {nullptr, nullptr};
    void *ovZ[2] = {nullptr, nullptr};
    size_t ovZcap[2] = {0, 0};
    int *ovE[2] = {nullptr, nullptr};
    size_t ovEcap[2] = {0, 0};
    void *ovJ[2] = {nullptr, nullptr};
    size_t ovJcap[2] = {0, 0};
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
    // pair elements of one slot kept resident between calls (gw_chi0_keep_pair_elements): written
    // by gw_chi0_compute, reused by gw_chi0_compute_subspace / gw_chi0_compute_real
    bool keep_m = false;
    double2 *Mres = nullptr;
    size_t Mres_cap = 0; // bytes
    int Mres_iq = -1;    // slot whose elements the buffer holds; -1: none
    // plasmon-pole self-energy work buffers (api_sigma.cu)
    struct Buf {
        void *p = nullptr;
        size_t cap = 0;
    } gpp[9];
    // stage (a) with the last-axis transform on the tensor cores (zdft.cu): valence slices of the
    // slot being computed and the transform output F of one chunk
    void *zdA = nullptr;
    size_t zdAcap = 0;  // bytes
    float4 *zdF = nullptr;
    size_t zdFcap = 0;  // bytes
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

namespace gwapi {

#define CK(h, x, what)                                   \
    do {                                                 \
        cudaError_t e_ = (x);                            \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    } while (0)

cudaEvent_t ev_get(gw_chi0 *h);

// Per-kernel timing: events around the enqueued work when the handle's timing is on.
struct Scope {
    gw_chi0 *h;
    const char *name;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    Scope(gw_chi0 *h_, const char *n, cudaStream_t s_ = nullptr) : h(h_), name(n), s(s_ ? s_ : h_->st)
    {
        if (h->timing) {
            a = ev_get(h);
            cudaEventRecord(a, s);
        }
    }
    ~Scope()
    {
        if (h->timing) {
            cudaEvent_t b = ev_get(h);
            cudaEventRecord(b, s);
            h->pending.push_back({name, a, b});
        }
    }
};

gw_status fail(gw_chi0 *h, gw_status s, const char *fmt, ...);
gw_status cuda_fail(gw_chi0 *h, cudaError_t e, const char *what);
gw_status dalloc(gw_chi0 *h, void **p, size_t n, const char *what);
void dfree(gw_chi0 *h, void *p, size_t n);
bool factor(int n, FftAxis &a);
int mod(int a, int n);
void drain_timing(gw_chi0 *h);
gw_status ensure_work(gw_chi0 *h, size_t m_elems, size_t d_elems);
gw_status make_tmap(gw_chi0 *h, CUtensorMap *map, const void *M, int64_t P, int ng, int bt);
int num_sms();
int contraction_bn(const gw_chi0 *h, int ng); // split-precision tile width: tuned, else by the wave count
void drop_graphs(gw_chi0 *h);
gw_status grow(gw_chi0 *h, void **p, size_t *cap, size_t bytes, const char *what);
gw_status upload_jobs(gw_chi0 *h, const void *src, size_t bytes, const void **dev);
gw_status f64_jobs(gw_chi0 *h, std::vector<gw::F64Job> &jobs, const double2 *M, int64_t P, int ng,
                   const double *delta, int64_t dstride, int nw, double2 *chi, int bt);
int f64_schedule(std::vector<gw::F64Job> &jobs, int waves);
gw_status launch_f64_jobs(gw_chi0 *h, std::vector<gw::F64Job> &jobs, int bt, int waves);
gw_status make_tmap_z(gw_chi0 *h, CUtensorMap *map, void *Z, int64_t kpad, int nrows, int s, int box_rows);
gw_status oz_job(gw_chi0 *h, gw::OzJob &j, void *Z, int64_t kpad, int ng, const int *E, double2 *chi, int bn);
int oz_schedule(std::vector<gw::OzJob> &jobs);
gw_status launch_oz_jobs(gw_chi0 *h, std::vector<gw::OzJob> &jobs, int bn);
gw_status contract_chunk_ozaki(gw_chi0 *h, const double2 *M, int64_t P, int ng, const double *delta, int64_t dstride,
                               int nw, double2 *chi);
gw_status contract_chunk(gw_chi0 *h, const double2 *M, int64_t P, int ng, const double *delta, int64_t dstride,
                         int nw, double2 *chi);
int64_t oz_kpad(int ka);
// nslices > 0 overrides the handle's slice count (both calls of one product must agree)
gw_status oz_prepare_b(gw_chi0 *h, const double2 *B, int ka, int nout, int nslices = 0);
gw_status oz_product(gw_chi0 *h, const double2 *A, int64_t rows, int ka, int nout, double2 *Y, int nslices = 0);
bool alias_free(const gw_chi0 *h, const BandSet &v, const BandSet &c, const Sphere &s, int *axis);
gw_status check_slot(gw_chi0 *h, int iq);
cudaError_t run_pair(gw_chi0 *h, const void *psiv, const void *psic, int nc, int64_t p0, int64_t cnt,
                     const gw::PairPlan &pp, double2 *M);
gw::PairPlan pair_plan(gw_chi0 *h, const Sphere &s);
void free_bands(gw_chi0 *h, BandSet &b);
void free_sphere(gw_chi0 *h, Sphere &s);

// resident pair elements: resident_begin makes room for slot iq's P x ng elements when keeping is
// on and they fit (*use), invalidating what the buffer held; resident_for(h, iq) is the buffer when
// it holds slot iq, else null
gw_status resident_begin(gw_chi0 *h, int64_t P, int ng, bool *use);
double2 *resident_for(gw_chi0 *h, int iq);
// overlapped split-precision streamed compute of one slot (api.cu); Mres: resident output or null
gw_status compute_overlap(gw_chi0 *h, int iq, const gw::OmegaList &om, double2 *cq, double *dq, double2 *Mres);
// Stage (a) with the last-axis transform on the tensor cores: whether slot iq takes it, the
// conduction bands per chunk, the valence slices (once per call), and one chunk's pair
// elements M[cl nv + v] for the conduction bands c0 .. c0 + cb - 1.
bool zd_route(gw_chi0 *h, int iq, bool resident);
gw_status ensure_overlap_stream(gw_chi0 *h);
int zd_chunk_bands(gw_chi0 *h, int iq);
gw_status zd_prepare(gw_chi0 *h, int iq, CUtensorMap *tmA, CUtensorMap *tmC);
gw_status zd_stage_a(gw_chi0 *h, int iq, const CUtensorMap &tmA, const CUtensorMap &tmC, int c0, int cb,
                     const gw::PairPlan &pp, double2 *M);
bool overlap_enabled(gw_chi0 *h, const gw::PairPlan &pp);

// batched path (api_batch.cu)
gw_status compute_batch(gw_chi0 *h, int nq, const int *iq, int nw, const double *omega, const gw::OmegaList &om,
                        double *chi, double *diag);

} // namespace gwapi
