// gw_chi0_contract_noalloc: the FP64 contraction for callers that must not allocate.
//
// Some callers cannot call cudaMalloc: plugins that run under a host framework which owns
// every device allocation through its own pool (a stray cudaMalloc there fragments the
// pool or fails once the pool has reserved the free memory), and services that forbid
// allocator calls on their hot path because cudaMalloc and cudaFree can synchronise the
// device and take unbounded time.  This entry point computes the same result as
// gw_chi0_contract in GW_PREC_FP64 mode, but the one piece of scratch it needs (the energy
// factors Delta, the kernel's job table and a status word) lives in a fixed, file-scope
// device array instead of memory obtained from an allocator.
#include "../../include/gw_chi0.h"
#include "internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

namespace {

// Scratch: 256 bytes for the status word, kMaxOmega job tables, then kNoAllocDelta
// doubles of Delta.  Every device that loads this library holds the array until exit.
constexpr size_t kNoAllocDelta = size_t(1) << 19; // nw * nv * nc must not exceed this
constexpr size_t kNoAllocJobs = gw::kMaxOmega * sizeof(gw::F64Job) / sizeof(double);
constexpr size_t kNoAllocHead = 256 / sizeof(double);
constexpr int kNoAllocTile = 64;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocHead + kNoAllocJobs + kNoAllocDelta];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch[kMaxDevices] = {nullptr};
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

// Once per device, with that device current: the device address of the scratch array.
// The host-side symbol is only a stand-in; kernels must be given this address.
gw_status setup(int dev, double **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= kMaxDevices) return GW_ERR_UNSUPPORTED;
    if (!g_scratch[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return GW_ERR_CUDA;
        }
        g_scratch[dev] = (double *)p;
    }
    if (!g_encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return GW_ERR_CUDA;
        }
        g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    *out = g_scratch[dev];
    return GW_OK;
}

// A bounded wait that gave up leaves its tile out of chi; mark such a result unusable by
// writing NaN on the diagonal of every block (the caller cannot read the status word).
__global__ void noalloc_poison_kernel(const int *status, double2 *chi, int ng, int nw)
{
    if (*status == 0) return;
    const int64_t n = (int64_t)ng * nw;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t w = i / ng, g = i - w * ng;
        chi[w * ng * ng + g * ng + g] = make_double2(__longlong_as_double(0x7ff8000000000000LL), 0.0);
    }
}

} // namespace

extern "C" gw_status gw_chi0_contract_noalloc(int nv, int nc, const double *ev, const double *ec, int ng,
                                              const double *M, int nw, const double *omega, double *chi,
                                              void *cuda_stream)
{
    if (nv < 1 || nc < 1 || ng < 1 || nw < 1 || nw > gw::kMaxOmega || !ev || !ec || !M || !omega || !chi)
        return GW_ERR_ARG;
    const int64_t P = (int64_t)nv * nc;
    if ((size_t)nw * (size_t)P > kNoAllocDelta) return GW_ERR_ARG; // beyond the fixed scratch
    if (((uintptr_t)M & 15) != 0) return GW_ERR_ARG;
    gw::OmegaList om;
    om.nw = nw;
    for (int i = 0; i < nw; ++i) {
        if (!(omega[i] >= 0.0) || !std::isfinite(omega[i])) return GW_ERR_ARG;
        om.w[i] = omega[i];
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GW_ERR_CUDA;
    }
    double *scratch = nullptr;
    gw_status s = setup(dev, &scratch);
    if (s) return s;
    int *status = (int *)scratch;
    double *delta = scratch + kNoAllocHead + kNoAllocJobs;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    // scratch layout: status word, kMaxOmega job tables, then Delta
    gw::F64Job job;
    std::memset(&job, 0, sizeof job);
    cuuint64_t dims[2] = {(cuuint64_t)2 * ng, (cuuint64_t)P};
    cuuint64_t strides[1] = {(cuuint64_t)2 * ng * sizeof(double)};
    cuuint32_t box[2] = {(cuuint32_t)(2 * kNoAllocTile), (cuuint32_t)gw::contract_f64_bk()};
    cuuint32_t es[2] = {1, 1};
    if (g_encode(&job.tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double *>(M), dims, strides, box, es,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return GW_ERR_CUDA;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nt = (ng + kNoAllocTile - 1) / kNoAllocTile;
    const int64_t tiles = (int64_t)nt * (nt + 1) / 2 * nw;
    int64_t ks = (8LL * sms + tiles - 1) / tiles;
    ks = std::max<int64_t>(1, std::min<int64_t>(ks, (P + 255) / 256));
    // one job per frequency, all sharing M
    static thread_local gw::F64Job jobs[gw::kMaxOmega];
    int items = 0;
    for (int w = 0; w < nw; ++w) {
        jobs[w] = job;
        jobs[w].delta = delta + (int64_t)w * P;
        jobs[w].chi = chi + 2 * (int64_t)w * ng * ng;
        jobs[w].P = P;
        jobs[w].ng = ng;
        jobs[w].ntile = nt;
        jobs[w].ksplit = (int)ks;
        jobs[w].item_start = items;
        items += (int)(ks * nt * (nt + 1) / 2);
    }
    gw::F64Job *djobs = (gw::F64Job *)(scratch + kNoAllocHead);

    // the scratch keeps the previous call's contents: the status word must start at zero
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess ||
        cudaMemcpyAsync(djobs, jobs, sizeof(gw::F64Job) * nw, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(chi, 0, sizeof(double) * 2 * (size_t)nw * ng * ng, st) != cudaSuccess ||
        gw::launch_delta(ev, ec, nc, 0, P, om, delta, st) != cudaSuccess) {
        cudaGetLastError();
        return GW_ERR_CUDA;
    }
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(items, 2LL * sms));
    if (gw::launch_contract_f64_jobs(kNoAllocTile, djobs, nw, items, grid, status, st) != cudaSuccess ||
        gw::launch_symmetrize((double2 *)chi, ng, nw, st) != cudaSuccess) {
        cudaGetLastError();
        return GW_ERR_CUDA;
    }
    noalloc_poison_kernel<<<(unsigned)std::min<int64_t>(((int64_t)ng * nw + 255) / 256, 1024), 256, 0, st>>>(
        status, (double2 *)chi, ng, nw);
    if (cudaGetLastError() != cudaSuccess) return GW_ERR_CUDA;
    return GW_OK;
}
