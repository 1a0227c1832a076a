// Stage (b), native FP64: the energy-weighted Hermitian contraction of Eq. chi_mat,
//
//     chi[G][G'] += sum_p conj(M[p][G]) Delta_p M[p][G'],
//
// on the FP64 tensor cores (DMMA, mma.sync m8n8k4 f64).  M tiles are brought into shared
// memory by TMA (cp.async.bulk.tensor.2d, mbarrier completion) through a 3-stage ring;
// Delta is applied to the G' operand as the fragments move from shared memory into
// registers.  Only tiles with I <= J (upper triangle) are computed; the lower triangle is
// filled by the symmetrisation step.
//
// The kernel is persistent and batched: a launch takes a table of jobs (one job = one
// (q-point, frequency) block with its own M, Delta, output and sphere size N_G) and a
// list of work items (job, upper tile, pair split), ordered largest job first; block b
// takes items b, b + gridDim.x, ...  Partial tiles are added into chi with FP64 atomics.
// The tile edge is a template parameter chosen by the autotuner (32 or 64 complex).
#include "internal.h"
#include "ptx.cuh"

namespace gw {

constexpr int kF64BK = 16;      // pairs per stage
constexpr int kF64Stages = 3;
constexpr int kF64Threads = 256;

template <int BT>
constexpr size_t f64_smem() { return 2 * (size_t)kF64Stages * kF64BK * 2 * BT * sizeof(double) + kF64Stages * 8; }

template <int BT>
__global__ void __launch_bounds__(kF64Threads) contract_f64_kernel(const F64Job *__restrict__ jobs, int njobs,
                                                                   int nitems, int *status)
{
    constexpr int WR = BT / 2, WC = BT / 4, MT = WR / 8, NT = WC / 8;
    constexpr unsigned kTileBytes = kF64BK * BT * 2 * sizeof(double);
    extern __shared__ __align__(1024) unsigned char smem[];
    double *sA = (double *)smem;                             // [stages][BK][2 BT]
    double *sB = sA + kF64Stages * kF64BK * 2 * BT;          // [stages][BK][2 BT]
    uint64_t *bar = (uint64_t *)(sB + kF64Stages * kF64BK * 2 * BT);

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int wm = wid & 1, wn = wid >> 1; // 2 x 4 warps
    if (tid == 0) {
        for (int s = 0; s < kF64Stages; ++s) bar_init(&bar[s], 1);
        bar_fence_init();
    }
    __syncthreads();

    uint32_t base = 0; // stages consumed so far by this block (ring position and phase)
    bool ok = true;
    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
        int lo = 0, hi = njobs - 1; // job with the largest item_start <= item
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].item_start <= item) lo = mid;
            else hi = mid - 1;
        }
        const F64Job &jb = jobs[lo];
        const int local = item - jb.item_start;
        const int tile = local / jb.ksplit, ks = local - tile * jb.ksplit;
        int I = 0, rem = tile;
        while (rem >= jb.ntile - I) { rem -= jb.ntile - I; ++I; }
        const int J = I + rem;
        const int64_t P = jb.P;
        const int ng = jb.ng;
        const int64_t nkt = (P + kF64BK - 1) / kF64BK;
        const int64_t kper = (nkt + jb.ksplit - 1) / jb.ksplit;
        const int64_t kt0 = ks * kper;
        const int64_t kt1 = kt0 + kper < nkt ? kt0 + kper : nkt;
        const int nk = kt1 > kt0 ? (int)(kt1 - kt0) : 0;
        if (nk == 0) continue;
        const CUtensorMap *tm = &jb.tm;
        const double *dl = jb.delta;

        auto issue = [&](int it) {
            const int s = (int)((base + it) % kF64Stages);
            const int y = (int)((kt0 + it) * kF64BK);
            bar_expect(&bar[s], 2 * kTileBytes);
            tma2(sA + s * kF64BK * 2 * BT, tm, &bar[s], 2 * BT * I, y);
            tma2(sB + s * kF64BK * 2 * BT, tm, &bar[s], 2 * BT * J, y);
        };
        if (tid == 0)
            for (int it = 0; it < kF64Stages && it < nk; ++it) issue(it);

        double cre[MT][NT][2], cim[MT][NT][2];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                cre[mt][nt][0] = cre[mt][nt][1] = 0.0;
                cim[mt][nt][0] = cim[mt][nt][1] = 0.0;
            }
        int it = 0;
        for (; it < nk; ++it) {
            const uint32_t g = base + it;
            const int s = (int)(g % kF64Stages);
            const bool got = bar_wait(&bar[s], (g / kF64Stages) & 1);
            if (!__syncthreads_and(got)) { ok = false; break; } // block-uniform exit
            const double *A = sA + s * kF64BK * 2 * BT;
            const double *B = sB + s * kF64BK * 2 * BT;
            const int64_t pbase = (kt0 + it) * kF64BK;
#pragma unroll
            for (int kk = 0; kk < kF64BK / 4; ++kk) {
                const int pr = kk * 4 + (lane & 3);
                const int64_t pg = pbase + pr;
                const double d = pg < P ? __ldg(dl + pg) : 0.0;
                double ar[MT], ai[MT], br[NT], bi[NT], nbr[NT];
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    double2 x = *(const double2 *)(A + pr * 2 * BT + 2 * (wm * WR + mt * 8 + (lane >> 2)));
                    ar[mt] = x.x;
                    ai[mt] = x.y;
                }
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    double2 x = *(const double2 *)(B + pr * 2 * BT + 2 * (wn * WC + nt * 8 + (lane >> 2)));
                    br[nt] = d * x.x; // Delta scaled into the G' operand on its way to registers
                    bi[nt] = d * x.y;
                    nbr[nt] = -br[nt];
                }
#pragma unroll
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt) {
                        // conj(a) b = (ar br + ai bi) + i (ar bi - ai br)
                        dmma884(cre[mt][nt][0], cre[mt][nt][1], ar[mt], br[nt]);
                        dmma884(cre[mt][nt][0], cre[mt][nt][1], ai[mt], bi[nt]);
                        dmma884(cim[mt][nt][0], cim[mt][nt][1], ar[mt], bi[nt]);
                        dmma884(cim[mt][nt][0], cim[mt][nt][1], ai[mt], nbr[nt]);
                    }
            }
            __syncthreads(); // every warp is done with stage s
            if (tid == 0 && it + kF64Stages < nk) issue(it + kF64Stages);
        }
        if (!ok) {
            if (tid == 0) {
                atomicOr(status, kStatusTimeout);
                // let copies already in flight land before the block's shared memory is released
                for (int j = it; j < nk && j < it + kF64Stages; ++j)
                    bar_wait(&bar[(base + j) % kF64Stages], ((base + j) / kF64Stages) & 1);
            }
            break;
        }
        base += (uint32_t)nk;
        double *cw = jb.chi;
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            const int G = I * BT + wm * WR + mt * 8 + (lane >> 2);
            if (G >= ng) continue;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int Gp = J * BT + wn * WC + nt * 8 + 2 * (lane & 3) + q;
                    if (Gp >= ng) continue;
                    double *dst = cw + 2 * ((int64_t)G * ng + Gp);
                    atomicAdd(dst, cre[mt][nt][q]);
                    atomicAdd(dst + 1, cim[mt][nt][q]);
                }
        }
    }
    __syncthreads();
}

int contract_f64_bk() { return kF64BK; }

size_t contract_f64_smem(int bt) { return bt == 32 ? f64_smem<32>() : f64_smem<64>(); }

cudaError_t launch_contract_f64_jobs(int bt, const F64Job *jobs, int njobs, int nitems, int grid, int *status,
                                     cudaStream_t st)
{
    if (nitems == 0) return cudaSuccess;
    if (bt == 32) {
        cudaError_t e = cudaFuncSetAttribute(contract_f64_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)f64_smem<32>());
        if (e != cudaSuccess) return e;
        contract_f64_kernel<32><<<grid, kF64Threads, f64_smem<32>(), st>>>(jobs, njobs, nitems, status);
    } else {
        cudaError_t e = cudaFuncSetAttribute(contract_f64_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)f64_smem<64>());
        if (e != cudaSuccess) return e;
        contract_f64_kernel<64><<<grid, kF64Threads, f64_smem<64>(), st>>>(jobs, njobs, nitems, status);
    }
    return cudaGetLastError();
}

} // namespace gw
