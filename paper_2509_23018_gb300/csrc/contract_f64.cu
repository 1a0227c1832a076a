// Stage (b), native FP64: the energy-weighted Hermitian contraction of Eq. chi_mat,
//
//     chi[w][G][G'] += sum_p conj(M[p][G]) Delta_p(w) M[p][G'],
//
// on the FP64 tensor cores (DMMA, mma.sync m8n8k4 f64).  M tiles are brought into
// shared memory by TMA (cp.async.bulk.tensor.2d, mbarrier completion), a 3-stage ring;
// Delta is applied to the G' operand as the fragments move from shared memory into
// registers.  Only tiles with I <= J (upper triangle) are computed; the lower triangle
// is filled by the symmetrisation step.  The pair range of one launch may be split over
// several blocks per tile; partial tiles are added into chi with FP64 atomics.
#include "internal.h"

namespace gw {

constexpr int kBT = 64;      // complex tile edge
constexpr int kBK = 16;      // pairs per stage
constexpr int kStages = 3;
constexpr int kThreads = 256;
constexpr unsigned kTileBytes = kBK * kBT * 2 * sizeof(double); // one operand tile
constexpr long long kWaitLimit = 1LL << 26;

int contract_f64_tile() { return kBT; }
int contract_f64_bk() { return kBK; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Bounded wait on phase `parity`; returns false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    uint32_t a = smem_u32(bar);
    for (long long it = 0; it < kWaitLimit; ++it) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void dmma(double &d0, double &d1, double a, double b)
{
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(d0), "+d"(d1)
                 : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(kThreads) contract_f64_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                const double *__restrict__ delta, int64_t dstride,
                                                                int64_t P, int ng, int ntile, int ksplit,
                                                                double *__restrict__ chi, int *status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    double *sA = (double *)smem;                       // [kStages][kBK][2*kBT]
    double *sB = sA + kStages * kBK * 2 * kBT;         // [kStages][kBK][2*kBT]
    uint64_t *bar = (uint64_t *)(sB + kStages * kBK * 2 * kBT);

    const int w = blockIdx.z;
    const int tile = blockIdx.x / ksplit, ks = blockIdx.x - tile * ksplit;
    int I = 0, rem = tile;
    while (rem >= ntile - I) { rem -= ntile - I; ++I; }
    const int J = I + rem;

    const int64_t nkt = (P + kBK - 1) / kBK;
    const int64_t kper = (nkt + ksplit - 1) / ksplit;
    const int64_t kt0 = ks * kper;
    const int64_t kt1 = kt0 + kper < nkt ? kt0 + kper : nkt;
    const int nk = kt1 > kt0 ? (int)(kt1 - kt0) : 0;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int wm = wid & 1, wn = wid >> 1;  // 2 x 4 warps, each 32 x 16 complex
    const double *dl = delta + (int64_t)w * dstride;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    auto issue = [&](int it) {
        int s = it % kStages;
        int y = (int)((kt0 + it) * kBK);
        mbar_expect_tx(&bar[s], 2 * kTileBytes);
        tma_load_2d(sA + s * kBK * 2 * kBT, &tmap, &bar[s], 2 * kBT * I, y);
        tma_load_2d(sB + s * kBK * 2 * kBT, &tmap, &bar[s], 2 * kBT * J, y);
    };
    if (tid == 0)
        for (int it = 0; it < kStages && it < nk; ++it) issue(it);

    double cre[4][2][2], cim[4][2][2];
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            cre[mt][nt][0] = cre[mt][nt][1] = 0.0;
            cim[mt][nt][0] = cim[mt][nt][1] = 0.0;
        }

    bool ok = true;
    int it = 0;
    for (; it < nk; ++it) {
        const int s = it % kStages;
        if (!mbar_wait(&bar[s], (unsigned)((it / kStages) & 1))) { ok = false; break; }
        const double *A = sA + s * kBK * 2 * kBT;
        const double *B = sB + s * kBK * 2 * kBT;
        const int64_t pbase = (kt0 + it) * kBK;
#pragma unroll
        for (int kk = 0; kk < kBK / 4; ++kk) {
            const int pr = kk * 4 + (lane & 3);
            const int64_t pg = pbase + pr;
            const double d = pg < P ? __ldg(dl + pg) : 0.0;
            double ar[4], ai[4], br[2], bi[2], nbr[2];
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
                double2 x = *(const double2 *)(A + pr * 2 * kBT + 2 * (wm * 32 + mt * 8 + (lane >> 2)));
                ar[mt] = x.x;
                ai[mt] = x.y;
            }
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                double2 x = *(const double2 *)(B + pr * 2 * kBT + 2 * (wn * 16 + nt * 8 + (lane >> 2)));
                br[nt] = d * x.x;   // Delta scaled into the G' operand on its way to registers
                bi[nt] = d * x.y;
                nbr[nt] = -br[nt];
            }
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    // conj(a) b = (ar br + ai bi) + i (ar bi - ai br)
                    dmma(cre[mt][nt][0], cre[mt][nt][1], ar[mt], br[nt]);
                    dmma(cre[mt][nt][0], cre[mt][nt][1], ai[mt], bi[nt]);
                    dmma(cim[mt][nt][0], cim[mt][nt][1], ar[mt], bi[nt]);
                    dmma(cim[mt][nt][0], cim[mt][nt][1], ai[mt], nbr[nt]);
                }
        }
        __syncthreads(); // every warp is done with stage s
        if (tid == 0 && it + kStages < nk) issue(it + kStages);
    }
    if (!ok) {
        if (tid == 0) atomicOr(status, kStatusTimeout);
        // let copies already in flight land before the block's shared memory is released
        if (tid == 0)
            for (int j = it; j < nk && j < it + kStages; ++j) mbar_wait(&bar[j % kStages], (unsigned)((j / kStages) & 1));
        __syncthreads();
        return;
    }

    double *cw = chi + (int64_t)w * ng * ng * 2;
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
        const int G = I * kBT + wm * 32 + mt * 8 + (lane >> 2);
        if (G >= ng) continue;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int Gp = J * kBT + wn * 16 + nt * 8 + 2 * (lane & 3) + q;
                if (Gp >= ng) continue;
                double *dst = cw + 2 * ((int64_t)G * ng + Gp);
                atomicAdd(dst, cre[mt][nt][q]);
                atomicAdd(dst + 1, cim[mt][nt][q]);
            }
    }
}

cudaError_t launch_contract_f64(const CUtensorMap *tmap, const double *delta, int64_t dstride, int64_t P, int ng,
                                int nw, double *chi, int ksplit, int *status, cudaStream_t st)
{
    if (P == 0 || nw == 0) return cudaSuccess;
    const int ntile = (ng + kBT - 1) / kBT;
    const int nup = ntile * (ntile + 1) / 2;
    const size_t sm = 2 * (size_t)kStages * kTileBytes + kStages * sizeof(uint64_t);
    cudaError_t e = cudaFuncSetAttribute(contract_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (ksplit < 1) ksplit = 1;
    contract_f64_kernel<<<dim3((unsigned)(nup * ksplit), 1, nw), kThreads, sm, st>>>(*tmap, delta, dstride, P, ng,
                                                                                    ntile, ksplit, chi, status);
    return cudaGetLastError();
}

} // namespace gw
