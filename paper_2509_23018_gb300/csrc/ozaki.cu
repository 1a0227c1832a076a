// Stage (b), split precision: the contraction of Eq. chi_mat as an Ozaki-style
// error-free slice expansion on the BF16 tensor cores (tcgen05, accumulators in TMEM).
//
// With A[p][G] = s_p M[p][G], s_p = sqrt(-Delta_p) (Delta < 0), chi = -A^H A.  In real
// form Z = [Re A | Im A] interleaved by column (j = 2G + {0: Re, 1: Im}) and
// chi_GG' = -(C[2G][2G'] + C[2G+1][2G'+1]) - i (C[2G][2G'+1] - C[2G+1][2G']),  C = Z^T Z.
//
// Splitting (per chunk of pairs and per complex column G, exponent E_G with
// max_p |Z[p][2G+c]| < 2^(E_G - 1)):
//     Z[p][j] = 2^E_G sum_{i=1..s} 2^(-6 i) z_i[p][j],   z_i integers, |z_i| <= 32,
// the slices are exact in BF16.  Products of slices are exact, and every partial sum of
//     C_t = sum_{i+k=t} z_i^T z_k     (t = 2 .. s+1, triangular truncation)
// over a chunk of at most 8192 pairs stays an integer of magnitude <= 2^24 for t <= 3,
// hence exact in the FP32 accumulator; for t >= 4 it stays exact while |C_t| <= 2^24,
// which holds unless the slices are adversarially correlated.  The FP64 recombination
//     chi += -2^(E_G + E_G' - 6t) (integer combination of C_t)
// happens once per chunk and group, in the epilogue.  FP64 is kept for Delta, the
// scaling, the recombination, the accumulation across chunks and the symmetrisation.
#include "internal.h"
#include <cuda_bf16.h>
#include <algorithm>

namespace gw {

constexpr int kOzBeta = 6;
constexpr int kOzBM = 128, kOzBN = 256, kOzBK = 64, kOzStages = 4;
constexpr int kOzThreads = 192;
constexpr unsigned kOzABytes = kOzBM * kOzBK * 2, kOzBBytes = kOzBN * kOzBK * 2;
constexpr int kOzNoColumn = -400; // exponent of an all-zero column
constexpr long long kOzWait = 1LL << 24;

// ------------------------------------------------------------------ split, step 1: column exponents
// E[g] = max_p ilogb(max(|Re A|, |Im A|)) + 2 over the chunk, A = s_p M[p][g].
__global__ void oz_sqrt_kernel(const double *__restrict__ delta, int64_t n, double *__restrict__ sp)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) sp[i] = sqrt(-delta[i]);
}

__global__ void oz_colexp_kernel(const double2 *__restrict__ M, int64_t P, int ng, const double *__restrict__ sp,
                                 int *__restrict__ E)
{
    __shared__ int red[8][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = blockIdx.x * 32 + lane;
    int e = kOzNoColumn;
    if (g < ng) {
        for (int64_t p = (int64_t)blockIdx.y * 8 + wid; p < P; p += (int64_t)gridDim.y * 8) {
            double2 m = M[p * ng + g];
            double a = fmax(fabs(m.x), fabs(m.y)) * sp[p];
            if (a > 0.0) {
                int be = (int)((__double_as_longlong(a) >> 52) & 0x7ff);
                int x = (be == 0 ? -1023 : be - 1023) + 2;
                e = max(e, x);
            }
        }
    }
    red[wid][lane] = e;
    __syncthreads();
    if (wid == 0 && g < ng) {
        for (int w = 1; w < 8; ++w) e = max(e, red[w][lane]);
        atomicMax(E + g, e);
    }
}

__global__ void oz_fill_kernel(int *E, int n, int v)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) E[i] = v;
}

// ------------------------------------------------------------------ split, step 2: slices
// Z[i][j][p] (bf16, K-major rows of length kpad) for a 64-pair x 32-column block.
__global__ void __launch_bounds__(256) oz_slice_kernel(const double2 *__restrict__ M, int64_t P, int ng,
                                                       const double *__restrict__ spv, const int *__restrict__ E,
                                                       int s, int64_t kpad, __nv_bfloat16 *__restrict__ Z)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint16_t *zs = (uint16_t *)smem; // [s][64 rows j][64 + 8 pairs] (padded)
    constexpr int LD = 72;
    const int64_t p0 = (int64_t)blockIdx.y * 64;
    const int g0 = blockIdx.x * 32;
    for (int e = threadIdx.x; e < 64 * 32; e += blockDim.x) {
        const int pl = e >> 5, gl = e & 31;
        const int64_t p = p0 + pl;
        const int g = g0 + gl;
        double2 a = make_double2(0.0, 0.0);
        int Eg = kOzNoColumn;
        if (p < P && g < ng) {
            const double sp = spv[p];
            double2 m = M[p * ng + g];
            a = make_double2(m.x * sp, m.y * sp);
            Eg = E[g];
        }
        // N = round(a 2^(6 s - E)): an exact power-of-two scaling, then round to nearest
        const int sh = kOzBeta * s - Eg;
        const double sc = __longlong_as_double((long long)(1023 + max(-1022, min(1023, sh))) << 52);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            long long N = __double2ll_rn((c ? a.y : a.x) * sc);
            // balanced base-64 digits, least significant first; the top digit keeps the rest
            for (int i = s - 1; i >= 1; --i) {
                int d = (int)((N + 32) & 63) - 32;
                N = (N - d) >> 6;
                zs[(i * 64 + 2 * gl + c) * LD + pl] = (uint16_t)(__float_as_uint((float)d) >> 16);
            }
            zs[(0 * 64 + 2 * gl + c) * LD + pl] = (uint16_t)(__float_as_uint((float)N) >> 16);
        }
    }
    __syncthreads();
    // rows j = 2 g0 .. 2 g0 + 63 of each slice, 64 consecutive pairs = 128 bytes
    const int nrows = 2 * ng;
    for (int e = threadIdx.x; e < s * 64 * 8; e += blockDim.x) {
        const int i = e / (64 * 8), r = (e >> 3) & 63, v = e & 7;
        const int j = 2 * g0 + r;
        if (j >= nrows) continue;
        const uint4 val = *(const uint4 *)(zs + (i * 64 + r) * LD + v * 8);
        *(uint4 *)(Z + ((int64_t)i * nrows + j) * kpad + p0 + v * 8) = val;
    }
}

// ------------------------------------------------------------------ tcgen05 GEMM
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t *b, unsigned c)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(c));
}
__device__ __forceinline__ void bar_expect(uint64_t *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool bar_wait(uint64_t *b, unsigned parity)
{
    const uint32_t a = su32(b);
    for (long long it = 0; it < kOzWait; ++it) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void tma3(void *dst, const CUtensorMap *m, uint64_t *b, int x, int y, int z)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                 ::"r"(su32(dst)), "l"(m), "r"(x), "r"(y), "r"(z), "r"(su32(b))
                 : "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *b)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

#define OZ_LD32(taddr, v)                                                                                        \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"  \
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                        \
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), \
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),        \
                   "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),      \
                   "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),      \
                   "=r"(v[29]), "=r"(v[30]), "=r"(v[31])                                                           \
                 : "r"(taddr))

struct OzParams {
    int ng, nrows, nk, s;
    int nJ;
    const int *E;
    double *chi;
    int *status;
};

// idesc: D = F32, A = B = BF16, both K-major, N = 256, M = 128
constexpr uint32_t kOzIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kOzBN >> 3) << 17) |
                              ((uint32_t)(kOzBM >> 4) << 24);

__global__ void __launch_bounds__(kOzThreads, 1) oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                               const __grid_constant__ CUtensorMap tmB, OzParams pr)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char *sm = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = sm;                                  // [stages][16 KB]
    unsigned char *sB = sA + kOzStages * kOzABytes;          // [stages][32 KB]
    uint64_t *full = (uint64_t *)(sB + kOzStages * kOzBBytes);
    uint64_t *empty = full + kOzStages;
    uint64_t *tfull = empty + kOzStages;
    uint64_t *tempty = tfull + 2;
    uint64_t *fin = tempty + 2;
    uint32_t *tslot = (uint32_t *)(fin + 1);
    int *Ecol = (int *)(tslot + 4);                          // [128] exponents of the tile's columns

    // tile (I, J): 128 real rows (64 complex) x 256 real columns (128 complex), with I <= 2J + 1
    const int nI = (pr.nrows + kOzBM - 1) / kOzBM;
    int rem = blockIdx.x, J = 0;
    for (;;) {
        const int c = min(2 * J + 2, nI);
        if (rem < c) break;
        rem -= c;
        ++J;
    }
    const int I = rem;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kOzStages; ++i) {
            bar_init(&full[i], 1);
            bar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            bar_init(&tfull[i], 1);
            bar_init(&tempty[i], 128);
        }
        bar_init(fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int c = threadIdx.x; c < 128; c += blockDim.x) {
        int g = J * 128 + c;
        Ecol[c] = g < pr.ng ? pr.E[g] : kOzNoColumn;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    const int s = pr.s, nk = pr.nk;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            for (int t = 2; t <= s + 1 && ok; ++t)
                for (int i = 1; i < t && ok; ++i) {
                    const int k = t - i;
                    for (int kb = 0; kb < nk; ++kb, ++it) {
                        const int st = it % kOzStages, n = it / kOzStages;
                        if (!bar_wait(&empty[st], (unsigned)((n & 1) ^ 1))) { ok = false; break; }
                        bar_expect(&full[st], kOzABytes + kOzBBytes);
                        tma3(sA + st * kOzABytes, &tmA, &full[st], kb * kOzBK, I * kOzBM, i - 1);
                        tma3(sB + st * kOzBBytes, &tmB, &full[st], kb * kOzBK, J * kOzBN, k - 1);
                    }
                }
            if (!ok) atomicOr(pr.status, kStatusTimeout);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0;
            for (int t = 2; t <= s + 1 && ok; ++t) {
                const int gi = t - 2, b = gi & 1, u = gi >> 1;
                if (!bar_wait(&tempty[b], (unsigned)((u & 1) ^ 1))) { ok = false; break; }
                tc_fence_after();
                const uint32_t d = tbase + (uint32_t)(b * kOzBN);
                bool first = true;
                for (int i = 1; i < t && ok; ++i)
                    for (int kb = 0; kb < nk; ++kb, ++it) {
                        const int st = it % kOzStages, n = it / kOzStages;
                        if (!bar_wait(&full[st], (unsigned)(n & 1))) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t a0 = su32(sA + st * kOzABytes), b0 = su32(sB + st * kOzBBytes);
#pragma unroll
                        for (int kk = 0; kk < kOzBK / 16; ++kk) {
                            umma(d, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), kOzIdesc, (first && kk == 0) ? 0u : 1u);
                        }
                        first = false;
                        umma_commit(&empty[st]);
                    }
                umma_commit(&tfull[b]);
            }
            // every issued MMA has completed before the block tears down
            umma_commit(fin);
            bar_wait(fin, 0);
            if (!ok) atomicOr(pr.status, kStatusTimeout);
        }
    } else {
        // epilogue: warps 2..5 -> TMEM lane quadrant (warp % 4), one tile row per thread
        const int q = warp & 3;
        const int r = q * 32 + lane;              // tile row (real index)
        const int g = I * 64 + (r >> 1);          // complex row G
        const int odd = r & 1;                    // 0: Re part, 1: Im part
        const int Eg = g < pr.ng ? pr.E[g] : kOzNoColumn;
        double *crow = pr.chi + 2 * ((int64_t)g * pr.ng) + odd;
        for (int t = 2; t <= s + 1; ++t) {
            const int gi = t - 2, b = gi & 1, u = gi >> 1;
            const bool got = bar_wait(&tfull[b], (unsigned)(u & 1));
            if (!__all_sync(0xffffffffu, got)) { ok = false; break; } // warp-uniform exit
            tc_fence_after();
            const uint32_t ta = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * kOzBN);
#pragma unroll 1
            for (int c0 = 0; c0 < kOzBN; c0 += 32) {
                uint32_t v[32];
                OZ_LD32(ta + c0, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int cc = 0; cc < 16; ++cc) {
                    const int ev = (int)__uint_as_float(v[2 * cc]);
                    const int od = (int)__uint_as_float(v[2 * cc + 1]);
                    const int rv = __shfl_xor_sync(0xffffffffu, od, 1);
                    const int val = odd ? (rv - ev) : (ev + rv);
                    const int cl = (c0 >> 1) + cc;    // complex column in the tile
                    const int gp = J * 128 + cl;
                    if (g < pr.ng && gp < pr.ng && g <= gp && val != 0) {
                        const int ex = Eg + Ecol[cl] - kOzBeta * t;
                        const double sc = -__longlong_as_double((long long)(1023 + max(-1022, ex)) << 52);
                        double *dst = crow + 2 * (int64_t)gp;
                        *dst = fma((double)val, sc, *dst);
                    }
                }
            }
            tc_fence_before();
            bar_arrive(&tempty[b]);
        }
        if (!ok) atomicOr(pr.status, kStatusTimeout);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512));
}

// ------------------------------------------------------------------ host launchers
int oz_tiles(int ng)
{
    const int nrows = 2 * ng;
    const int nI = (nrows + kOzBM - 1) / kOzBM, nJ = (nrows + kOzBN - 1) / kOzBN;
    int n = 0;
    for (int J = 0; J < nJ; ++J) n += std::min(2 * J + 2, nI);
    return n;
}

size_t oz_smem_bytes()
{
    return 1024 + kOzStages * (size_t)(kOzABytes + kOzBBytes) + (2 * kOzStages + 5) * 8 + 16 + 128 * 4;
}

cudaError_t launch_oz_sqrt(const double *delta, int64_t n, double *sp, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    oz_sqrt_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(delta, n, sp);
    return cudaGetLastError();
}

cudaError_t launch_oz_colexp(const double2 *M, int64_t P, int ng, const double *sp, int *E, cudaStream_t st)
{
    oz_fill_kernel<<<(ng + 255) / 256, 256, 0, st>>>(E, ng, kOzNoColumn);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || P == 0) return e;
    int gy = (int)std::min<int64_t>((P + 63) / 64, 256);
    oz_colexp_kernel<<<dim3((ng + 31) / 32, gy), 256, 0, st>>>(M, P, ng, sp, E);
    return cudaGetLastError();
}

cudaError_t launch_oz_slice(const double2 *M, int64_t P, int ng, const double *sp, const int *E, int s,
                            int64_t kpad, void *Z, cudaStream_t st)
{
    const size_t sm = (size_t)s * 64 * 72 * sizeof(uint16_t);
    cudaError_t e = cudaFuncSetAttribute(oz_slice_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    oz_slice_kernel<<<dim3((ng + 31) / 32, (unsigned)(kpad / 64)), 256, sm, st>>>(M, P, ng, sp, E, s, kpad,
                                                                                  (__nv_bfloat16 *)Z);
    return cudaGetLastError();
}

cudaError_t launch_oz_gemm(const CUtensorMap *tmA, const CUtensorMap *tmB, int ng, int64_t kpad, int s, const int *E,
                           double *chi, int *status, cudaStream_t st)
{
    OzParams pr;
    pr.ng = ng;
    pr.nrows = 2 * ng;
    pr.nk = (int)(kpad / kOzBK);
    pr.s = s;
    pr.nJ = (pr.nrows + kOzBN - 1) / kOzBN;
    pr.E = E;
    pr.chi = chi;
    pr.status = status;
    const size_t sm = oz_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    oz_gemm_kernel<<<oz_tiles(ng), kOzThreads, sm, st>>>(*tmA, *tmB, pr);
    return cudaGetLastError();
}

int oz_box_rows_a() { return kOzBM; }
int oz_box_rows_b() { return kOzBN; }
int oz_box_k() { return kOzBK; }

} // namespace gw
