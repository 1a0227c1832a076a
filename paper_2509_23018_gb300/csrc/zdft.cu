// Stage (a), last-axis transform of the pair products on the BF16 tensor cores.
//
// For a line l = (i0, i1) of the grid and a pair (v, c), the pruned transform of the pair
// product along the last axis at the kept frequencies kz[q] is
//     F[v][c][l][q] = sum_{i2} conj(psi_v[l][i2]) W_q[i2] psi_c[l][i2],   W_q[i2] = e^{+2 pi i kz[q] i2 / N},
// the first stage of the forward transform of the product (the definition after Eq. ff-ch).
// Over the pairs of a chunk it is, line by line, a complex matrix product whose operands
// belong to one band each: rows conj(psi_v[l]) (valence), columns W_q psi_c[l] (conduction).
// Written in real form (K = 2 N: Re and Im of each point interleaved), it runs as an
// Ozaki-style split product (the scheme of stage (b)):
//   * each operand row / column is scaled by its own power of two 2^E (|x| < 2^E) and cut into
//     six balanced base-256 digits, x = 2^E sum_{i<6} d_i 2^(-7-8i), |d_i| <= 128; a digit
//     times its scale is exact in BF16 (eight significant bits), so the slices carry their
//     scales and the tensor cores accumulate true values;
//   * the slice products i + j <= 5 are kept (the rest lies below 2^-48 of the operands'
//     scales); the products with i + j = 0, 1, 2 go to three FP32 accumulators of their own:
//     each of their terms is a multiple of one unit of that group with |sum| <= 3 * 96 * 2^14
//     < 2^24, so those sums are exact; i + j = 3..5 share a fourth accumulator (its rounding
//     lies 2^-48 below the leading group);
//   * the four accumulators are summed in two-float arithmetic (two-sums for the exact groups)
//     into F, which the pair kernel's remaining stages (middle and first axis) take from there.
// The valence slices are formed once per call (band setup); the conduction columns are formed
// per tile on the chip, from psi_c and the twiddles, by producer warps.
#include "internal.h"
#include "ptx.cuh"
#include "fft_tf.cuh"

#include <algorithm>

namespace gw {

// ------------------------------------------------------------------ digits
// Balanced base-256 digits of y = (h + l) 2^(7 - E), |y| < 128 (two-float value, exponent E):
// N = round(y 2^40) = T 2^24 + U with T, U exact FP32 integers, digits taken from the low end,
// each digit times its weight 2^(E - 7 - 8i) returned as the BF16 bits of slice i.
__device__ __forceinline__ void zd_digits(float h, float l, int E, uint16_t out[kZdSlices])
{
    // 2^(47 - E) in two factors so that each stays a normal FP32 for any E in [-100, 100]
    const int sh = 47 - E;
    const float s1 = __int_as_float((127 + sh / 2) << 23), s2 = __int_as_float((127 + sh - sh / 2) << 23);
    const float Y = __fmul_rn(__fmul_rn(h, s1), s2), L = __fmul_rn(__fmul_rn(l, s1), s2);
    const float T = rintf(__fmul_rn(Y, 0x1p-24f));
    float U = __fadd_rn(rintf(__fmaf_rn(-0x1p24f, T, Y)), rintf(L)); // |U| <= 2^24
    float d[kZdSlices];
#pragma unroll
    for (int i = kZdSlices - 1; i >= 3; --i) {
        const float q = rintf(__fmul_rn(U, 0.00390625f));
        d[i] = __fmaf_rn(-256.0f, q, U);
        U = q;
    }
    float V = __fadd_rn(T, U); // |V| < 2^23 + 2
#pragma unroll
    for (int i = 2; i >= 1; --i) {
        const float q = rintf(__fmul_rn(V, 0.00390625f));
        d[i] = __fmaf_rn(-256.0f, q, V);
        V = q;
    }
    d[0] = V;
    // weights: slice i holds d_i 2^(E - 7 - 8 i)
#pragma unroll
    for (int i = 0; i < kZdSlices; ++i) {
        const int e = E - 7 - 8 * i;
        const float w = __int_as_float((127 + max(-126, e)) << 23);
        out[i] = (uint16_t)(__float_as_uint(__fmul_rn(d[i], w)) >> 16);
    }
}

// The same digits with the line's scale sc = 2^(47 - E) and the slice weights w[i] = 2^(E - 7 - 8i)
// precomputed (-70 <= E <= 60, so that both stay normal FP32 numbers).
__device__ __forceinline__ void zd_digits_w(float h, float l, float sc, const float w[kZdSlices],
                                            uint16_t out[kZdSlices])
{
    const float Y = __fmul_rn(h, sc), L = __fmul_rn(l, sc);
    const float T = rintf(__fmul_rn(Y, 0x1p-24f));
    float U = __fadd_rn(rintf(__fmaf_rn(-0x1p24f, T, Y)), rintf(L));
    float d[kZdSlices];
#pragma unroll
    for (int i = kZdSlices - 1; i >= 3; --i) {
        const float q = rintf(__fmul_rn(U, 0.00390625f));
        d[i] = __fmaf_rn(-256.0f, q, U);
        U = q;
    }
    float V = __fadd_rn(T, U);
#pragma unroll
    for (int i = 2; i >= 1; --i) {
        const float q = rintf(__fmul_rn(V, 0.00390625f));
        d[i] = __fmaf_rn(-256.0f, q, V);
        V = q;
    }
    d[0] = V;
#pragma unroll
    for (int i = 0; i < kZdSlices; ++i) out[i] = (uint16_t)(__float_as_uint(__fmul_rn(d[i], w[i])) >> 16);
}

// exponent E with |x| < 2^E for a line's largest component magnitude m (E = -126 for m = 0)
__device__ __forceinline__ int zd_expo(float m)
{
    if (!(m > 0.0f)) return -126;
    const int be = (int)((__float_as_uint(m) >> 23) & 0xff);
    return (be == 0 ? -126 : be - 127) + 1;
}

// ------------------------------------------------------------------ valence slices
// A[i][l][v][k] (BF16, k = 2 i2 + {Re, Im}) of the rows psi_v[l][.]: one warp per (v, l).
__global__ void __launch_bounds__(256) zd_aslices_kernel(const float4 *__restrict__ psi, int nv, int n, int nlines,
                                                         uint16_t *__restrict__ A)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= nv * nlines) return;
    const int v = warp % nv, l = warp / nv;
    const float4 *row = psi + ((int64_t)v * nlines + l) * n;
    float m = 0.0f;
    for (int i = lane; i < n; i += 32) {
        const float4 x = row[i];
        m = fmaxf(m, fmaxf(fabsf(x.x), fabsf(x.z)) * (1.0f + 0x1p-20f));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int E = zd_expo(m);
    const int64_t plane = (int64_t)nlines * nv * 2 * n;
    uint16_t *dst = A + ((int64_t)l * nv + v) * 2 * n;
    for (int i = lane; i < n; i += 32) {
        const float4 x = row[i];
        uint16_t dr[kZdSlices], di[kZdSlices];
        zd_digits(x.x, x.y, E, dr);
        zd_digits(x.z, x.w, E, di);
#pragma unroll
        for (int s = 0; s < kZdSlices; ++s)
            *(uint32_t *)(dst + s * plane + 2 * i) = (uint32_t)dr[s] | ((uint32_t)di[s] << 16);
    }
}

cudaError_t launch_zd_aslices(const void *psiv, int nv, int n, uint16_t *A, cudaStream_t st)
{
    const int nlines = n * n;
    const int64_t warps = (int64_t)nv * nlines;
    zd_aslices_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>((const float4 *)psiv, nv, n, nlines, A);
    return cudaGetLastError();
}

__host__ __device__ __forceinline__ int zd_conduction_per_tile_d(int K2)
{
    const int ct = 128 / (2 * K2);
    return ct < 4 ? ct : 4;
}

// ------------------------------------------------------------------ the product
// One block per SM, persistent over units u = (line l, row tile mt); per unit the block keeps
// the valence slices of its 128 rows resident (three K-chunks of 32 real entries, TMA) and
// runs over the conduction tiles ct of the chunk (CT bands, 2 K2 real columns each, padded to
// 128 columns): producer warps form the tile's column slices in stages of 16 real entries into a
// 2-deep ring, one thread issues the tcgen05 products into four accumulators of 128 TMEM columns
// each, and the epilogue warps sum the accumulators into F.  A 128 x N x 16 product costs about
// the same time at N = 64 as at N = 128 (the probe's 128 x 64 rate is 2/3 of its 128 x 128 rate:
// feeding the 128 x 16 A operand sets the pace, whether A is read from shared memory or from TMEM),
// so the tile is 128 columns wide; its four accumulators then fill the 512 TMEM columns and are
// not double-buffered.  The epilogue hands them back as soon as its last TMEM loads have landed,
// before that chunk's arithmetic and stores.  (64-column tiles with two accumulator buffers took
// 2.40 against 2.30 ms per 48^3 chunk; eight epilogue warps of 16-column chunks 2.36 ms; a Re/Im
// column order without the producers' shared-memory store conflicts 2.34 ms.)
//  warp 0: TMA; warp 1: MMA (and TMEM); warps 2..5: epilogue (TMEM lane quadrant warp % 4);
//  warps 6..11: producers.
constexpr int kZdN = 128;                              // columns per tile
constexpr int kZdKC = 32;                              // real K entries per valence K-chunk
constexpr int kZdKB = 16;                              // real K entries per column stage
constexpr int kZdStages = 6;                           // column stages per tile (K = 96)
constexpr int kZdThreads = 384;
constexpr int kZdProducers = 6;                        // producer warps
constexpr unsigned kZdASlice = 128 * kZdKC * 2;        // one slice of one K-chunk: 8 KB
constexpr unsigned kZdAChunk = kZdSlices * kZdASlice;  // 48 KB
constexpr unsigned kZdBSlice = kZdN * kZdKB * 2;       // 4 KB
constexpr unsigned kZdBStage = kZdSlices * kZdBSlice;  // 24 KB
// idesc: D = F32, A = B = BF16, both K-major, N = 128, M = 128
constexpr uint32_t kZdIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kZdN >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);

// K-major operand tiles.  Valence slices (written by TMA), 64-byte swizzling: row r of 64 bytes
// (32 BF16), 8-row atoms of 512 bytes, 16-byte chunk j of row r stored at chunk j ^ ((r % 8) >> 1).
// Column stages (written by the producers), 32-byte swizzling: row r of 32 bytes (16 BF16), 8-row
// atoms of 256 bytes, chunk j of row r stored at chunk j ^ ((r % 8) >> 2).
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
__device__ __forceinline__ uint64_t sdesc_sw32(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(256 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)6 << 61);
}
__device__ __forceinline__ uint32_t sw32_off(int r, int k) // byte offset of element k (< 16) of row r
{
    return (uint32_t)((r >> 3) * 256 + (r & 7) * 32 + ((((k >> 3) ^ ((r & 7) >> 2)) & 1) << 4) + (k & 7) * 2);
}

__device__ __forceinline__ void tma4(void *dst, const CUtensorMap *m, uint64_t *b, int x, int y, int z, int w)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
                 "%5}], [%6];" ::"r"(su32(dst)),
                 "l"(m), "r"(x), "r"(y), "r"(z), "r"(w), "r"(su32(b))
                 : "memory");
}
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// two-sum with the sum's rounding error
__device__ __forceinline__ float zd_2sum(float a, float b, float &e)
{
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

constexpr int kZdPsiSlots = 4; // ring of conduction-band line tiles

struct ZdArgs {
    CUtensorMap tmA;        // A slices [6][lines][nv][2N] bf16, box {32, 128, 1, 6}, 64-byte swizzle
    CUtensorMap tmC;        // conduction grids as FP32 [nc][lines][4N], box {4N, 1, CT}
    const int *kz;          // [K2] kept last-axis frequencies
    float4 *F;              // [lines][R][K2] two-float, R = rows of the chunk = nv * cb, r = cl * nv + v
    int *status;
    int n, nv, c0, cb, K2, CT, nunits, nmt;
    // work items: units (line, row tile) 0 .. nfull - 1 whole, then each remaining unit split
    // into nsplit parts by conduction tiles (the last wave of the persistent blocks)
    int nct, nfull, nsplit, nitems;
};

// work item -> line l, row tile mt and conduction tiles [ct0, ct1)
__device__ __forceinline__ void zd_item(const ZdArgs &a, int item, int &l, int &mt, int &ct0, int &ct1)
{
    int unit = item, part = 0, np = 1;
    if (item >= a.nfull) {
        const int k = item - a.nfull;
        unit = a.nfull + k / a.nsplit;
        part = k - (k / a.nsplit) * a.nsplit;
        np = a.nsplit;
    }
    l = unit / a.nmt;
    mt = unit - l * a.nmt;
    ct0 = part * a.nct / np;
    ct1 = (part + 1) * a.nct / np;
}

__global__ void __launch_bounds__(kZdThreads, 1) zd_gemm_kernel(const __grid_constant__ ZdArgs a,
                                                                const float4 *__restrict__ twf)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char *sm = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = sm;                               // 3 K-chunks x 48 KB
    unsigned char *sB = sA + 3 * kZdAChunk;               // 2 stages x 24 KB
    float4 *ring = (float4 *)(sB + 2 * kZdBStage);        // [slots][CT][N] conduction line tiles
    float4 *wt = ring + kZdPsiSlots * a.CT * a.n;         // [K2][N] twiddles W^{kz[q] i2}
    int2 *ctab = (int2 *)(wt + a.K2 * a.n);               // [64] column pair -> (band, F offset)
    uint64_t *bar = (uint64_t *)(ctab + kZdN / 2);
    uint64_t *aFull = bar, *aEmpty = bar + 1, *bFull = bar + 2, *bEmpty = bar + 4, *tFull = bar + 6,
             *tEmpty = bar + 8, *fin = bar + 10, *pFull = bar + 11, *pEmpty = pFull + kZdPsiSlots;
    uint32_t *tslot = (uint32_t *)(pEmpty + kZdPsiSlots);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < a.K2 * a.n; i += blockDim.x) {
        const int q = i / a.n, i2 = i - q * a.n;
        wt[i] = twf[(a.kz[q] * i2) % a.n];
    }
    // the epilogue's column pairs (Re, Im of kept frequency q of band cl of the tile): cl and the
    // offset cl nv K2 + q of its F entry from the row's first (padding pairs: cl >= CT)
    for (int pi = threadIdx.x; pi < kZdN / 2; pi += blockDim.x) {
        const int cl = pi / a.K2, q = pi - cl * a.K2;
        ctab[pi] = make_int2(cl, cl * a.nv * a.K2 + q);
    }
    {
        // the padding columns of both stages stay zero (their products never reach F)
        const int ncol = 2 * a.K2, npad = kZdN - zd_conduction_per_tile_d(a.K2) * ncol;
        for (int e = threadIdx.x; e < 2 * kZdSlices * npad * (kZdKB / 2); e += blockDim.x) {
            const int st = e / (kZdSlices * npad * (kZdKB / 2)), r1 = e % (kZdSlices * npad * (kZdKB / 2));
            const int sl = r1 / (npad * (kZdKB / 2)), r2 = r1 % (npad * (kZdKB / 2));
            const int col = kZdN - npad + r2 / (kZdKB / 2), k = 2 * (r2 % (kZdKB / 2));
            *(uint32_t *)(sB + st * kZdBStage + sl * kZdBSlice + sw32_off(col, k)) = 0u;
        }
    }
    if (threadIdx.x == 0) {
        bar_init(aFull, 1);
        bar_init(aEmpty, 1);
        for (int i = 0; i < 2; ++i) {
            bar_init(&bFull[i], kZdProducers);
            bar_init(&bEmpty[i], 1);
            bar_init(&tFull[i], 1);
            bar_init(&tEmpty[i], 128);
        }
        bar_init(fin, 1);
        for (int i = 0; i < kZdPsiSlots; ++i) {
            bar_init(&pFull[i], 1);
            bar_init(&pEmpty[i], kZdProducers);
        }
        bar_fence_init();
    }
    if (warp == 1) tmem_alloc(tslot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    const int ncol = 2 * a.K2;                // real columns per conduction band
    bool ok = true;

    if (warp == 0) {
        // ---- TMA: the unit's valence slices, once the previous unit's products are done
        if (lane == 0) {
            uint32_t u = 0, tile = 0;
            const unsigned pbytes = (unsigned)a.CT * a.n * 16; // CT lines of N two-float points
            for (int item = blockIdx.x; item < a.nitems && ok; item += gridDim.x, ++u) {
                int l, mt, ct0, ct1;
                zd_item(a, item, l, mt, ct0, ct1);
                if (!bar_wait(aEmpty, (u & 1) ^ 1)) { ok = false; break; }
                bar_expect(aFull, 3 * kZdAChunk);
                for (int kc = 0; kc < 3; ++kc) tma4(sA + kc * kZdAChunk, &a.tmA, aFull, kc * kZdKC, mt * 128, l, 0);
                for (int ct = ct0; ct < ct1 && ok; ++ct, ++tile) {
                    const uint32_t ps = tile % kZdPsiSlots, pn = tile / kZdPsiSlots;
                    if (!bar_wait(&pEmpty[ps], (pn & 1) ^ 1)) { ok = false; break; }
                    bar_expect(&pFull[ps], pbytes);
                    tma3(ring + ps * a.CT * a.n, &a.tmC, &pFull[ps], 0, l, a.c0 + ct * a.CT);
                }
            }
            // every load has landed before the block may leave
            if (u > 0 && ok && !bar_wait(aFull, (u - 1) & 1)) ok = false;
            for (uint32_t t = tile > kZdPsiSlots ? tile - kZdPsiSlots : 0; t < tile && ok; ++t)
                if (!bar_wait(&pFull[t % kZdPsiSlots], (t / kZdPsiSlots) & 1)) ok = false;
            if (!ok) atomicOr(a.status, kStatusTimeout);
        }
    } else if (warp == 1) {
        // ---- MMA issue
        if (lane == 0) {
            // descriptor address fields count 16-byte units: offsets below 256 KB add in place
            const uint64_t ad0 = sdesc_sw64(su32(sA)), bd0 = sdesc_sw32(su32(sB));
            uint32_t u = 0, it = 0, tile = 0;
            for (int item = blockIdx.x; item < a.nitems && ok; item += gridDim.x, ++u) {
                int l, mt, ct0, ct1;
                zd_item(a, item, l, mt, ct0, ct1);
                if (!bar_wait(aFull, u & 1)) { ok = false; break; }
                for (int ct = ct0; ct < ct1 && ok; ++ct, ++tile) {
                    if (!bar_wait(&tEmpty[0], (tile & 1) ^ 1)) { ok = false; break; }
                    tc_fence_after();
                    for (int ks = 0; ks < kZdStages && ok; ++ks, ++it) {
                        const uint32_t st = it & 1;
                        if (!bar_wait(&bFull[st], (it >> 1) & 1)) { ok = false; break; }
                        tc_fence_after();
                        // the 21 products of the stage, unrolled: A is K-chunk ks / 2 from its
                        // 32-byte half ks % 2, descriptors advance by constant offsets, and a
                        // group's first product of the tile (stage 0, i = 0, j = group) starts its
                        // accumulator
                        const uint64_t ad = ad0 + (uint64_t)(((ks >> 1) * kZdAChunk + (ks & 1) * 32) >> 4);
                        const uint64_t bd = bd0 + (uint64_t)((st * kZdBStage) >> 4);
                        const uint32_t acc0 = ks > 0 ? 1u : 0u;
#pragma unroll
                        for (int i = 0; i < kZdSlices; ++i)
#pragma unroll
                            for (int j = 0; j < kZdSlices - i; ++j) {
                                const int g = i + j < 3 ? i + j : 3;
                                const bool first = i == 0 && j <= 3;
                                umma_f16(tbase + g * kZdN, ad + (uint64_t)((i * kZdASlice) >> 4),
                                         bd + (uint64_t)((j * kZdBSlice) >> 4), kZdIdesc, first ? acc0 : 1u);
                            }
                        umma_commit(&bEmpty[st]);
                    }
                    umma_commit(&tFull[0]);
                }
                umma_commit(aEmpty);
            }
            umma_commit(fin);
            bar_wait(fin, 0);
            if (!ok) atomicOr(a.status, kStatusTimeout);
        }
    } else if (warp < 6) {
        // ---- epilogue: one tile row (valence band) per thread
        const int q4 = warp & 3, r = q4 * 32 + lane;
        uint32_t tile = 0;
        for (int item = blockIdx.x; item < a.nitems && ok; item += gridDim.x) {
            int l, mt, ct0, ct1;
            zd_item(a, item, l, mt, ct0, ct1);
            const int v = mt * 128 + r;
            for (int ct = ct0; ct < ct1; ++ct, ++tile) {
                // F index of the row's first entry in this tile, and the bands the tile holds
                const int64_t rowbase = ((int64_t)l * a.cb * a.nv + (int64_t)ct * a.CT * a.nv + v) * a.K2;
                const int clmax = min(a.CT, a.cb - ct * a.CT);
                const bool got = bar_wait(&tFull[0], tile & 1);
                if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
                tc_fence_after();
                const uint32_t ta = tbase + ((uint32_t)(q4 * 32) << 16);
                const int cend = a.CT * ncol; // columns holding bands
#pragma unroll 1
                for (int c0 = 0; c0 < cend; c0 += 32) {
                    uint32_t g0[32], g1[32], g2[32], g3[32];
                    GW_TMEM_LD32(ta + 0 * kZdN + c0, g0);
                    GW_TMEM_LD32(ta + 1 * kZdN + c0, g1);
                    GW_TMEM_LD32(ta + 2 * kZdN + c0, g2);
                    GW_TMEM_LD32(ta + 3 * kZdN + c0, g3);
                    tmem_wait_ld();
                    if (c0 + 32 >= cend) {
                        // the accumulators are in registers: the next tile's products may start
                        tc_fence_before();
                        bar_arrive(&tEmpty[0]);
                    }
                    if (v < a.nv) {
#pragma unroll
                        for (int cc = 0; cc < 32; cc += 2) {
                            const int2 cp = ctab[(c0 + cc) >> 1]; // Re column c0 + cc, Im column + 1
                            if (cp.x < clmax) {
                                float x[2], y[2];
#pragma unroll
                                for (int p = 0; p < 2; ++p) {
                                    float e1, e2;
                                    const float s1 = zd_2sum(__uint_as_float(g0[cc + p]), __uint_as_float(g1[cc + p]), e1);
                                    const float s2 = zd_2sum(s1, __uint_as_float(g2[cc + p]), e2);
                                    const float t = __fadd_rn(__fadd_rn(e1, e2), __uint_as_float(g3[cc + p]));
                                    x[p] = __fadd_rn(s2, t);
                                    y[p] = __fsub_rn(t, __fsub_rn(x[p], s2));
                                }
                                const int64_t fi = rowbase + cp.y;
                                if (!GW_IN(fi, (int64_t)a.n * a.n * a.cb * a.nv * a.K2, a.status)) continue;
                                a.F[fi] = make_float4(x[0], y[0], x[1], y[1]);
                            }
                        }
                    }
                }
            }
        }
        if (!ok && lane == 0) atomicOr(a.status, kStatusTimeout);
    } else {
        // ---- producers: column slices of the conduction tile, stage by stage.  Lane (cl, k2) =
        // (lane / 8, lane % 8) owns the points i2 = 8 ks + k2 of band cl, loaded once per tile for
        // the six stages; producer warp pw forms the frequencies q = pw, pw + 6, ...
        const int pw = warp - 6;
        const int ncomb = a.CT * 8; // lanes holding a band (CT <= 4)
        const int cl = lane >> 3, k2 = lane & 7;
        uint32_t it = 0, tile = 0;
        for (int item = blockIdx.x; item < a.nitems && ok; item += gridDim.x) {
            int l, mt, ct0, ct1;
            zd_item(a, item, l, mt, ct0, ct1);
            for (int ct = ct0; ct < ct1 && ok; ++ct, ++tile) {
                // the tile's conduction lines, staged by the TMA warp
                const uint32_t ps = tile % kZdPsiSlots, pn = tile / kZdPsiSlots;
                const bool pgot = bar_wait(&pFull[ps], pn & 1);
                if (!__all_sync(0xffffffffu, pgot)) { ok = false; break; }
                const float4 *pl = ring + ps * a.CT * a.n;
                const int c = ct * a.CT + cl;
                float4 x[kZdStages];
                float m = 0.0f;
#pragma unroll
                for (int ks = 0; ks < kZdStages; ++ks) {
                    x[ks] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (lane < ncomb && c < a.cb) x[ks] = pl[cl * a.n + ks * 8 + k2];
                    m = fmaxf(m, (fabsf(x[ks].x) + fabsf(x[ks].z)) * (1.0f + 0x1p-20f));
                }
                // the 8 lanes of one band hold its whole line: the band's maximum
                for (int o = 4; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                const int E = max(-70, zd_expo(m)); // keeps the scale and every weight normal
                const float sc = __int_as_float((127 + 47 - E) << 23);
                float w[kZdSlices];
#pragma unroll
                for (int i = 0; i < kZdSlices; ++i) w[i] = __int_as_float((127 + E - 7 - 8 * i) << 23);
                __syncwarp();
                if (lane == 0) bar_arrive(&pEmpty[ps]); // the slot's values are in registers
#pragma unroll
                for (int ks = 0; ks < kZdStages; ++ks, ++it) {
                    if (!ok) continue;
                    const uint32_t st = it & 1;
                    const bool got = bar_wait(&bEmpty[st], ((it >> 1) & 1) ^ 1);
                    if (!__all_sync(0xffffffffu, got)) { ok = false; continue; } // warp-uniform exit
                    unsigned char *B = sB + st * kZdBStage;
                    if (lane < ncomb) {
                        const tcx xv = {{x[ks].x, x[ks].y}, {x[ks].z, x[ks].w}};
                        const float4 *wrow = wt + ks * 8 + k2;
                        for (int q = pw; q < a.K2; q += kZdProducers) {
                            const tcx b = tc_mul(xv, tc_load(wrow + q * a.n));
                            uint16_t dr[kZdSlices], di[kZdSlices];
                            zd_digits_w(b.re.hi, b.re.lo, sc, w, dr);
                            zd_digits_w(b.im.hi, b.im.lo, sc, w, di);
                            const int colr = cl * ncol + 2 * q;
                            if (!GW_IN(colr + 1, kZdN, a.status)) continue;
                            unsigned char *pr = B + sw32_off(colr, 2 * k2), *pi = B + sw32_off(colr + 1, 2 * k2);
#pragma unroll
                            for (int sl = 0; sl < kZdSlices; ++sl) {
                                // Re column: (Re b, Im b); Im column: (Im b, -Re b)
                                *(uint32_t *)(pr + sl * kZdBSlice) = (uint32_t)dr[sl] | ((uint32_t)di[sl] << 16);
                                *(uint32_t *)(pi + sl * kZdBSlice) = (uint32_t)di[sl] | ((uint32_t)(dr[sl] ^ 0x8000u) << 16);
                            }
                        }
                    }
                    fence_async_shared();
                    __syncwarp();
                    if (lane == 0) bar_arrive(&bFull[st]);
                }
            }
        }
        if (!ok && lane == 0) atomicOr(a.status, kStatusTimeout);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tbase, 512);
}

size_t zd_smem_bytes(int n, int K2)
{
    return 1024 + 3 * kZdAChunk + 2 * kZdBStage + 16 * (size_t)kZdPsiSlots * zd_conduction_per_tile_d(K2) * n +
           16 * (size_t)K2 * n +
           8 * (kZdN / 2) + 8 * 24 + 64;
}

// The route's shapes: 48-point lines (three valence K-chunks of 32 real entries, six column
// stages of 16), at most 32 kept frequencies, and the block's shared memory (valence slices,
// column stages, ring, twiddle table) within the 227 KB a block may opt into.
bool zd_supported(int n, int K2, int nv)
{
    return n == 48 && K2 >= 1 && K2 <= 32 && nv >= 1 && 2 * n == 3 * kZdKC && 2 * n == kZdStages * kZdKB &&
           zd_smem_bytes(n, K2) <= (size_t)227 * 1024;
}

int zd_conduction_per_tile(int K2) { return zd_conduction_per_tile_d(K2); }

cudaError_t launch_zd_gemm(const CUtensorMap &tmA, const CUtensorMap &tmC, const void *, const int *kz,
                           const float4 *twf, int n, int nv, int c0, int cb, int K2, float4 *F, int *status,
                           cudaStream_t st)
{
    ZdArgs a;
    a.tmA = tmA;
    a.tmC = tmC;
    a.kz = kz;
    a.F = F;
    a.status = status;
    a.n = n;
    a.nv = nv;
    a.c0 = c0;
    a.cb = cb;
    a.K2 = K2;
    a.CT = zd_conduction_per_tile(K2);
    a.nmt = (nv + 127) / 128;
    a.nunits = n * n * a.nmt;
    const size_t sm = zd_smem_bytes(n, K2);
    cudaError_t e = cudaFuncSetAttribute(zd_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    const int grid = std::min(a.nunits, sms);
    // the persistent blocks take items b, b + grid, ...: whole units while every block gets one,
    // then the rem remaining units in parts, so that the last wave ends evenly
    a.nct = (cb + a.CT - 1) / a.CT;
    a.nfull = a.nunits / grid * grid;
    const int rem = a.nunits - a.nfull;
    a.nsplit = rem > 0 ? std::max(1, std::min(a.nct, grid / rem)) : 1;
    a.nitems = a.nfull + rem * a.nsplit;
    zd_gemm_kernel<<<grid, kZdThreads, sm, st>>>(a, twf);
    return cudaGetLastError();
}

} // namespace gw
