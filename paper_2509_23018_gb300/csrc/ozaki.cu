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
// happens once per chunk and group, in the epilogue, with FP64 atomic adds so that the
// chunks (pair segments) of one chi block may run concurrently in one launch.  FP64 is kept for Delta, the
// scaling, the recombination, the accumulation across chunks and the symmetrisation.
#include "internal.h"
#include "ptx.cuh"
#include "fft_tf.cuh"
#include "oz_digits.cuh"
#include <cuda_bf16.h>
#include <algorithm>

namespace gw {

constexpr int kOzBeta = 6;
constexpr int kOzBM = 128, kOzBN = 256, kOzBK = 64, kOzStages = 4;
constexpr int kOzThreads = 192;
constexpr unsigned kOzABytes = kOzBM * kOzBK * 2, kOzBBytes = kOzBN * kOzBK * 2;
constexpr int kOzNoColumn = -400; // exponent of an all-zero column
// K-steps of one accumulation segment: 128 x 64 = 8192 real K entries, the length over which a
// slice group's FP32 sum is exact (|z_i z_k| <= 2^10, two products per entry for t = 3).  Longer
// K (the general product with more than 4096 complex inner entries) is summed segment by segment,
// each segment's groups recombined in FP64 by the epilogue.
constexpr int kOzKSeg = 128;

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
            const double2 m = M[p * ng + g];
            const double a = oz_bits_d(oz_absmax_bits(m.x, m.y)) * sp[p];
            e = max(e, oz_expo_pos(a, kOzNoColumn));
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
// A block forms the slices of a 64-pair x 32-column tile of M and stores them straight into
// Z[i][j][p] (j = 2 g + {Re, Im}, K-major rows of kpad pairs).  Thread roles: warp w takes tile
// rows 32 (w & 1) .. + 31 (lane = row: column g = row / 2, component row & 1) and pairs
// 16 (w >> 1) .. + 15, so a warp reads 32 consecutive doubles of M per pair, and each thread
// writes each slice's 16 digits of its row as one aligned 32-byte segment (two 16-byte stores).
struct OzTileThread {
    int row, gl, c, pl0;
};
__device__ __forceinline__ OzTileThread oz_tile_thread()
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    OzTileThread t;
    t.row = 32 * (w & 1) + lane;
    t.gl = t.row >> 1;
    t.c = t.row & 1;
    t.pl0 = 16 * (w >> 1);
    return t;
}

// the s slices of the 16 biased integers nb[t] = N_t + bias (consecutive pairs of one row) into
// out + i plane + [0, 16)
__device__ __forceinline__ void oz_store_row_digits(const long long nb[16], int s, __nv_bfloat16 *out, int64_t plane)
{
    for (int i = 0; i < s; ++i) {
        uint32_t w[8];
#pragma unroll
        for (int t = 0; t < 16; t += 2) {
            uint16_t d[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const long long v = nb[t + u];
                d[u] = i == 0 ? oz_small_bf16((int)(v >> (kOzBeta * (s - 1))))
                              : oz_small_bf16((int)((v >> (kOzBeta * (s - 1 - i))) & 63) - 32);
            }
            w[t >> 1] = (uint32_t)d[0] | ((uint32_t)d[1] << 16);
        }
        uint4 *o = (uint4 *)(out + i * plane);
        o[0] = make_uint4(w[0], w[1], w[2], w[3]);
        o[1] = make_uint4(w[4], w[5], w[6], w[7]);
    }
}

// Z[i][j][p] (bf16, K-major rows of length kpad) for a 64-pair x 32-column block.
// Five blocks per SM (48 registers, a 24-byte spill) keep more of the 16 loads per thread in flight
// than the four the unconstrained build allows: the split preparation of a 48^3 q-point (16 chunks)
// takes 5.04 against 5.32 ms (six blocks, 40 registers and a 60-byte spill: 5.17 ms).
__global__ void __launch_bounds__(256, 5) oz_slice_kernel(const double2 *__restrict__ M, int64_t P, int ng,
                                                       const double *__restrict__ spv, const int *__restrict__ E,
                                                       int s, int64_t kpad, __nv_bfloat16 *__restrict__ Z)
{
    const int64_t p0 = (int64_t)blockIdx.y * 64;
    const OzTileThread tt = oz_tile_thread();
    const int g = blockIdx.x * 32 + tt.gl;
    if (g >= ng) return;
    // N = round(a 2^(6 s - E)) and its balanced base-64 digits, in integer arithmetic
    const int sh = kOzBeta * s - E[g];
    const double *Md = (const double *)M;
    const long long bias = oz_digit_bias(s);
    long long nb[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        const int64_t p = p0 + tt.pl0 + t;
        const double a = p < P ? Md[2 * (p * ng + g) + tt.c] * spv[p] : 0.0;
        nb[t] = oz_round_scaled(a, sh) + bias;
    }
    const int64_t j = 2 * (int64_t)g + tt.c;
    oz_store_row_digits(nb, s, Z + j * kpad + p0 + tt.pl0, 2 * (int64_t)ng * kpad);
}

// ------------------------------------------------------------------ split for several frequencies
// The scale s_p(w) = sqrt(-Delta_p(w)) is the only thing that changes with the frequency, so a
// group of up to kOzGroupW frequencies shares one read of M: exponents E[w][g] in one pass,
// slices Z_w in another (each frequency's slices at Z + w zstride), the digits as in
// oz_slice_kernel.
constexpr int kOzGroupW = 8;

__global__ void __launch_bounds__(256) oz_colexp_multi_kernel(const double2 *__restrict__ M, int64_t P, int ng,
                                                              const double *__restrict__ sp, int64_t dstride,
                                                              int nw, int *__restrict__ E)
{
    __shared__ int red[8][32][kOzGroupW];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = blockIdx.x * 32 + lane;
    int e[kOzGroupW];
#pragma unroll
    for (int w = 0; w < kOzGroupW; ++w) e[w] = kOzNoColumn;
    if (g < ng) {
        for (int64_t p = (int64_t)blockIdx.y * 8 + wid; p < P; p += (int64_t)gridDim.y * 8) {
            const double2 m = M[p * ng + g];
            const double a0 = oz_bits_d(oz_absmax_bits(m.x, m.y));
#pragma unroll
            for (int w = 0; w < kOzGroupW; ++w)
                if (w < nw) {
                    const double a = a0 * sp[(int64_t)w * dstride + p];
                    e[w] = max(e[w], oz_expo_pos(a, kOzNoColumn));
                }
        }
    }
#pragma unroll
    for (int w = 0; w < kOzGroupW; ++w) red[wid][lane][w] = e[w];
    __syncthreads();
    if (wid == 0 && g < ng) {
#pragma unroll
        for (int w = 0; w < kOzGroupW; ++w)
            if (w < nw) {
                int v = red[0][lane][w];
                for (int k = 1; k < 8; ++k) v = max(v, red[k][lane][w]);
                atomicMax(E + (int64_t)w * ng + g, v);
            }
    }
}

__global__ void __launch_bounds__(256) oz_slice_multi_kernel(const double2 *__restrict__ M, int64_t P, int ng,
                                                             const double *__restrict__ spv, int64_t dstride, int nw,
                                                             const int *__restrict__ E, int s, int64_t kpad,
                                                             int64_t zstride, __nv_bfloat16 *__restrict__ Z)
{
    const int64_t p0 = (int64_t)blockIdx.y * 64;
    const OzTileThread tt = oz_tile_thread();
    const int g = blockIdx.x * 32 + tt.gl;
    if (g >= ng) return;
    const long long bias = oz_digit_bias(s);
    // the thread's 16 entries of the block's tile of M, read once for every frequency
    const double *Md = (const double *)M;
    double m[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        const int64_t p = p0 + tt.pl0 + t;
        m[t] = p < P ? Md[2 * (p * ng + g) + tt.c] : 0.0;
    }
    const int64_t j = 2 * (int64_t)g + tt.c;
    for (int w = 0; w < nw; ++w) {
        const int sh = kOzBeta * s - E[(int64_t)w * ng + g];
        long long nb[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int64_t p = p0 + tt.pl0 + t;
            const double a = p < P ? m[t] * spv[(int64_t)w * dstride + p] : 0.0;
            nb[t] = oz_round_scaled(a, sh) + bias;
        }
        oz_store_row_digits(nb, s, Z + w * zstride + j * kpad + p0 + tt.pl0, 2 * (int64_t)ng * kpad);
    }
}

// ------------------------------------------------------------------ general product: slices
// Y = A B with A split by rows and B by columns: x = 2^E sum_{i=1..s} 2^(-6 i) z_i, the same
// balanced base-64 digits as oz_slice_kernel, with E = max(ilogb) + 2 over a row of A or a
// column of B (both parts of a complex entry).
// exponent of a complex entry: ilogb(max(|Re|, |Im|)) + 2
__device__ __forceinline__ int oz_expo(double2 x)
{
    return oz_expo_bits(oz_absmax_bits(x.x, x.y), kOzNoColumn);
}

__device__ __forceinline__ void oz_digits(double x, int E, int s, uint16_t *out, int64_t plane)
{
    oz_store_digits(oz_round_scaled(x, kOzBeta * s - E), s, oz_digit_bias(s), out, plane);
}

__device__ __forceinline__ int oz_block_max(int e, int *red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if (lane == 0) red[wid] = e;
    __syncthreads();
    if (threadIdx.x < 32) {
        e = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : kOzNoColumn;
        for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
        if (threadIdx.x == 0) red[0] = e;
    }
    __syncthreads();
    return red[0];
}

// One block per row p of A [rows][ka] (complex): E[p], then Z[i][p][k], k = 2 g + {Re, Im},
// zero for k >= 2 ka.  CONJ: the rows of conj(A).
template <bool CONJ>
__global__ void __launch_bounds__(256) oz_split_rows_kernel(const double2 *__restrict__ A, int64_t rows, int ka,
                                                            int s, int64_t kpad, uint16_t *__restrict__ Z,
                                                            int *__restrict__ E)
{
    __shared__ int red[8];
    const int64_t p = blockIdx.x;
    const double2 *a = A + p * ka;
    int e = kOzNoColumn;
    for (int g = threadIdx.x; g < ka; g += blockDim.x) {
        const double2 x = a[g];
        e = max(e, oz_expo(x));
    }
    e = oz_block_max(e, red);
    if (threadIdx.x == 0) E[p] = e;
    uint16_t *zr = Z + p * kpad;
    for (int64_t k = threadIdx.x; k < kpad; k += blockDim.x) {
        const int g = (int)(k >> 1);
        const double x = g < ka ? ((k & 1) ? (CONJ ? -a[g].y : a[g].y) : a[g].x) : 0.0;
        oz_digits(x, e, s, zr + k, rows * kpad);
    }
}

// One block per column b of B [ka][nout] (complex): E[b], then rows 2b (Re of the product)
// and 2b + 1 (Im) of the real K-major operand B^T: row 2b = (Re B, -Im B), row 2b + 1 =
// (Im B, Re B) interleaved by g, so that [Re A, Im A] interleaved times them gives Re and
// Im of (A B)[p][b].
// B[g][b] is read at B[g sk + b sj] (sk = nout, sj = 1 for a row-major B; sk = 1, sj = ka for
// the transpose of a row-major [nout][ka] matrix).  CONJ: the columns of conj(B).
template <bool CONJ>
__global__ void __launch_bounds__(256) oz_split_cols_kernel(const double2 *__restrict__ B, int ka, int nout,
                                                            int64_t sk, int64_t sj, int s, int64_t kpad,
                                                            uint16_t *__restrict__ Z, int *__restrict__ E)
{
    __shared__ int red[8];
    const int b = blockIdx.x;
    int e = kOzNoColumn;
    for (int g = threadIdx.x; g < ka; g += blockDim.x) {
        const double2 x = B[(int64_t)g * sk + (int64_t)b * sj];
        e = max(e, oz_expo(x));
    }
    e = oz_block_max(e, red);
    if (threadIdx.x == 0) E[b] = e;
    const int64_t plane = (int64_t)2 * nout * kpad;
    uint16_t *z0 = Z + (int64_t)(2 * b) * kpad, *z1 = z0 + kpad;
    for (int64_t k = threadIdx.x; k < kpad; k += blockDim.x) {
        const int g = (int)(k >> 1);
        double x0 = 0.0, x1 = 0.0;
        if (g < ka) {
            double2 x = B[(int64_t)g * sk + (int64_t)b * sj];
            if (CONJ) x.y = -x.y;
            x0 = (k & 1) ? -x.y : x.x;
            x1 = (k & 1) ? x.x : x.y;
        }
        oz_digits(x0, e, s, z0 + k, plane);
        oz_digits(x1, e, s, z1 + k, plane);
    }
}

// ------------------------------------------------------------------ plasmon-pole prep. step, split
// The A operand of X^T = P^T conj(M_n)^T straight from the pole parameters, P never stored:
// P[g][c] = A[g][c] / (d - sgn wt[g][c]) with A = v Omega^2 / (2 wt) (gpp_setup_tf_kernel),
// d = E - E_n, sgn = -1 for an occupied band n and +1 for an empty one.  At / Wt hold A and wt
// transposed ([c][g]) in two-float form, so that row c of P^T is one contiguous row and the
// pole runs on the FP32 pipes.  One block per row c and up to kGppMaxE energies per launch,
// sharing each read of the row:
//  * pass 1, the row exponent per energy, from P in FP32 after the exact two-float subtraction
//    x = d - sgn wt (relative error ~2^-22 however close the pole), padded by 2^-10 so that the
//    exponent is never below the one of the exact maximum;
//  * pass 2, P = A conj(x) / |x|^2 in two-float arithmetic (the reciprocal by one Newton step,
//    relative error near 2^-46, below the 2^-42 the seven slices keep), then the balanced
//    base-64 digits of N = round(P 2^sh) in the layout of oz_split_rows_kernel, (Re P, Im P)
//    interleaved by g.  The digits are taken in FP32, where every step is exact: v = hi 2^sh
//    splits into t 2^24 + r (|r| <= 2^23), the low part L = rint(r) + rint(lo 2^sh) (|L| < 2^24)
//    gives four digits by q = rint(L / 64), d = L - 64 q, and t + q the rest.  N differs from
//    round((hi + lo) 2^sh) by one unit of the last digit at most; |d| <= 32 as before.
__device__ __forceinline__ tf tf_recip(tf d)
{
    const float r0 = __frcp_rn(d.hi);
    const tf p = tf_mul(d, tf{r0, 0.0f});
    const tf e = tf_sub(tf{1.0f, 0.0f}, p); // 1 - d r0, of order 2^-23
    return tf_fast2sum(r0, __fmul_rn(r0, e.hi));
}

__device__ __forceinline__ tcx gpp_pole_tf(float4 a4, float4 w4, tf d, float sgn)
{
    const tcx a{{a4.x, a4.y}, {a4.z, a4.w}};
    // x = d - sgn wt (sgn = +-1: exact negation)
    const tcx x{tf_sub(d, tf{sgn * w4.x, sgn * w4.y}), tf{-sgn * w4.z, -sgn * w4.w}};
    const tf den = tf_add(tf_mul(x.re, x.re), tf_mul(x.im, x.im));
    return tc_rmul(tc_mulc(x, a), tf_recip(den)); // conj(x) a / |x|^2
}

// max(|Re P|, |Im P|) in FP32 from the exact two-float x
__device__ __forceinline__ float gpp_pole_mag(float4 a4, float4 w4, tf d, float sgn)
{
    const float xr = tf_sub(d, tf{sgn * w4.x, sgn * w4.y}).hi, xi = -sgn * w4.z;
    const float r = __frcp_rn(__fmaf_rn(xr, xr, __fmul_rn(xi, xi)));
    const float pr = __fmaf_rn(a4.x, xr, __fmul_rn(a4.z, xi)), pi = __fmaf_rn(a4.z, xr, -__fmul_rn(a4.x, xi));
    return fmaxf(fabsf(pr), fabsf(pi)) * r;
}

__device__ __forceinline__ int tf_expo(float a)
{
    if (!(a > 0.0f)) return kOzNoColumn;
    const int be = (int)((__float_as_uint(a) >> 23) & 0xff);
    return (be == 0 ? -127 : be - 127) + 2;
}

__device__ __forceinline__ uint32_t bf16_pair(float lo, float hi)
{
    return (__float_as_uint(lo) >> 16) | (__float_as_uint(hi) & 0xffff0000u);
}

// Digits of round(v 2^sh) for v = Re P and Im P side by side (sc = (s1, s2), s1 s2 = 2^sh),
// stored as they come: slice i of row zr (u32 pairs, slice planes plane32 apart), element g.
__device__ __forceinline__ float tf_low(tf v, float s1, float s2, float &t)
{
    const float vh = __fmul_rn(__fmul_rn(v.hi, s1), s2);
    t = rintf(__fmul_rn(vh, 0x1p-24f));
    return __fadd_rn(rintf(__fmaf_rn(-0x1p24f, t, vh)), rintf(__fmul_rn(__fmul_rn(v.lo, s1), s2)));
}

__device__ __forceinline__ void tf_digits_store(tcx p, float s1, float s2, int s, uint32_t *zr, int64_t plane32,
                                                int64_t g)
{
    float tr, ti;
    float Lr = tf_low(p.re, s1, s2, tr), Li = tf_low(p.im, s1, s2, ti);
    for (int i = s - 1; i >= 1; --i) {
        if (i == s - 5) { // four digits taken from the low parts: carry into the high parts
            Lr = __fadd_rn(Lr, tr);
            Li = __fadd_rn(Li, ti);
        }
        const float qr = rintf(__fmul_rn(Lr, 0.015625f)), qi = rintf(__fmul_rn(Li, 0.015625f));
        zr[i * plane32 + g] = bf16_pair(__fmaf_rn(-64.0f, qr, Lr), __fmaf_rn(-64.0f, qi, Li));
        Lr = qr;
        Li = qi;
    }
    if (s <= 5) { // at most four digits taken: the high parts join the top digit (zero for s <= 4)
        Lr = __fadd_rn(Lr, tr);
        Li = __fadd_rn(Li, ti);
    }
    zr[g] = bf16_pair(Lr, Li);
}

template <int NE>
__global__ void __launch_bounds__(256, NE > 4 ? 3 : 4) gpp_prep_split_kernel(const float4 *__restrict__ At,
                                                                const float4 *__restrict__ Wt, int ng, GppEnergies en,
                                                                int cnt, float sgn, int s, int64_t kpad,
                                                                int64_t zstride, uint16_t *__restrict__ Z,
                                                                int *__restrict__ E)
{
    __shared__ int red[8][NE];
    __shared__ float2 dsm[NE];
    __shared__ float2 ssm[NE];
    const int c = blockIdx.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x < NE) {
        const tf t = tf_from(threadIdx.x < cnt ? en.d[threadIdx.x] : 0.0);
        dsm[threadIdx.x] = make_float2(t.hi, t.lo);
    }
    __syncthreads();
    const float4 *a = At + (int64_t)c * ng, *w = Wt + (int64_t)c * ng;
    float mx[NE];
#pragma unroll
    for (int j = 0; j < NE; ++j) mx[j] = 0.0f;
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        const float4 a4 = a[g], w4 = w[g];
#pragma unroll
        for (int j = 0; j < NE; ++j)
            if (j < cnt) mx[j] = fmaxf(mx[j], gpp_pole_mag(a4, w4, tf{dsm[j].x, dsm[j].y}, sgn));
    }
#pragma unroll
    for (int j = 0; j < NE; ++j) {
        float v = mx[j];
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) red[wid][j] = __float_as_int(v);
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
        float v = 0.0f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v = fmaxf(v, __int_as_float(red[k][threadIdx.x]));
        const int e = tf_expo(v * (1.0f + 0x1p-10f));
        E[(int64_t)threadIdx.x * ng + c] = e;
        // 2^sh in two factors, each inside the FP32 exponent range
        const int sh = max(-250, min(250, kOzBeta * s - e));
        ssm[threadIdx.x] = make_float2(__int_as_float((127 + sh / 2) << 23), __int_as_float((127 + sh - sh / 2) << 23));
    }
    __syncthreads();
    const int64_t plane = (int64_t)ng * kpad;
    for (int64_t g = threadIdx.x; g < kpad / 2; g += blockDim.x) {
        float4 a4 = make_float4(0.f, 0.f, 0.f, 0.f), w4 = make_float4(1.f, 0.f, 0.f, 0.f);
        if (g < ng) {
            a4 = a[g];
            w4 = w[g];
        }
        for (int j = 0; j < cnt; ++j) {
            // padding entries (g >= ng) have a = 0, so p = 0 there
            const tcx p = gpp_pole_tf(a4, w4, tf{dsm[j].x, dsm[j].y}, sgn);
            const float2 sc = ssm[j];
            tf_digits_store(p, sc.x, sc.y, s, (uint32_t *)(Z + j * zstride + (int64_t)c * kpad), plane >> 1, g);
        }
    }
}

// ------------------------------------------------------------------ tcgen05 GEMM
// Persistent and batched: a launch takes a table of jobs (one job = one chunk's slices
// for one chi block, each with its own N_G, tensor maps and exponents) and the list of
// their upper tiles; block b takes items b, b + gridDim.x, ... in the same order in every
// role, so the TMA producer warp, the MMA warp and the epilogue warps need no exchange
// beyond the mbarriers.  The tile width BN (128, 240 or 256 real columns) is chosen by the
// autotuner or by the wave count (oz_pick_bn); two BN-column FP32 accumulators in TMEM alternate
// between slice groups so the epilogue of group t overlaps the MMAs of group t+1.  At BN = 240 the
// accumulators sit 256 columns apart and the epilogue's last 32-column chunk is cut at BN.
template <int BN, int ST = kOzStages>
struct OzCfg {
    static constexpr int Stages = ST;                        // TMA ring depth
    static constexpr int BM = kOzBM;
    static constexpr int BNC = BN / 2;                       // complex columns per tile
    static constexpr unsigned ABytes = kOzBM * kOzBK * 2, BBytes = BN * kOzBK * 2;
    static constexpr uint32_t TmemBuf = BN > 128 ? 256 : 128; // TMEM columns per accumulator buffer
    static constexpr uint32_t TmemCols = 2 * TmemBuf;        // 256 or 512 (a power of two)
    // idesc: D = F32, A = B = BF16, both K-major, N = BN, M = 128
    static constexpr uint32_t Idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                      ((uint32_t)(kOzBM >> 4) << 24);
    static constexpr size_t Smem = 1024 + ST * (size_t)(ABytes + BBytes) + (2 * ST + 5) * 8 + 16;
};

// tile -> (I, J): J-major, rows I = 0 .. min((BNC (J+1) - 1)/64 + 1, nI) - 1
__device__ __forceinline__ void oz_tile_ij(int tile, int nI, int bnc, int &I, int &J)
{
    int rem = tile;
    J = 0;
    for (;;) {
        const int c = min((bnc * (J + 1) - 1) / 64 + 1, nI);
        if (rem < c) break;
        rem -= c;
        ++J;
    }
    I = rem;
}

// tile -> (I, J) for the general product: I-major (blocks that run together share A rows)
template <bool GEN, int BN>
__device__ __forceinline__ void oz_tile(const OzJob &jb, int tile, int &I, int &J)
{
    if constexpr (GEN) {
        const int nJ = (jb.rows_b + BN - 1) / BN;
        I = tile / nJ;
        J = tile - I * nJ;
    } else {
        oz_tile_ij(tile, (2 * jb.ng + kOzBM - 1) / kOzBM, BN / 2, I, J);
    }
}

__device__ __forceinline__ int oz_find_job(const OzJob *jobs, int njobs, int item)
{
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].item_start <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// GEN = false: the Hermitian contraction above (upper tiles, chi epilogue).  GEN = true:
// the general product out += A B (all tiles, each owned by one block, plain FP64 adds).
// ST: depth of the TMA ring (2 leaves shared memory for other kernels' blocks on the SM).
template <int BN, bool GEN, int ST = kOzStages>
__global__ void __launch_bounds__(kOzThreads, 1) oz_gemm_kernel(const OzJob *__restrict__ jobs, int njobs, int nitems,
                                                               int *status)
{
    using C = OzCfg<BN, ST>;
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char *sm = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = sm;                                  // [stages][ABytes]
    unsigned char *sB = sA + ST * C::ABytes;          // [stages][BBytes]
    uint64_t *full = (uint64_t *)(sB + ST * C::BBytes);
    uint64_t *empty = full + ST;
    uint64_t *tfull = empty + ST;
    uint64_t *tempty = tfull + 2;
    uint64_t *fin = tempty + 2;
    uint32_t *tslot = (uint32_t *)(fin + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < ST; ++i) {
            bar_init(&full[i], 1);
            bar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            bar_init(&tfull[i], 1);
            bar_init(&tempty[i], 128);
        }
        bar_init(fin, 1);
        bar_fence_init();
    }
    if (warp == 1) tmem_alloc(tslot, C::TmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                const OzJob &jb = jobs[oz_find_job(jobs, njobs, item)];
                int I, J;
                oz_tile<GEN, BN>(jb, item - jb.item_start, I, J);
                for (int k0 = 0; k0 < jb.nk && ok; k0 += kOzKSeg)
                for (int t = 2; t <= jb.s + 1 && ok; ++t)
                    for (int i = 1; i < t && ok; ++i)
                        for (int kb = k0; kb < min(jb.nk, k0 + kOzKSeg); ++kb, ++it) {
                            const int st = it % ST;
                            const uint32_t n = it / ST;
                            if (!bar_wait(&empty[st], (n & 1) ^ 1)) { ok = false; break; }
                            bar_expect(&full[st], C::ABytes + C::BBytes);
                            tma3(sA + st * C::ABytes, &jb.tmA, &full[st], (jb.kb0 + kb) * kOzBK, I * kOzBM, i - 1);
                            tma3(sB + st * C::BBytes, &jb.tmB, &full[st], (jb.kb0 + kb) * kOzBK, J * BN, t - i - 1);
                        }
            }
            if (!ok) atomicOr(status, kStatusTimeout);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t it = 0, grp = 0;
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                const OzJob &jb = jobs[oz_find_job(jobs, njobs, item)];
                for (int k0 = 0; k0 < jb.nk && ok; k0 += kOzKSeg)
                for (int t = 2; t <= jb.s + 1 && ok; ++t, ++grp) {
                    const uint32_t b = grp & 1, u = grp >> 1;
                    if (!bar_wait(&tempty[b], (u & 1) ^ 1)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t d = tbase + b * C::TmemBuf;
                    bool first = true;
                    for (int i = 1; i < t && ok; ++i)
                        for (int kb = k0; kb < min(jb.nk, k0 + kOzKSeg); ++kb, ++it) {
                            const int st = it % ST;
                            if (!bar_wait(&full[st], (it / ST) & 1)) { ok = false; break; }
                            tc_fence_after();
                            const uint32_t a0 = su32(sA + st * C::ABytes), b0 = su32(sB + st * C::BBytes);
#pragma unroll
                            for (int kk = 0; kk < kOzBK / 16; ++kk)
                                umma_f16(d, sdesc_sw128(a0 + kk * 32), sdesc_sw128(b0 + kk * 32), C::Idesc,
                                         (first && kk == 0) ? 0u : 1u);
                            first = false;
                            umma_commit(&empty[st]);
                        }
                    umma_commit(&tfull[b]);
                }
            }
            // every issued MMA has completed before the block tears down
            umma_commit(fin);
            bar_wait(fin, 0);
            if (!ok) atomicOr(status, kStatusTimeout);
        }
    } else {
        // epilogue: warps 2..5 -> TMEM lane quadrant (warp % 4), one tile row per thread
        const int q = warp & 3;
        const int r = q * 32 + lane;              // tile row
        uint32_t grp = 0;
        if constexpr (GEN) {
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                const OzJob &jb = jobs[oz_find_job(jobs, njobs, item)];
                int I, J;
                oz_tile<GEN, BN>(jb, item - jb.item_start, I, J);
                const int pr = I * kOzBM + r;     // output row
                const int Ea = pr < jb.rows_a ? __ldg(jb.E + pr) : kOzNoColumn;
                double *orow = jb.out + (int64_t)pr * jb.ldo;
                for (int k0 = 0; k0 < jb.nk && ok; k0 += kOzKSeg)
                for (int t = 2; t <= jb.s + 1; ++t, ++grp) {
                    const uint32_t b = grp & 1, u = grp >> 1;
                    const bool got = bar_wait(&tfull[b], u & 1);
                    if (!__all_sync(0xffffffffu, got)) { ok = false; break; } // warp-uniform exit
                    tc_fence_after();
                    const uint32_t ta = tbase + ((uint32_t)(q * 32) << 16) + b * C::TmemBuf;
#pragma unroll 1
                    for (int c0 = 0; c0 < BN; c0 += 32) {
                        uint32_t v[32];
                        GW_TMEM_LD32(ta + c0, v);
                        tmem_wait_ld();
                        if (pr < jb.rows_a) {
#pragma unroll
                            for (int cc = 0; cc < 32; ++cc) {
                                const int j = J * BN + c0 + cc; // output real column
                                const int val = (int)__uint_as_float(v[cc]);
                                if ((BN % 32 == 0 || c0 + cc < BN) && j < jb.rows_b && val != 0) {
                                    const int ex = Ea + __ldg(jb.E2 + (j >> 1)) - kOzBeta * t;
                                    // the tile belongs to this block alone: a plain add
                                    orow[j] += (double)val * __longlong_as_double((long long)(1023 + max(-1022, ex)) << 52);
                                }
                            }
                        }
                    }
                    tc_fence_before();
                    bar_arrive(&tempty[b]);
                }
            }
        } else {
            const int odd = r & 1;                    // 0: Re part, 1: Im part
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                const OzJob &jb = jobs[oz_find_job(jobs, njobs, item)];
                int I, J;
                oz_tile<GEN, BN>(jb, item - jb.item_start, I, J);
                const int ng = jb.ng;
                const int g = I * 64 + (r >> 1);      // complex row G
                const int Eg = g < ng ? __ldg(jb.E + g) : kOzNoColumn;
                double *crow = jb.chi + 2 * ((int64_t)g * ng) + odd;
                for (int k0 = 0; k0 < jb.nk && ok; k0 += kOzKSeg)
                for (int t = 2; t <= jb.s + 1; ++t, ++grp) {
                    const uint32_t b = grp & 1, u = grp >> 1;
                    const bool got = bar_wait(&tfull[b], u & 1);
                    if (!__all_sync(0xffffffffu, got)) { ok = false; break; } // warp-uniform exit
                    tc_fence_after();
                    const uint32_t ta = tbase + ((uint32_t)(q * 32) << 16) + b * C::TmemBuf;
#pragma unroll 1
                    for (int c0 = 0; c0 < BN; c0 += 32) {
                        uint32_t v[32];
                        GW_TMEM_LD32(ta + c0, v);
                        tmem_wait_ld();
#pragma unroll
                        for (int cc = 0; cc < 16; ++cc) {
                            const int ev = (int)__uint_as_float(v[2 * cc]);
                            const int od = (int)__uint_as_float(v[2 * cc + 1]);
                            const int rv = __shfl_xor_sync(0xffffffffu, od, 1);
                            const int val = odd ? (rv - ev) : (ev + rv);
                            const int gp = J * C::BNC + (c0 >> 1) + cc;
                            if ((BN % 32 == 0 || (c0 >> 1) + cc < C::BNC) && g < ng && gp < ng && g <= gp && val != 0) {
                                const int ex = Eg + __ldg(jb.E + gp) - kOzBeta * t;
                                const double sc = -__longlong_as_double((long long)(1023 + max(-1022, ex)) << 52);
                                // atomic: blocks of other pair segments may add into the same entry
                                atomicAdd(crow + 2 * (int64_t)gp, (double)val * sc);
                            }
                        }
                    }
                    tc_fence_before();
                    bar_arrive(&tempty[b]);
                }
            }
        }
        if (!ok) atomicOr(status, kStatusTimeout);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tbase, C::TmemCols);
}

// ------------------------------------------------------------------ host launchers
int oz_tiles(int ng, int bn)
{
    const int nrows = 2 * ng, bnc = bn / 2;
    const int nI = (nrows + kOzBM - 1) / kOzBM, nJ = (nrows + bn - 1) / bn;
    int n = 0;
    for (int J = 0; J < nJ; ++J) n += std::min((bnc * (J + 1) - 1) / 64 + 1, nI);
    return n;
}

size_t oz_smem_bytes(int bn, int stages)
{
    if (stages == 2) return bn == 128 ? OzCfg<128, 2>::Smem : bn == 240 ? OzCfg<240, 2>::Smem : OzCfg<256, 2>::Smem;
    return bn == 128 ? OzCfg<128>::Smem : bn == 240 ? OzCfg<240>::Smem : OzCfg<256>::Smem;
}

// Tile width of the Hermitian contraction without a tuned value: 240 or 256 real columns,
// whichever leaves less work on the busiest SM (tiles per SM rounded up, times the width).  At
// N_G = 2000 on 152 SMs, 294 tiles of 240 fill two waves to 97 % where 272 tiles of 256 fill them
// to 89 %.
int oz_pick_bn(int ng, int nsm)
{
    int best = 256;
    long long bestw = 0;
    for (int bn : {256, 240}) {
        const long long w = (long long)((oz_tiles(ng, bn) + nsm - 1) / nsm) * bn;
        if (bn == 256 || w < bestw) {
            best = bn;
            bestw = w;
        }
    }
    return best;
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

int oz_group_w() { return kOzGroupW; }

cudaError_t launch_oz_split_multi(const double2 *M, int64_t P, int ng, const double *sp, int64_t dstride, int nw,
                                  int *E, int s, int64_t kpad, void *Z, int64_t zstride, cudaStream_t st)
{
    if (nw < 1 || nw > kOzGroupW) return cudaErrorInvalidValue;
    oz_fill_kernel<<<(unsigned)(((int64_t)nw * ng + 255) / 256), 256, 0, st>>>(E, nw * ng, kOzNoColumn);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (P > 0) {
        const int gy = (int)std::min<int64_t>((P + 63) / 64, 256);
        oz_colexp_multi_kernel<<<dim3((ng + 31) / 32, gy), 256, 0, st>>>(M, P, ng, sp, dstride, nw, E);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    oz_slice_multi_kernel<<<dim3((ng + 31) / 32, (unsigned)(kpad / 64)), 256, 0, st>>>(
        M, P, ng, sp, dstride, nw, E, s, kpad, zstride, (__nv_bfloat16 *)Z);
    return cudaGetLastError();
}

cudaError_t launch_oz_slice(const double2 *M, int64_t P, int ng, const double *sp, const int *E, int s,
                            int64_t kpad, void *Z, cudaStream_t st)
{
    oz_slice_kernel<<<dim3((ng + 31) / 32, (unsigned)(kpad / 64)), 256, 0, st>>>(M, P, ng, sp, E, s, kpad,
                                                                                  (__nv_bfloat16 *)Z);
    return cudaGetLastError();
}

template <int BN, int ST>
static cudaError_t launch_oz_chi(const OzJob *jobs, int njobs, int nitems, int grid, int *status, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel<BN, false, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)OzCfg<BN, ST>::Smem);
    if (e != cudaSuccess) return e;
    oz_gemm_kernel<BN, false, ST><<<grid, kOzThreads, OzCfg<BN, ST>::Smem, st>>>(jobs, njobs, nitems, status);
    return cudaGetLastError();
}

cudaError_t launch_oz_gemm_jobs(int bn, const OzJob *jobs, int njobs, int nitems, int grid, int *status,
                                cudaStream_t st, int stages)
{
    if (nitems == 0) return cudaSuccess;
    if (stages == 2)
        return bn == 128   ? launch_oz_chi<128, 2>(jobs, njobs, nitems, grid, status, st)
               : bn == 240 ? launch_oz_chi<240, 2>(jobs, njobs, nitems, grid, status, st)
                           : launch_oz_chi<256, 2>(jobs, njobs, nitems, grid, status, st);
    return bn == 128   ? launch_oz_chi<128, kOzStages>(jobs, njobs, nitems, grid, status, st)
           : bn == 240 ? launch_oz_chi<240, kOzStages>(jobs, njobs, nitems, grid, status, st)
                       : launch_oz_chi<256, kOzStages>(jobs, njobs, nitems, grid, status, st);
}

cudaError_t launch_oz_split_rows(const double2 *A, int64_t rows, int ka, int s, int64_t kpad, void *ZA, int *EA,
                                 cudaStream_t st, bool conj)
{
    if (rows == 0) return cudaSuccess;
    if (conj) oz_split_rows_kernel<true><<<(unsigned)rows, 256, 0, st>>>(A, rows, ka, s, kpad, (uint16_t *)ZA, EA);
    else oz_split_rows_kernel<false><<<(unsigned)rows, 256, 0, st>>>(A, rows, ka, s, kpad, (uint16_t *)ZA, EA);
    return cudaGetLastError();
}

cudaError_t launch_oz_split_cols(const double2 *B, int ka, int nout, int64_t sk, int64_t sj, bool conj, int s,
                                 int64_t kpad, void *ZB, int *EB, cudaStream_t st)
{
    if (nout == 0) return cudaSuccess;
    if (conj) oz_split_cols_kernel<true><<<(unsigned)nout, 256, 0, st>>>(B, ka, nout, sk, sj, s, kpad, (uint16_t *)ZB, EB);
    else oz_split_cols_kernel<false><<<(unsigned)nout, 256, 0, st>>>(B, ka, nout, sk, sj, s, kpad, (uint16_t *)ZB, EB);
    return cudaGetLastError();
}

cudaError_t launch_gpp_prep_split(const float4 *At, const float4 *Wt, int ng, const double *d, int cnt, float sgn,
                                  int s, int64_t kpad, int64_t zstride, void *Z, int *E, cudaStream_t st)
{
    if (ng == 0 || cnt == 0) return cudaSuccess;
    if (cnt > kGppMaxE) return cudaErrorInvalidValue;
    GppEnergies en{};
    for (int j = 0; j < cnt; ++j) en.d[j] = d[j];
    if (cnt <= 4)
        gpp_prep_split_kernel<4><<<(unsigned)ng, 256, 0, st>>>(At, Wt, ng, en, cnt, sgn, s, kpad, zstride,
                                                               (uint16_t *)Z, E);
    else
        gpp_prep_split_kernel<kGppMaxE><<<(unsigned)ng, 256, 0, st>>>(At, Wt, ng, en, cnt, sgn, s, kpad, zstride,
                                                                      (uint16_t *)Z, E);
    return cudaGetLastError();
}

cudaError_t launch_oz_gemm_general(int bn, const OzJob *jobs, int njobs, int nitems, int grid, int *status,
                                   cudaStream_t st)
{
    if (nitems == 0) return cudaSuccess;
    cudaError_t e;
    if (bn == 128) {
        e = cudaFuncSetAttribute(oz_gemm_kernel<128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)OzCfg<128>::Smem);
        if (e != cudaSuccess) return e;
        oz_gemm_kernel<128, true><<<grid, kOzThreads, OzCfg<128>::Smem, st>>>(jobs, njobs, nitems, status);
    } else {
        e = cudaFuncSetAttribute(oz_gemm_kernel<256, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)OzCfg<256>::Smem);
        if (e != cudaSuccess) return e;
        oz_gemm_kernel<256, true><<<grid, kOzThreads, OzCfg<256>::Smem, st>>>(jobs, njobs, nitems, status);
    }
    return cudaGetLastError();
}

int oz_box_rows_a() { return kOzBM; }
int oz_box_k() { return kOzBK; }

} // namespace gw
