// Two-float pair kernel specialised for a slab shape N1 x N2 known at compile time
// (instantiated per grid in pair_tf_g*.cu so the translation units compile in parallel).
// It is the algorithm of pair_kernel_tf in mtxel.cu with constant index arithmetic.
#pragma once
#include "internal.h"
#include "fft_tf.cuh"

namespace gw {

constexpr int kPairThreads = 256;

// Grid-specialised version: slab dimensions N1 x N2 known at compile time.  Warp w owns
// slab lines [w N1/8, (w+1) N1/8) for the product and the i2 transform (private ping-pong
// regions A/B, __syncwarp between stages); the kept i2-frequencies land transposed in C;
// the block transforms the K2 columns along i1 (C <-> D); the i0 sum reads the result.
// One block barrier before the i1 transform and one after each of its stages.
template <int NPT, int N1, int N2>
__global__ void __launch_bounds__(kPairThreads, 2) pair_kernel_tf_ct(const float4 *__restrict__ psiv,
                                                                   const float4 *__restrict__ psic, int nc, int64_t p0,
                                                                   PairPlan pp, TfConsts kc, tf inv_nr,
                                                                   double2 *__restrict__ M)
{
    static_assert(N1 % (kPairThreads / 32) == 0, "slab rows must split evenly over the warps");
    constexpr int NW = kPairThreads / 32, LPW = N1 / NW; // warps, lines per warp
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int ns = N1 * N2;
    const int n0 = pp.n[0];
    const int K2 = pp.K2;
    float4 *A = (float4 *)smem, *B = A + ns, *C = B + ns, *D = C + K2 * N1;
    float4 *tw0 = D + K2 * N1, *tw1 = tw0 + n0, *tw2 = tw1 + N1;
    int *pos = (int *)(tw2 + N2); // pos[k2] = index of k2 among the kept i2-frequencies, or -1
    for (int i = threadIdx.x; i < n0; i += blockDim.x) tw0[i] = pp.ax[0].twf[i];
    for (int i = threadIdx.x; i < N1; i += blockDim.x) tw1[i] = pp.ax[1].twf[i];
    for (int i = threadIdx.x; i < N2; i += blockDim.x) {
        tw2[i] = pp.ax[2].twf[i];
        pos[i] = -1;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < K2; i += blockDim.x) pos[pp.kz[i]] = i;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t p = p0 + blockIdx.x;
    const int v = (int)(p / nc), c = (int)(p - (int64_t)v * nc);
    const int64_t nr = (int64_t)n0 * ns;
    const float4 *pv = psiv + (int64_t)v * nr + warp * LPW * N2;
    const float4 *pc = psic + (int64_t)c * nr + warp * LPW * N2;
    float4 *Aw = A + warp * LPW * N2, *Bw = B + warp * LPW * N2;

    tcx F[NPT];
    int sel[NPT], k0[NPT], e0[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        int g = threadIdx.x + j * kPairThreads;
        F[j] = {{0.f, 0.f}, {0.f, 0.f}};
        int pk = (g < pp.ng) ? pp.gpack[g] : 0;
        k0[j] = pk & 255;
        sel[j] = (pk >> 16) * N1 + ((pk >> 8) & 255);
        e0[j] = 0;
    }
    __syncthreads();

    constexpr int WPTS = LPW * N2;                     // points per warp
    constexpr int PER = (WPTS + 31) / 32;
    constexpr int PF = PER < 3 ? PER : 3;
    for (int i0 = 0; i0 < n0; ++i0) {
        const float4 *sv = pv + (int64_t)i0 * ns, *sc = pc + (int64_t)i0 * ns;
        if (i0 + 1 < n0) {
            // pull this warp's part of the next slab of both bands towards L2
            const char *nv = (const char *)(sv + ns), *nc2 = (const char *)(sc + ns);
            for (int o = lane * 128; o < WPTS * 16; o += 32 * 128) {
                asm volatile("prefetch.global.L2 [%0];" ::"l"(nv + o));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(nc2 + o));
            }
        }
        for (int i = lane; i < WPTS; i += PF * 32) {
            tcx xv[PF], xc[PF];
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                const int kk = i + u * 32;
                if (kk < WPTS) {
                    xv[u] = tc_load(sv + kk);
                    xc[u] = tc_load(sc + kk);
                }
            }
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                const int kk = i + u * 32;
                if (kk < WPTS) tc_store(Aw + kk, tc_mulc(xv[u], xc[u]));
            }
        }
        __syncwarp();
        // along i2 on this warp's lines; kept frequencies go to C as columns [k2'][i1]
        wstages_ct<N2, 0, 1, true>(Aw, Bw, LPW, N2, tw2, kc, pos, C, N1, warp * LPW);
        __syncthreads(); // C complete
        // along i1 on the K2 kept columns, the whole block on each stage (a column alone
        // would leave most lanes of a warp idle); ends with a barrier
        float4 *t = tfft_lines_ct<N1>(C, D, K2, N1, tw1, kc);
        constexpr bool in_d = (make_rad_plan(N1).nst & 1) != 0;
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            tcx u = tc_mul(tc_load(t + sel[j]), tc_load(tw0 + e0[j]));
            F[j] = tc_add(F[j], u);
            e0[j] += k0[j];
            if (e0[j] >= n0) e0[j] -= n0;
        }
        // With the result in D no barrier is needed here: the next slab writes A, B
        // (warp-private), C only in its last i2 stage, and D only after the next "C
        // complete" barrier.  With the result in C, C must not be rewritten before every
        // warp has read it.
        if constexpr (!in_d) __syncthreads();
    }
    double2 *out = M + (int64_t)blockIdx.x * pp.ng;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        int g = threadIdx.x + j * kPairThreads;
        if (g < pp.ng) out[g] = make_double2(tf_to_d(tf_mul(F[j].re, inv_nr)), tf_to_d(tf_mul(F[j].im, inv_nr)));
    }
}

template <int NPT, int N1, int N2>
inline cudaError_t launch_pair_tf_ct(const float4 *psiv, const float4 *psic, int nc, int64_t p0, int64_t count,
                                     const PairPlan &pp, const TfConsts &kc, tf inv_nr, double2 *M, cudaStream_t st)
{
    size_t sm = sizeof(float4) * (2 * (size_t)N1 * N2 + 2 * (size_t)pp.K2 * N1 + pp.n[0] + N1 + N2) + sizeof(int) * N2;
    cudaError_t e =
        cudaFuncSetAttribute(pair_kernel_tf_ct<NPT, N1, N2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    pair_kernel_tf_ct<NPT, N1, N2><<<(unsigned)count, kPairThreads, sm, st>>>(psiv, psic, nc, p0, pp, kc, inv_nr, M);
    return cudaGetLastError();
}

template <int N1, int N2>
inline cudaError_t launch_pair_tf_grid(const float4 *a, const float4 *b, int nc, int64_t p0, int64_t count,
                                       const PairPlan &pp, const TfConsts &kc, tf inv, double2 *M, cudaStream_t st)
{
    int need = (pp.ng + kPairThreads - 1) / kPairThreads;
    if (need <= 2) return launch_pair_tf_ct<2, N1, N2>(a, b, nc, p0, count, pp, kc, inv, M, st);
    if (need <= 4) return launch_pair_tf_ct<4, N1, N2>(a, b, nc, p0, count, pp, kc, inv, M, st);
    if (need <= 8) return launch_pair_tf_ct<8, N1, N2>(a, b, nc, p0, count, pp, kc, inv, M, st);
    if (need <= 12) return launch_pair_tf_ct<12, N1, N2>(a, b, nc, p0, count, pp, kc, inv, M, st);
    if (need <= 16) return launch_pair_tf_ct<16, N1, N2>(a, b, nc, p0, count, pp, kc, inv, M, st);
    if (need <= 24) return launch_pair_tf_ct<24, N1, N2>(a, b, nc, p0, count, pp, kc, inv, M, st);
    return launch_pair_tf_ct<32, N1, N2>(a, b, nc, p0, count, pp, kc, inv, M, st);
}


// Band setup in two-float arithmetic for a cubic N^3 grid: the (band, i0) slab kernel
// transforms along i2 then i1, the (band, i1) plane kernel along i0.
template <int N>
__global__ void __launch_bounds__(256) band_slab_tf_ct(float4 *__restrict__ psi, FftAxis ax, TfConsts kc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int ns = N * N;
    float4 *a = (float4 *)smem, *b = a + ns, *tw = b + ns;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = ax.twf[i];
    float4 *g = psi + ((int64_t)blockIdx.y * N + blockIdx.x) * ns;
    for (int i = threadIdx.x; i < ns; i += blockDim.x) a[i] = g[i];
    __syncthreads();
    float4 *r = tfft_lines_ct<N>(a, b, N, N, tw, kc);         // along i2
    float4 *o = (r == a) ? b : a;
    r = tfft_lines_ct<N>(r, o, N, 1, tw, kc, N);              // along i1 (element stride N)
    for (int i = threadIdx.x; i < ns; i += blockDim.x) g[i] = r[i];
}

template <int N>
__global__ void __launch_bounds__(256) band_axis0_tf_ct(float4 *__restrict__ psi, FftAxis ax, TfConsts kc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int np = N * N;
    float4 *a = (float4 *)smem, *b = a + np, *tw = b + np;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = ax.twf[i];
    float4 *g = psi + (int64_t)blockIdx.y * N * N * N + (int64_t)blockIdx.x * N;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const int i0 = i / N, i2 = i - i0 * N;
        a[i] = g[(int64_t)i0 * N * N + i2];
    }
    __syncthreads();
    float4 *r = tfft_lines_ct<N>(a, b, N, 1, tw, kc, N);      // lines along i0, element stride N
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const int i0 = i / N, i2 = i - i0 * N;
        g[(int64_t)i0 * N * N + i2] = r[i];
    }
}

template <int N>
inline cudaError_t launch_band_fft_tf_ct(float4 *psi, int nb, const FftAxis *ax, const TfConsts &kc,
                                         cudaStream_t st)
{
    const size_t sm = sizeof(float4) * (2 * (size_t)N * N + N);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(band_slab_tf_ct<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(band_axis0_tf_ct<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
            cudaSuccess)
        return e;
    band_slab_tf_ct<N><<<dim3(N, nb), 256, sm, st>>>(psi, ax[2], kc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    band_axis0_tf_ct<N><<<dim3(N, nb), 256, sm, st>>>(psi, ax[0], kc);
    return cudaGetLastError();
}

cudaError_t launch_band_fft_tf_g24(float4 *, int, const FftAxis *, const TfConsts &, cudaStream_t);
cudaError_t launch_band_fft_tf_g40(float4 *, int, const FftAxis *, const TfConsts &, cudaStream_t);
cudaError_t launch_band_fft_tf_g48(float4 *, int, const FftAxis *, const TfConsts &, cudaStream_t);
cudaError_t launch_band_fft_tf_g72(float4 *, int, const FftAxis *, const TfConsts &, cudaStream_t);

cudaError_t launch_pair_tf_g24(const float4 *, const float4 *, int, int64_t, int64_t, const PairPlan &,
                               const TfConsts &, tf, double2 *, cudaStream_t);
cudaError_t launch_pair_tf_g40(const float4 *, const float4 *, int, int64_t, int64_t, const PairPlan &,
                               const TfConsts &, tf, double2 *, cudaStream_t);
cudaError_t launch_pair_tf_g48(const float4 *, const float4 *, int, int64_t, int64_t, const PairPlan &,
                               const TfConsts &, tf, double2 *, cudaStream_t);
cudaError_t launch_pair_tf_g72(const float4 *, const float4 *, int, int64_t, int64_t, const PairPlan &,
                               const TfConsts &, tf, double2 *, cudaStream_t);

} // namespace gw
