// Two-float pair kernel specialised for a slab shape N1 x N2 known at compile time
// (instantiated per grid in pair_tf_g*.cu so the translation units compile in parallel).
// It computes what pair_kernel_tf in mtxel.cu computes, organised for this GPU's FP32 pipes.
#pragma once
#include "internal.h"
#include "fft_tf.cuh"

namespace gw {

// Threads per block: warps own whole slab lines, and 6 warps give every radix-4 stage of
// a 48-point line a full round of lanes (8 lines x 12 butterflies = 3 x 32).
template <int N1>
constexpr int pair_threads()
{
    return N1 % 6 == 0 ? 192 : 256;
}

// One block per pair, looping over the i0 slabs of the grid.  Per slab:
//  i2: warp w owns slab lines [w L, (w+1) L).  The first stage of make_prune_plan(N2) is
//      fused with the product conj(psi_v) psi_c read from global memory and writes the
//      warp's part of A; a second full stage (when the plan has one) goes A -> B; the
//      pruned last stage forms only the K2 kept i2-frequencies, written transposed into
//      C[q][i1] (column stride N1 + 1).
// Pairs: with vgroup > 0 the chunk holds vgroup whole valence rows and block b takes
// valence row b % vgroup, conduction band b / vgroup, so the blocks that read the same
// conduction band run side by side and share its slabs in L2; otherwise pair p0 + b.
//  i1: the block transforms the K2 columns (C <-> A, barrier after each stage); the
//      pruned last stage forms only the K12 (i1, i2) cells that hold sphere points, into T.
//  i0: each thread adds T[cell] W^{i0 k0} to its sphere points (direct sum over slabs).
//      Threads take the points in the order of pp.gorder (by k0, then cell), so the lanes
//      of a warp read the same twiddle and neighbouring cells.
// Barriers per slab: "C complete", one per full i1 stage, "T complete".
template <int NPT, int N1, int N2>
__global__ void __launch_bounds__(pair_threads<N1>(), NPT <= 12 ? 2 : 1)
    pair_kernel_tf_ct(const float4 *__restrict__ psiv, const float4 *__restrict__ psic, int nc, int64_t p0,
                      int vgroup, PairPlan pp, TfConsts kc, tf inv_nr, double2 *__restrict__ M)
{
    constexpr int NT = pair_threads<N1>();
    static_assert(N1 % (NT / 32) == 0, "slab rows must split evenly over the warps");
    constexpr int L = N1 / (NT / 32); // lines per warp
    constexpr int CS = N1 + 1;        // column stride of C and of the i1 stages
    constexpr int ns = N1 * N2;
    constexpr RadPlan P2 = make_prune_plan(N2);
    static_assert(P2.nst == 2 || P2.nst == 3, "one or two full i2 stages before the pruned one");
    constexpr int R0 = P2.r[0], nb0 = N2 / R0;
    constexpr bool two = P2.nst == 3;
    constexpr int sizeA = ns, sizeB = two ? ns : 0;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n0 = pp.n[0];
    const int K2 = pp.K2, K12 = pp.K12;
    const int sizeAB = sizeA + sizeB > K2 * CS ? sizeA + sizeB : K2 * CS; // A (+B) also serve the i1 stages
    float4 *A = (float4 *)smem, *B = A + sizeA, *C = A + sizeAB, *T = C + K2 * CS;
    float4 *tw0 = T + K12, *tw1 = tw0 + n0, *tw2 = tw1 + N1;
    int *kz = (int *)(tw2 + N2), *cell = kz + K2;
    for (int i = threadIdx.x; i < n0; i += NT) tw0[i] = pp.ax[0].twf[i];
    for (int i = threadIdx.x; i < N1; i += NT) tw1[i] = pp.ax[1].twf[i];
    for (int i = threadIdx.x; i < N2; i += NT) tw2[i] = pp.ax[2].twf[i];
    for (int i = threadIdx.x; i < K2; i += NT) kz[i] = pp.kz[i];
    for (int i = threadIdx.x; i < K12; i += NT) cell[i] = pp.cell[i];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = vgroup > 0 ? (int64_t)(blockIdx.x % vgroup) * nc + blockIdx.x / vgroup : blockIdx.x;
    const int64_t p = p0 + row;
    const int v = (int)(p / nc), c = (int)(p - (int64_t)v * nc);
    const int64_t nr = (int64_t)n0 * ns;
    const float4 *pv = psiv + (int64_t)v * nr + warp * L * N2;
    const float4 *pc = psic + (int64_t)c * nr + warp * L * N2;
    float4 *Aw = A + warp * L * N2, *Bw = B + warp * L * N2;
    // b -> (line, kept column) of the pruned i2 stage: b / K2 by multiply-high (b K2 < 2^32)
    const uint32_t magic = K2 > 1 ? 0xffffffffu / (uint32_t)K2 + 1u : 0u;

    tcx F[NPT];
    int gc[NPT], e0[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int s = threadIdx.x + j * NT;
        F[j] = {{0.f, 0.f}, {0.f, 0.f}};
        gc[j] = (s < pp.ng) ? pp.gcell[s] : 0; // k0 | cell << 8 of the point in slot s
        e0[j] = 0;
    }
    __syncthreads();

    for (int i0 = 0; i0 < n0; ++i0) {
        const float4 *sv = pv + (int64_t)i0 * ns, *sc = pc + (int64_t)i0 * ns;
        if (i0 + 1 < n0) {
            // bulk-prefetch this warp's part of the next slab of both bands into L2 (TMA unit)
            const char *nv = (const char *)(sv + ns), *nc2 = (const char *)(sc + ns);
            if (lane == 0) {
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(nv), "r"(L * N2 * 16) : "memory");
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(nc2), "r"(L * N2 * 16) : "memory");
            }
        }
        // i2, first stage fused with the product
        {
            constexpr int total = L * nb0, rounds = (total + 31) / 32;
#pragma unroll
            for (int it = 0; it < rounds; ++it) {
                const int b = lane + 32 * it;
                if (total % 32 == 0 || b < total) {
                    const int l = b / nb0, j = b - l * nb0;
                    const float4 *xv = sv + l * N2 + j, *xc = sc + l * N2 + j;
                    tcx x[R0];
#pragma unroll
                    for (int r = 0; r < R0; ++r) x[r] = tc_mulc(tc_load(xv + r * nb0), tc_load(xc + r * nb0));
                    tdftR<R0>(x, kc);
                    float4 *yl = Aw + l * N2 + j * R0;
#pragma unroll
                    for (int r = 0; r < R0; ++r) tc_store(yl + r, x[r]);
                }
            }
        }
        __syncwarp();
        // i2, second full stage and pruned last stage: kept frequency kz[q] of line l -> C[q][warp L + l]
        if constexpr (two) {
            wstage_ct<N2, P2.r[1], R0, L>(Aw, Bw, tw2, kc);
            __syncwarp();
        }
        const float4 *y2 = two ? Bw : Aw;
        for (int b = lane; b < L * K2; b += 32) {
            const int l = K2 > 1 ? (int)__umulhi((uint32_t)b, magic) : b, q = b - l * K2;
            tc_store(C + q * CS + warp * L + l, tprune_ct<N2>(y2 + l * N2, kz[q], tw2));
        }
        __syncthreads(); // C complete
        // i1 on the K2 columns; A (and B after it) are free until the next slab
        const float4 *y1 = tstages_ct<N1, 0, 1, true>(C, A, K2, CS, tw1, kc, 1);
        for (int d = threadIdx.x; d < K12; d += NT) {
            const int cl = cell[d];
            tc_store(T + d, tprune_ct<N1>(y1 + (cl >> 8) * CS, cl & 255, tw1));
        }
        __syncthreads(); // T complete
        // i0: direct sum over the slabs, lazy accumulation renormalised every 8 slabs
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            tc_acc(F[j], tc_load(T + (gc[j] >> 8)), tc_load(tw0 + e0[j]));
            e0[j] += gc[j] & 255;
            if (e0[j] >= n0) e0[j] -= n0;
            if ((i0 & 7) == 7) F[j] = tc_norm(F[j]);
        }
    }
    double2 *out = M + row * pp.ng;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int s = threadIdx.x + j * NT;
        const tcx f = tc_norm(F[j]);
        if (s < pp.ng)
            out[pp.gorder[s]] = make_double2(tf_to_d(tf_mul(f.re, inv_nr)), tf_to_d(tf_mul(f.im, inv_nr)));
    }
}

// Shared memory of pair_kernel_tf_ct for a plan: A (+ B) (at least the i1 columns), C, T,
// the three twiddle tables, kz and the cell table.
template <int N1, int N2>
inline size_t pair_tf_ct_smem(const PairPlan &pp)
{
    constexpr RadPlan P2 = make_prune_plan(N2);
    constexpr size_t ab = (size_t)N1 * N2 * (P2.nst == 3 ? 2 : 1);
    const size_t cols = (size_t)pp.K2 * (N1 + 1);
    return sizeof(float4) * ((ab > cols ? ab : cols) + cols + pp.K12 + pp.n[0] + N1 + N2) +
           sizeof(int) * ((size_t)pp.K2 + pp.K12);
}

template <int NPT, int N1, int N2>
inline cudaError_t launch_pair_tf_ct(const float4 *psiv, const float4 *psic, int nc, int64_t p0, int64_t count,
                                     const PairPlan &pp, const TfConsts &kc, tf inv_nr, double2 *M, cudaStream_t st)
{
    const size_t sm = pair_tf_ct_smem<N1, N2>(pp);
    // whole valence rows: valence index fastest over the blocks (see the kernel)
    const int vgroup = (p0 % nc == 0 && count % nc == 0) ? (int)(count / nc) : 0;
    cudaError_t e =
        cudaFuncSetAttribute(pair_kernel_tf_ct<NPT, N1, N2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    pair_kernel_tf_ct<NPT, N1, N2>
        <<<(unsigned)count, pair_threads<N1>(), sm, st>>>(psiv, psic, nc, p0, vgroup, pp, kc, inv_nr, M);
    return cudaGetLastError();
}

template <int N1, int N2>
inline cudaError_t launch_pair_tf_grid(const float4 *a, const float4 *b, int nc, int64_t p0, int64_t count,
                                       const PairPlan &pp, const TfConsts &kc, tf inv, double2 *M, cudaStream_t st)
{
    constexpr int NT = pair_threads<N1>();
    const int need = (pp.ng + NT - 1) / NT;
    if (need <= 2) return launch_pair_tf_ct<2, N1, N2>(a, b, nc, p0, count, pp, kc, inv, M, st);
    if (need <= 4) return launch_pair_tf_ct<4, N1, N2>(a, b, nc, p0, count, pp, kc, inv, M, st);
    if (need <= 8) return launch_pair_tf_ct<8, N1, N2>(a, b, nc, p0, count, pp, kc, inv, M, st);
    if (need <= 11) return launch_pair_tf_ct<11, N1, N2>(a, b, nc, p0, count, pp, kc, inv, M, st);
    if (need <= 16) return launch_pair_tf_ct<16, N1, N2>(a, b, nc, p0, count, pp, kc, inv, M, st);
    if (need <= 22) return launch_pair_tf_ct<22, N1, N2>(a, b, nc, p0, count, pp, kc, inv, M, st);
    if (need <= 32) return launch_pair_tf_ct<32, N1, N2>(a, b, nc, p0, count, pp, kc, inv, M, st);
    return cudaErrorInvalidValue;
}

// Whether the grid-specialised kernel takes this plan: at most 32 sphere points per thread
// and a shared-memory footprint within the 227 KB a block may opt into.
inline bool pair_tf_ct_fits(const PairPlan &pp)
{
    const int n1 = pp.n[1];
    if (pp.n[2] != n1) return false;
    size_t sm;
    switch (n1) {
    case 24: sm = pair_tf_ct_smem<24, 24>(pp); break;
    case 40: sm = pair_tf_ct_smem<40, 40>(pp); break;
    case 48: sm = pair_tf_ct_smem<48, 48>(pp); break;
    case 72: sm = pair_tf_ct_smem<72, 72>(pp); break;
    default: return false;
    }
    const int nt = n1 % 6 == 0 ? 192 : 256;
    return (pp.ng + nt - 1) / nt <= 32 && sm <= 227 * 1024;
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
