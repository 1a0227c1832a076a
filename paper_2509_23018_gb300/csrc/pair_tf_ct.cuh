// Two-float pair kernel specialised for a slab shape N1 x N2 known at compile time
// (instantiated per grid in pair_tf_g*.cu so the translation units compile in parallel).
// It computes what pair_kernel_tf in mtxel.cu computes, organised for this GPU's FP32 pipes.
#pragma once
#include "internal.h"
#include "fft_tf.cuh"
#include "ptx.cuh"

namespace gw {

// Threads per block: warps own whole slab lines.  6 warps give every radix-4 stage of a
// 48-point line a full round of lanes (8 lines x 12 butterflies = 3 x 32); 5 warps of 8
// 40-point lines give the radix-5 stage two full rounds (8 x 8 = 2 x 32) and measured 18 %
// faster than 8 warps of 5 lines (27.5 vs 33.4 ms per 32768 pairs on 40^3).
template <int N>
constexpr int pair_threads()
{
    return N % 6 == 0 ? 192 : (N % 5 == 0 ? 160 : 256);
}
// Resident blocks per SM the register budget is sized for.
template <int N>
constexpr int pair_min_blocks()
{
    return N <= 48 ? (pair_threads<N>() == 256 ? 2 : 4) : 2;
}
// The second full i2 stage (when the plan has one) runs in place when a lane's inputs for
// all its butterflies fit in registers (at most 16 complex values): over all of a warp's L
// lines at once, or over the largest divisor of L that fits, subset by subset (the lines are
// independent).  Returns the lines per in-place pass, 0 when none fits (the stage then goes
// from A to a second slab buffer B).
template <int N>
constexpr int pair_inplace_lines()
{
    constexpr RadPlan P = make_prune_plan(N);
    constexpr int L = N / (pair_threads<N>() / 32);
    if (P.nst < 3) return L;
    for (int ls = L; ls >= 1; --ls)
        if (L % ls == 0 && ((ls * (N / P.r[1]) + 31) / 32) * P.r[1] <= 16) return ls;
    return 0;
}
template <int N>
constexpr bool pair_inplace()
{
    return pair_inplace_lines<N>() > 0;
}

// Lazy butterfly: outputs left unrenormalised where the radix has that form (they feed
// another lazy stage, whose sums renormalise).
template <int R>
__device__ __forceinline__ void tdft_lazy(tcx *v, const TfConsts &k)
{
    if constexpr (R == 4) tdft4<false>(v);
    else tdftR<R>(v, k);
}

// Warp-level full stage S >= 1 (radix R, NS) in place on the warp's L lines: every lane
// loads the inputs of all its butterflies, the warp synchronises, then all store.
template <int N, int R, int NS, int L>
__device__ __forceinline__ void wstage_inplace(float4 *x, const float4 *__restrict__ tw, const TfConsts &k)
{
    constexpr int nb = N / R, total = L * nb, rounds = (total + 31) / 32;
    constexpr int tstride = N / (NS * R);
    const int lane = threadIdx.x & 31;
    tcx v[rounds][R];
#pragma unroll
    for (int it = 0; it < rounds; ++it) {
        const int b = lane + 32 * it;
        if (total % 32 == 0 || b < total) {
            const int l = b / nb, j = b - l * nb;
#pragma unroll
            for (int r = 0; r < R; ++r) v[it][r] = tc_load(x + l * N + j + r * nb);
        }
    }
    __syncwarp();
#pragma unroll
    for (int it = 0; it < rounds; ++it) {
        const int b = lane + 32 * it;
        if (total % 32 == 0 || b < total) {
            const int l = b / nb, j = b - l * nb, kk = j % NS;
            const int e = kk * tstride;
#pragma unroll
            for (int r = 1; r < R; ++r) v[it][r] = tc_mull(v[it][r], tc_load(tw + r * e));
            tdft_lazy<R>(v[it], k);
            const int o = (j / NS) * (NS * R) + kk;
#pragma unroll
            for (int r = 0; r < R; ++r) tc_store(x + l * N + o + r * NS, v[it][r]);
        }
    }
}

// One block per pair on a cubic N^3 grid.
//  Pairs: with vgroup > 0 the chunk holds vgroup whole valence rows and block b takes
//  valence row b % vgroup, conduction band b / vgroup, so the blocks that read the same
//  conduction band run side by side and share its slabs in L2; otherwise pair p0 + b.
//  Phase 1, per i0 slab:
//   i2: warp w owns slab lines [w L, (w+1) L).  The first stage of make_prune_plan(N) is
//       fused with the product conj(psi_v) psi_c read from global memory and writes the
//       warp's part of A; a second full stage (when the plan has one) runs in place (or
//       A -> B); the pruned last stage forms only the K2 kept i2-frequencies, written
//       transposed into C[q][i1] (column stride N + 1).
//   i1: the block transforms the K2 columns (C <-> A, barrier after each stage); the
//       pruned last stage forms only the K12 (i1, i2) cells that hold sphere points and
//       stores them in the block's scratch slot, S[i0][cell] (global memory, L2-resident).
//  Phase 2: for batches of cells, the block loads S[.][cell] as lines along i0, runs the
//   pruned i0 transform and writes each sphere point's element straight into M.
//  Scratch slots: a pool larger than the number of blocks that can be resident at once;
//  a block claims a free slot with a bounded probe at its start and frees it at its end.
template <int N>
__global__ void __launch_bounds__(pair_threads<N>(), pair_min_blocks<N>())
    pair_kernel_tf_ct(const float4 *__restrict__ psiv, const float4 *__restrict__ psic, int nc, int64_t p0,
                      int vgroup, PairPlan pp, TfConsts kc, tf inv_nr, double2 *__restrict__ M)
{
    constexpr int NT = pair_threads<N>();
    static_assert(N % (NT / 32) == 0, "slab rows must split evenly over the warps");
    constexpr int L = N / (NT / 32); // lines per warp
    constexpr int CS = N + 1;        // column stride of C and of the i1 stages
    constexpr int ns = N * N;
    constexpr RadPlan P = make_prune_plan(N);
    static_assert(P.nst == 2 || P.nst == 3, "one or two full stages before the pruned one");
    constexpr int R0 = P.r[0], nb0 = N / R0;
    constexpr bool two = P.nst == 3, inplace = pair_inplace<N>();
    constexpr int sizeA = ns, sizeB = (two && !inplace) ? ns : 0;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int slot_s;
    const int K2 = pp.K2, K12 = pp.K12;
    const int sizeAB = sizeA + sizeB > K2 * CS ? sizeA + sizeB : K2 * CS; // A (+B) also serve the i1 stages
    float4 *A = (float4 *)smem, *B = A + sizeA, *C = A + sizeAB;
    float4 *tw = C + K2 * CS; // the three axes of a cubic grid share one table
    int *kz = (int *)(tw + N), *cell = kz + K2;
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = pp.ax[0].twf[i];
    for (int i = threadIdx.x; i < K2; i += NT) kz[i] = pp.kz[i];
    for (int i = threadIdx.x; i < K12; i += NT) cell[i] = pp.cell[i];
    if (threadIdx.x == 0) {
        int got = -1;
        int c = (int)((blockIdx.x * 2654435761u) % (unsigned)pp.nslots);
        for (int t = 0; t < pp.nslots; ++t) {
            if (atomicCAS(pp.slot_flags + c, 0, 1) == 0) {
                got = c;
                break;
            }
            if (++c == pp.nslots) c = 0;
        }
        slot_s = got;
    }
    __syncthreads();
    const int slot = slot_s;
    if (slot < 0) { // cannot happen with the pool sized by the occupancy; reported, not hung
        if (threadIdx.x == 0) atomicOr(pp.status, kStatusNoSlot);
        return;
    }
    float4 *S = pp.scr + (size_t)slot * N * K12;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = vgroup > 0 ? (int64_t)(blockIdx.x % vgroup) * nc + blockIdx.x / vgroup : blockIdx.x;
    const int64_t p = p0 + row;
    const int v = (int)(p / nc), c = (int)(p - (int64_t)v * nc);
    const int64_t nr = (int64_t)N * ns;
    const float4 *pv = psiv + (int64_t)v * nr + warp * L * N;
    const float4 *pc = psic + (int64_t)c * nr + warp * L * N;
    float4 *Aw = A + warp * L * N, *Bw = B + warp * L * N;
    // b -> (line, kept column) of the pruned i2 stage: b / K2 by multiply-high (b K2 < 2^32)
    const uint32_t magic = K2 > 1 ? 0xffffffffu / (uint32_t)K2 + 1u : 0u;

    for (int i0 = 0; i0 < N; ++i0) {
        const float4 *sv = pv + (int64_t)i0 * ns, *sc = pc + (int64_t)i0 * ns;
        if (i0 + 1 < N && lane == 0) {
            // bulk-prefetch this warp's part of the next slab of both bands into L2 (TMA unit)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(sv + ns), "r"(L * N * 16) : "memory");
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(sc + ns), "r"(L * N * 16) : "memory");
        }
        // i2, first stage fused with the product
        {
            constexpr int total = L * nb0, rounds = (total + 31) / 32;
#pragma unroll
            for (int it = 0; it < rounds; ++it) {
                const int b = lane + 32 * it;
                if (total % 32 == 0 || b < total) {
                    const int l = b / nb0, j = b - l * nb0;
                    const float4 *xv = sv + l * N + j, *xc = sc + l * N + j;
                    tcx x[R0];
#pragma unroll
                    for (int r = 0; r < R0; ++r) x[r] = tc_mulcl(tc_load(xv + r * nb0), tc_load(xc + r * nb0));
                    tdft_lazy<R0>(x, kc);
                    float4 *yl = Aw + l * N + j * R0;
#pragma unroll
                    for (int r = 0; r < R0; ++r) tc_store(yl + r, x[r]);
                }
            }
        }
        __syncwarp();
        if constexpr (two) {
            if constexpr (inplace) {
                constexpr int LS = pair_inplace_lines<N>();
#pragma unroll
                for (int l0 = 0; l0 < L; l0 += LS) wstage_inplace<N, P.r[1], R0, LS>(Aw + l0 * N, tw, kc);
            } else {
                wstage_ct<N, P.r[1], R0, L>(Aw, Bw, tw, kc);
            }
            __syncwarp();
        }
        // i2, pruned last stage: kept frequency kz[q] of line l -> C[q][warp L + l]
        const float4 *y2 = (two && !inplace) ? Bw : Aw;
        for (int b = lane; b < L * K2; b += 32) {
            const int l = K2 > 1 ? (int)__umulhi((uint32_t)b, magic) : b, q = b - l * K2;
            tc_store(C + q * CS + warp * L + l, tprune_ct<N>(y2 + l * N, kz[q], tw));
        }
        __syncthreads(); // C complete
        // i1 on the K2 columns; A (and B after it) are free until the next slab
        const float4 *y1 = tstages_ct<N, 0, 1, true, true>(C, A, K2, CS, tw, kc, 1);
        float4 *Si = S + (size_t)i0 * K12;
        for (int d = threadIdx.x; d < K12; d += NT) {
            const int cl = cell[d];
            if (!GW_IN((cl >> 8), K2, pp.status)) continue;
            tc_store(Si + d, tprune_ct<N>(y1 + (cl >> 8) * CS, cl & 255, tw));
        }
        __syncthreads(); // i1 done with C and A
    }
    __syncthreads(); // all slabs done: A and C become phase-2 buffers

    // Phase 2: i0 transforms of the cell columns, in batches that fit in A..C (lines of
    // stride N + 1, so the transposing stores from the scratch do not collide in banks)
    const int NB = (sizeAB + K2 * CS) / (2 * CS);
    float4 *X = A, *Y = A + NB * CS;
    double2 *out = M + row * pp.ng;
    for (int d0 = 0; d0 < K12; d0 += NB) {
        const int nbat = K12 - d0 < NB ? K12 - d0 : NB;
        {
            // element (x, dl) = i / nbat, i % nbat for i = threadIdx.x, threadIdx.x + NT, ...
            int x = (int)threadIdx.x / nbat, dl = (int)threadIdx.x - x * nbat;
            const int dx = NT / nbat, ddl = NT - dx * nbat;
            while (x < N) {
                X[dl * CS + x] = S[(size_t)x * K12 + d0 + dl];
                dl += ddl;
                x += dx;
                if (dl >= nbat) {
                    dl -= nbat;
                    ++x;
                }
            }
        }
        __syncthreads();
        const float4 *y0 = tstages_ct<N, 0, 1, true, true>(X, Y, nbat, CS, tw, kc, 1);
        const int m1 = pp.cstart[d0 + nbat];
        for (int m = pp.cstart[d0] + threadIdx.x; m < m1; m += NT) {
            const int2 pt = pp.cpts[m]; // point index, k0 | cell << 8
            if (!GW_IN(pt.x, pp.ng, pp.status) || !GW_IN((pt.y >> 8) - d0, nbat, pp.status)) continue;
            const tcx f = tprune_ct<N>(y0 + ((pt.y >> 8) - d0) * CS, pt.y & 255, tw);
            out[pt.x] = make_double2(tf_to_d(tf_mul(f.re, inv_nr)), tf_to_d(tf_mul(f.im, inv_nr)));
        }
        __syncthreads(); // before the next batch overwrites X and Y
    }
    if (threadIdx.x == 0) {
        __threadfence();
        atomicExch(pp.slot_flags + slot, 0);
    }
}

// Shared memory of pair_kernel_tf_ct<N> for a plan: A (+ B) (at least the i1 columns), C,
// the twiddle table, kz and the cell table (48^3 workload: 50 KB, 4 blocks per SM).
template <int N>
inline size_t pair_tf_ct_smem(const PairPlan &pp)
{
    constexpr RadPlan P = make_prune_plan(N);
    constexpr size_t ab = (size_t)N * N * ((P.nst == 3 && !pair_inplace<N>()) ? 2 : 1);
    const size_t cols = (size_t)pp.K2 * (N + 1);
    return sizeof(float4) * ((ab > cols ? ab : cols) + cols + N) + sizeof(int) * ((size_t)pp.K2 + pp.K12);
}

template <int N>
inline cudaError_t launch_pair_tf_cube(const float4 *psiv, const float4 *psic, int nc, int64_t p0, int64_t count,
                                       const PairPlan &pp, const TfConsts &kc, tf inv_nr, double2 *M, cudaStream_t st)
{
    const size_t sm = pair_tf_ct_smem<N>(pp);
    // whole valence rows: valence index fastest over the blocks (see the kernel)
    const int vgroup = (p0 % nc == 0 && count % nc == 0) ? (int)(count / nc) : 0;
    cudaError_t e = cudaFuncSetAttribute(pair_kernel_tf_ct<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(pp.slot_flags, 0, sizeof(int) * pp.nslots, st)) != cudaSuccess) return e;
    pair_kernel_tf_ct<N><<<(unsigned)count, pair_threads<N>(), sm, st>>>(psiv, psic, nc, p0, vgroup, pp, kc, inv_nr, M);
    return cudaGetLastError();
}

// Whether the grid-specialised kernel takes this plan: a cubic 24/40/48/72 grid and a
// shared-memory footprint within the 227 KB a block may opt into.
inline bool pair_tf_ct_fits(const PairPlan &pp)
{
    const int n = pp.n[0];
    if (pp.n[1] != n || pp.n[2] != n) return false;
    size_t sm;
    switch (n) {
    case 24: sm = pair_tf_ct_smem<24>(pp); break;
    case 40: sm = pair_tf_ct_smem<40>(pp); break;
    case 48: sm = pair_tf_ct_smem<48>(pp); break;
    case 72: sm = pair_tf_ct_smem<72>(pp); break;
    default: return false;
    }
    return sm <= 227 * 1024 - 64;
}

// The middle and first axes of the pair transform from the last-axis output F of the tensor-core
// stage (zdft.cu): one block per pair row r of the chunk.  The slabs go in pairs: the block
// transforms the 2 K2 columns of slabs i0 and i0 + 1 (F[i0 N + i1][r][q], the kept last-axis
// frequencies of every line) along i1 at once, two butterflies per thread per stage, and stores
// the K12 cells of each slab in its scratch slot.  Two buffers alternate: the i1 stages run X -> Y
// -> X, after which Y is free and receives the next pair of slabs while the pruned stage reads X;
// the next step starts from Y.  A slab pair's F arrives by one TMA load (tensor map over F as
// [lines][R K2] two-float entries, box of 2N lines x K2 entries) in line-major order, which the
// first i1 stage reads directly (tstage0_rows); every later stage works on the column layout.
// Phase 2 is that of pair_kernel_tf_ct.
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// L2 eviction-priority policies (per access, no device setting): the scratch cells are written
// once and read back once by the same block, the pool (SMs x blocks x 148 KB on 48^3) fits in L2,
// and the F stream passing through L2 beside it is read once
__device__ __forceinline__ uint64_t l2_policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void cp_async16_hint(void *dst, const void *src, uint64_t pol)
{
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st_hint(float4 *p, float4 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ float4 ld_hint(const float4 *p, uint64_t pol)
{
    float4 v;
    asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(pol)
                 : "memory");
    return v;
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void tma2_hint(void *dst, const CUtensorMap *m, uint64_t *b, int x, int y, uint64_t pol)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, "
                 "{%2, %3}], [%4], %5;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(m), "r"(x), "r"(y), "r"((uint32_t)__cvta_generic_to_shared(b)), "l"(pol)
                 : "memory");
}

// First stage (lazy radix 4, no twiddles: make_prune_plan(N)'s stage 0) of nlines lines stored
// row-major as a TMA box leaves them: line l = sl half + q (sl = 0 or 1) has its point k at
// x[(sl N + k) es + q].  The slab pair's F rows: half = K2, es = K2; a phase-2 batch of cells:
// half = nlines, es = the box width.  Output in the column layout y[l CS + k]; lines fastest
// over the threads (lm).
template <int N>
__device__ __forceinline__ void tstage0_rows(const float4 *__restrict__ x, float4 *__restrict__ y, int half, int es,
                                             int nlines, int CS, LMap lm)
{
    constexpr int R = make_prune_plan(N).r[0], nb = N / R;
    static_assert(R == 4, "the first stage is radix 4");
    int l = lm.l0, j = lm.j0;
    while (j < nb) {
        const int sl = l >= half ? 1 : 0;
        const float4 *xl = x + sl * N * es + (l - sl * half);
        tcx v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = tc_load(xl + (j + r * nb) * es);
        tdft4<false>(v);
        float4 *yl = y + l * CS + j * R;
#pragma unroll
        for (int r = 0; r < R; ++r) tc_store(yl + r, v[r]);
        l += lm.dl;
        j += lm.dj;
        if (l >= nlines) {
            l -= nlines;
            ++j;
        }
    }
}

// buffer of a slab pair's columns, in float4, rounded to 128 bytes (TMA destinations)
__host__ __device__ constexpr int from_f_buf(int ncols, int cs) { return (ncols * cs + 7) / 8 * 8; }

template <int N>
__global__ void __launch_bounds__(pair_threads<N>(), pair_min_blocks<N>())
    pair_kernel_tf_from_f(const __grid_constant__ CUtensorMap tmF, const __grid_constant__ CUtensorMap tmS, int64_t R,
                          PairPlan pp, TfConsts kc, tf inv_nr, double2 *__restrict__ M)
{
    static_assert(N % 2 == 0, "slabs go in pairs");
    static_assert(make_prune_plan(N).nst == 3, "two full i1 stages: the result returns to the input buffer");
    constexpr int NT = pair_threads<N>();
    constexpr int CS = N + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int slot_s;
    __shared__ uint64_t fbar; // a slab pair's F has landed
    const int K2 = pp.K2, K12 = pp.K12;
    const int ncols = 2 * K2;                  // columns of a slab pair
    const int BUF = from_f_buf(ncols, CS);
    float4 *Xb = (float4 *)(((uintptr_t)smraw + 127) & ~(uintptr_t)127); // [2][BUF]
    float4 *tw = Xb + 2 * BUF;
    int *cell = (int *)(tw + N);
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = pp.ax[0].twf[i];
    for (int i = threadIdx.x; i < K12; i += NT) cell[i] = pp.cell[i];
    if (threadIdx.x == 0) {
        bar_init(&fbar, 1);
        bar_fence_init();
        int got = -1;
        int c = (int)((blockIdx.x * 2654435761u) % (unsigned)pp.nslots);
        for (int t = 0; t < pp.nslots; ++t) {
            if (atomicCAS(pp.slot_flags + c, 0, 1) == 0) {
                got = c;
                break;
            }
            if (++c == pp.nslots) c = 0;
        }
        slot_s = got;
    }
    __syncthreads();
    const int slot = slot_s;
    if (slot < 0) {
        if (threadIdx.x == 0) atomicOr(pp.status, kStatusNoSlot);
        return;
    }
    float4 *S = pp.scr + (size_t)slot * N * K12;
    const int64_t row = blockIdx.x;
    // F of slabs i0, i0 + 1: lines i0 N .. i0 N + 2N - 1 of this row, K2 entries each (one TMA load;
    // the buffer's earlier readers have passed a barrier)
    const uint64_t keep = l2_policy_evict_last(), stream = l2_policy_evict_first();
    const unsigned fbytes = (unsigned)(2 * N * K2 * 16);
    auto fetch = [&](int i0, float4 *C) {
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            bar_expect(&fbar, fbytes);
            tma2_hint(C, &tmF, &fbar, (int)(row * K2 * 4), i0 * N, stream);
        }
    };
    const LMap lm = lmap_lines_fastest(ncols);
    fetch(0, Xb);
    uint32_t nf = 0;
    for (int i0 = 0, b = 0; i0 < N; i0 += 2, b ^= 1, ++nf) {
        float4 *X = Xb + b * BUF, *Y = Xb + (b ^ 1) * BUF;
        const bool late = !bar_wait(&fbar, nf & 1);
        if (__syncthreads_or(late)) { // X complete (or the wait ran out, for every thread alike)
            if (threadIdx.x == 0) atomicOr(pp.status, kStatusTimeout);
            return;
        }
        tstage0_rows<N>(X, Y, K2, K2, ncols, CS, lm);
        __syncthreads();
        const float4 *y1 = tstages_ct<N, 1, make_prune_plan(N).r[0], true, true>(Y, X, ncols, CS, tw, kc, 1, -1, lm);
        // y1 = X, after a barrier: Y is free
        if (i0 + 2 < N) fetch(i0 + 2, Y);
        for (int d = threadIdx.x; d < 2 * K12; d += NT) {
            const int sl = d >= K12, dd = d - sl * K12;
            const int cl = cell[dd];
            if (!GW_IN(cl >> 8, K2, pp.status)) continue;
            const tcx c = tprune_ct<N>(y1 + (sl * K2 + (cl >> 8)) * CS, cl & 255, tw);
            st_hint(S + (size_t)(i0 + sl) * K12 + dd, make_float4(c.re.hi, c.re.lo, c.im.hi, c.im.lo), keep);
        }
        __syncthreads(); // X read before the next step's first stage writes it
    }

    // Phase 2 (as in pair_kernel_tf_ct) in the two buffers: batches of NB cells of the slot, each one
    // TMA box of the scratch (tensor map over the slots as [nslots N rows][K12] entries, box
    // N x NB; cells past K12 read as zero), the next batch loaded while the current one is written
    // out.  The scratch was written by this block's generic stores: each thread orders its own
    // before the loads of the async proxy.
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    const int NB = ncols;
    const unsigned sbytes = (unsigned)(N * NB * 16);
    auto fetch_cells = [&](int d0, float4 *C) {
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            bar_expect(&fbar, sbytes);
            tma2_hint(C, &tmS, &fbar, d0 * 4, slot * N, stream);
        }
    };
    double2 *out = M + row * pp.ng;
    fetch_cells(0, Xb);
    for (int d0 = 0, b = 0; d0 < K12; d0 += NB, b ^= 1, ++nf) {
        float4 *X = Xb + b * BUF, *Y = Xb + (b ^ 1) * BUF;
        const int nbat = K12 - d0 < NB ? K12 - d0 : NB;
        const bool late = !bar_wait(&fbar, nf & 1);
        if (__syncthreads_or(late)) {
            if (threadIdx.x == 0) atomicOr(pp.status, kStatusTimeout);
            return;
        }
        const LMap lm2 = lmap_lines_fastest(nbat);
        tstage0_rows<N>(X, Y, nbat, NB, nbat, CS, lm2);
        __syncthreads();
        const float4 *y0 = tstages_ct<N, 1, make_prune_plan(N).r[0], true, true>(Y, X, nbat, CS, tw, kc, 1, -1, lm2);
        // y0 = X, after a barrier: Y is free
        if (d0 + NB < K12) fetch_cells(d0 + NB, Y);
        const int m1 = pp.cstart[d0 + nbat];
        for (int m = pp.cstart[d0] + threadIdx.x; m < m1; m += NT) {
            const int2 pt = pp.cpts[m];
            if (!GW_IN(pt.x, pp.ng, pp.status) || !GW_IN((pt.y >> 8) - d0, nbat, pp.status)) continue;
            const tcx f = tprune_ct<N>(y0 + ((pt.y >> 8) - d0) * CS, pt.y & 255, tw);
            out[pt.x] = make_double2(tf_to_d(tf_mul(f.re, inv_nr)), tf_to_d(tf_mul(f.im, inv_nr)));
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        atomicExch(pp.slot_flags + slot, 0);
    }
}

template <int N>
inline size_t pair_tf_from_f_smem(const PairPlan &pp)
{
    const int cs = N + 1, ncols = 2 * pp.K2;
    return 128 + sizeof(float4) * (2 * (size_t)from_f_buf(ncols, cs) + N) + sizeof(int) * (size_t)pp.K12;
}

template <int N>
inline cudaError_t launch_pair_tf_from_f_cube(const CUtensorMap &tmF, const CUtensorMap &tmS, int64_t R,
                                              const PairPlan &pp, const TfConsts &kc, tf inv_nr, double2 *M,
                                              cudaStream_t st)
{
    const size_t sm = pair_tf_from_f_smem<N>(pp);
    cudaError_t e =
        cudaFuncSetAttribute(pair_kernel_tf_from_f<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(pp.slot_flags, 0, sizeof(int) * pp.nslots, st)) != cudaSuccess) return e;
    pair_kernel_tf_from_f<N><<<(unsigned)R, pair_threads<N>(), sm, st>>>(tmF, tmS, R, pp, kc, inv_nr, M);
    return cudaGetLastError();
}

// Scratch slots the kernel needs for this plan: SMs x resident blocks + 32.
template <int N>
inline cudaError_t pair_tf_cube_slots(const PairPlan &pp, int *nslots)
{
    const size_t sm = pair_tf_ct_smem<N>(pp);
    cudaError_t e = cudaFuncSetAttribute(pair_kernel_tf_ct<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int occ = 0, dev = 0, nsm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pair_kernel_tf_ct<N>, pair_threads<N>(), sm)) !=
            cudaSuccess ||
        (e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if constexpr (N == 48) { // the pool also serves the kernel that starts from the tensor-core output
        const size_t sm2 = pair_tf_from_f_smem<N>(pp);
        int occ2 = 0;
        if ((e = cudaFuncSetAttribute(pair_kernel_tf_from_f<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sm2)) != cudaSuccess ||
            (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, pair_kernel_tf_from_f<N>, pair_threads<N>(),
                                                               sm2)) != cudaSuccess)
            return e;
        occ = occ > occ2 ? occ : occ2;
    }
    *nslots = nsm * (occ > 0 ? occ : 1) + 32;
    return cudaSuccess;
}

// Band setup in two-float arithmetic for a cubic N^3 grid: the (band, i0) slab kernel
// transforms along i2 then i1, the (band, i1) plane kernel along i0.
// Input pruning: the coefficients fill |G_a| <= m_a (m >= 0; -1: unknown), so slabs with
// |G_0| > m_0 are zero and stay zero, and in a slab the i2 lines with |G_1| > m_1 are zero.
template <int N>
__global__ void __launch_bounds__(256) band_slab_tf_ct(float4 *__restrict__ psi, FftAxis ax, TfConsts kc, int m0,
                                                       int m1)
{
    const int i0 = blockIdx.x;
    if (m0 >= 0 && (i0 <= N / 2 ? i0 : N - i0) > m0) return; // zero slab (the grid was zeroed)
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int ns = N * N;
    float4 *a = (float4 *)smem, *b = a + ns, *tw = b + ns;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = ax.twf[i];
    float4 *g = psi + ((int64_t)blockIdx.y * N + i0) * ns;
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
        a[i] = g[i];
        b[i] = make_float4(0.f, 0.f, 0.f, 0.f); // skipped lines stay zero in both buffers
    }
    __syncthreads();
    float4 *r = tfft_lines_ct<N>(a, b, N, N, tw, kc, 1, m1); // along i2, zero lines skipped
    float4 *o = (r == a) ? b : a;
    r = tfft_lines_ct<N, true>(r, o, N, 1, tw, kc, N);        // along i1 (element stride N)
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
    float4 *r = tfft_lines_ct<N, true>(a, b, N, 1, tw, kc, N); // lines along i0, element stride N
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const int i0 = i / N, i2 = i - i0 * N;
        g[(int64_t)i0 * N * N + i2] = r[i];
    }
}

template <int N>
inline cudaError_t launch_band_fft_tf_ct(float4 *psi, int nb, const FftAxis *ax, const TfConsts &kc, int m0, int m1,
                                         cudaStream_t st)
{
    const size_t sm = sizeof(float4) * (2 * (size_t)N * N + N);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(band_slab_tf_ct<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(band_axis0_tf_ct<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
            cudaSuccess)
        return e;
    band_slab_tf_ct<N><<<dim3(N, nb), 256, sm, st>>>(psi, ax[2], kc, m0, m1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    band_axis0_tf_ct<N><<<dim3(N, nb), 256, sm, st>>>(psi, ax[0], kc);
    return cudaGetLastError();
}

cudaError_t launch_band_fft_tf_g24(float4 *, int, const FftAxis *, const TfConsts &, int, int, cudaStream_t);
cudaError_t launch_band_fft_tf_g40(float4 *, int, const FftAxis *, const TfConsts &, int, int, cudaStream_t);
cudaError_t launch_band_fft_tf_g48(float4 *, int, const FftAxis *, const TfConsts &, int, int, cudaStream_t);
cudaError_t launch_band_fft_tf_g72(float4 *, int, const FftAxis *, const TfConsts &, int, int, cudaStream_t);

cudaError_t launch_pair_tf_g24(const float4 *, const float4 *, int, int64_t, int64_t, const PairPlan &,
                               const TfConsts &, tf, double2 *, cudaStream_t);
cudaError_t pair_tf_slots_g24(const PairPlan &, int *);
cudaError_t launch_pair_tf_g40(const float4 *, const float4 *, int, int64_t, int64_t, const PairPlan &,
                               const TfConsts &, tf, double2 *, cudaStream_t);
cudaError_t pair_tf_slots_g40(const PairPlan &, int *);
cudaError_t launch_pair_tf_g48(const float4 *, const float4 *, int, int64_t, int64_t, const PairPlan &,
                               const TfConsts &, tf, double2 *, cudaStream_t);
cudaError_t pair_tf_slots_g48(const PairPlan &, int *);
cudaError_t launch_pair_tf_g72(const float4 *, const float4 *, int, int64_t, int64_t, const PairPlan &,
                               const TfConsts &, tf, double2 *, cudaStream_t);
cudaError_t pair_tf_slots_g72(const PairPlan &, int *);
cudaError_t launch_pair_tf_from_f_g48(const CUtensorMap &, const CUtensorMap &, int64_t, const PairPlan &,
                                      const TfConsts &, tf, double2 *, cudaStream_t);

} // namespace gw
