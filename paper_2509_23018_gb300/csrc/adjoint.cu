// Adjoint of L = Re Tr(W chi0) with respect to band energies and plane-wave coefficients.
//
// With m_p = M[p][:] (a row) and a Hermitian W, L = sum_p Delta_p q_p where
// q_p = sum_{G,G'} m_p(G) W[G][G'] conj(m_p(G')) (real).  Wirtinger calculus gives
//   dL/dDelta_p       = q_p = Re sum_G' Y_p(G') conj(m_p(G')),   Y = M W
//   dL/dconj(m_p(G')) = g_p(G') = Delta_p Y_p(G')
// and, through M_vc(G) = (1/N_r) sum_r conj(psi_v(r)) psi_c(r) e^{+iG.r},
//   dL/dconj(psi_c(r)) = psi_v(r) h_p(r),  dL/dconj(psi_v(r)) = psi_c(r) conj(h_p(r)),
//   h_p(r) = (1/N_r) sum_G g_p(G) e^{-iG.r},
// and through psi_n(r) = sum_K c_n(K) e^{+iK.r},
//   dL/dconj(c_n(K)) = sum_r psibar_n(r) e^{-iK.r}.
// Gradients are reported as dL/dRe + i dL/dIm = 2 dL/dconj.  Energies enter through
// x = E_v - E_c and dDelta/dx = 4 (w^2 - x^2) / (x^2 + w^2)^2.
// (GWPT's derivative of the self-energy, Eq. gwpt, is what motivates this sensitivity.)
#include "internal.h"
#include "fft.cuh"
#include "fft_tf.cuh"

#include <algorithm>

namespace gw {

// ------------------------------------------------------------------ Y = M W (FP64 DMMA)
// C[m][n] = sum_k A[m][k] B[k][n], complex row-major A [mr x kd], B [kd x nc], C [mr x nc].
constexpr int kGT = 64, kGK = 16;

__device__ __forceinline__ void dmma8(double &d0, double &d1, double a, double b)
{
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(d0), "+d"(d1)
                 : "d"(a), "d"(b));
}

// CA: conj(A) in place of A.  TB: B given as its transpose, row-major [nc][kd].  ACC: C += A B.
template <bool CA, bool TB, bool ACC>
__global__ void __launch_bounds__(256) zgemm_kernel(const double2 *__restrict__ A, const double2 *__restrict__ B,
                                                    double2 *__restrict__ C, int64_t mr, int kd, int nc)
{
    __shared__ double2 sa[kGT][kGK + 1];   // [m][k]
    __shared__ double2 sb[kGK][kGT + 1];   // [k][n]
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int wm = wid & 1, wn = wid >> 1;
    const int64_t m0 = (int64_t)blockIdx.y * kGT;
    const int n0 = blockIdx.x * kGT;
    double cre[4][2][2] = {}, cim[4][2][2] = {};
    for (int k0 = 0; k0 < kd; k0 += kGK) {
        for (int e = tid; e < kGT * kGK; e += blockDim.x) {
            int r = e / kGK, k = e % kGK;
            int64_t gm = m0 + r;
            int gk = k0 + k;
            double2 x = (gm < mr && gk < kd) ? A[gm * kd + gk] : make_double2(0.0, 0.0);
            if (CA) x.y = -x.y;
            sa[r][k] = x;
        }
        for (int e = tid; e < kGK * kGT; e += blockDim.x) {
            if (TB) {
                int n = e / kGK, k = e % kGK;
                int gk = k0 + k, gn = n0 + n;
                sb[k][n] = (gk < kd && gn < nc) ? B[(int64_t)gn * kd + gk] : make_double2(0.0, 0.0);
            } else {
                int k = e / kGT, n = e % kGT;
                int gk = k0 + k, gn = n0 + n;
                sb[k][n] = (gk < kd && gn < nc) ? B[(int64_t)gk * nc + gn] : make_double2(0.0, 0.0);
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK / 4; ++kk) {
            const int k = kk * 4 + (lane & 3);
            double ar[4], ai[4], nai[4], br[2], bi[2];
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
                double2 x = sa[wm * 32 + mt * 8 + (lane >> 2)][k];
                ar[mt] = x.x;
                ai[mt] = x.y;
                nai[mt] = -x.y;
            }
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                double2 x = sb[k][wn * 16 + nt * 8 + (lane >> 2)];
                br[nt] = x.x;
                bi[nt] = x.y;
            }
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    // (ar + i ai)(br + i bi) = (ar br - ai bi) + i (ar bi + ai br)
                    dmma8(cre[mt][nt][0], cre[mt][nt][1], ar[mt], br[nt]);
                    dmma8(cre[mt][nt][0], cre[mt][nt][1], nai[mt], bi[nt]);
                    dmma8(cim[mt][nt][0], cim[mt][nt][1], ar[mt], bi[nt]);
                    dmma8(cim[mt][nt][0], cim[mt][nt][1], ai[mt], br[nt]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
        const int64_t gm = m0 + wm * 32 + mt * 8 + (lane >> 2);
        if (gm >= mr) continue;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int gn = n0 + wn * 16 + nt * 8 + 2 * (lane & 3) + q;
                if (gn < nc) {
                    double2 v = make_double2(cre[mt][nt][q], cim[mt][nt][q]);
                    if (ACC) {
                        const double2 o = C[gm * nc + gn];
                        v.x += o.x;
                        v.y += o.y;
                    }
                    C[gm * nc + gn] = v;
                }
            }
    }
}

cudaError_t launch_zgemm(const double2 *A, const double2 *B, double2 *C, int64_t mr, int kd, int nc, cudaStream_t st)
{
    if (mr == 0 || nc == 0) return cudaSuccess;
    dim3 grid((nc + kGT - 1) / kGT, (unsigned)((mr + kGT - 1) / kGT));
    zgemm_kernel<false, false, false><<<grid, 256, 0, st>>>(A, B, C, mr, kd, nc);
    return cudaGetLastError();
}

cudaError_t launch_zgemm_ex(const double2 *A, const double2 *B, double2 *C, int64_t mr, int kd, int nc, bool conj_a,
                            bool trans_b, bool accumulate, cudaStream_t st)
{
    if (mr == 0 || nc == 0) return cudaSuccess;
    dim3 grid((nc + kGT - 1) / kGT, (unsigned)((mr + kGT - 1) / kGT));
    if (conj_a && !trans_b && !accumulate) zgemm_kernel<true, false, false><<<grid, 256, 0, st>>>(A, B, C, mr, kd, nc);
    else if (!conj_a && trans_b && accumulate) zgemm_kernel<false, true, true><<<grid, 256, 0, st>>>(A, B, C, mr, kd, nc);
    else if (!conj_a && !trans_b && !accumulate) zgemm_kernel<false, false, false><<<grid, 256, 0, st>>>(A, B, C, mr, kd, nc);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ per-pair reductions
// One warp per pair: q_p = Re sum_G Y conj(M); g_p = Delta_p Y_p written over Y;
// L, dE_v, dE_c accumulated with atomics.
__global__ void adj_rows_kernel(const double2 *__restrict__ M, double2 *__restrict__ Y, int64_t P, int ng, int nc,
                                int64_t p0, const double *__restrict__ ev, const double *__restrict__ ec, double w,
                                double *__restrict__ Lacc, double *__restrict__ dEv, double *__restrict__ dEc)
{
    const int lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= P) return;
    const double2 *m = M + p * ng;
    double2 *y = Y + p * ng;
    double q = 0.0;
    for (int g = lane; g < ng; g += 32) {
        double2 a = y[g], b = m[g];
        q = fma(a.x, b.x, fma(a.y, b.y, q));
    }
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    const int64_t pg = p0 + p;
    const int v = (int)(pg / nc), c = (int)(pg - (int64_t)v * nc);
    const double x = ev[v] - ec[c];
    const double den = fma(x, x, w * w);
    const double dl = 4.0 * x / den;
    const double dd = 4.0 * (w * w - x * x) / (den * den);
    for (int g = lane; g < ng; g += 32) {
        double2 a = y[g];
        y[g] = make_double2(dl * a.x, dl * a.y);
    }
    if (lane == 0) {
        atomicAdd(Lacc, dl * q);
        atomicAdd(dEv + v, q * dd);
        atomicAdd(dEc + c, -q * dd);
    }
}

cudaError_t launch_adj_rows(const double2 *M, double2 *Y, int64_t P, int ng, int nc, int64_t p0, const double *ev,
                            const double *ec, double w, double *L, double *dEv, double *dEc, cudaStream_t st)
{
    if (P == 0) return cudaSuccess;
    adj_rows_kernel<<<(unsigned)((P + 7) / 8), 256, 0, st>>>(M, Y, P, ng, nc, p0, ev, ec, w, L, dEv, dEc);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ back-projection of g_p onto the grid
// h_p(r) = (1/N_r) sum_G g_p(G) e^{-iG.r} = conj( (1/N_r) sum_G conj(g_p(G)) e^{+iG.r} ).
// One block per pair; per i0 slab: the sphere values of each kept (k1, k2) cell are summed
// with e^{+2 pi i k0 i0/n0} (conjugated input), zero-padded columns are transformed along
// i1, zero-padded lines along i2, and the conjugated slab is written to H.
template <bool TF>
__global__ void __launch_bounds__(256) adj_pair_kernel(const double2 *__restrict__ Gb, int64_t P, PairPlan pp,
                                                       const int *__restrict__ cell_start,
                                                       const int *__restrict__ cell_g, int ncell,
                                                       double2 *__restrict__ H)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int n0 = pp.n[0], n1 = pp.n[1], n2 = pp.n[2];
    const int ns = n1 * n2;
    double2 *a = (double2 *)smem, *b = a + ns;
    double2 *tw0 = b + ns, *tw1 = tw0 + n0, *tw2 = tw1 + n1;
    double2 *gs = tw2 + n2;                       // [ng] conj(g_p)
    int *kz = (int *)(gs + pp.ng);
    for (int i = threadIdx.x; i < n0; i += blockDim.x) tw0[i] = pp.ax[0].tw[i];
    for (int i = threadIdx.x; i < n1; i += blockDim.x) tw1[i] = pp.ax[1].tw[i];
    for (int i = threadIdx.x; i < n2; i += blockDim.x) tw2[i] = pp.ax[2].tw[i];
    for (int i = threadIdx.x; i < pp.K2; i += blockDim.x) kz[i] = pp.kz[i];
    const int64_t p = blockIdx.x;
    for (int g = threadIdx.x; g < pp.ng; g += blockDim.x) {
        double2 x = Gb[p * pp.ng + g];
        gs[g] = make_double2(x.x, -x.y);
    }
    __syncthreads();
    const double sc = 1.0 / ((double)n0 * ns);
    double2 *out = H + p * (int64_t)n0 * ns;
    for (int i0 = 0; i0 < n0; ++i0) {
        // kept columns k2' (K2 of them), each a zero-padded line of n1 values
        for (int i = threadIdx.x; i < pp.K2 * n1; i += blockDim.x) a[i] = make_double2(0.0, 0.0);
        __syncthreads();
        for (int cidx = threadIdx.x; cidx < ncell; cidx += blockDim.x) {
            double2 acc = make_double2(0.0, 0.0);
            int cell_pos = 0;
            for (int t = cell_start[cidx]; t < cell_start[cidx + 1]; ++t) {
                const int g = cell_g[t];
                const int pk = pp.gpack[g];
                const int k0 = pk & 255;
                cell_pos = (pk >> 16) * n1 + ((pk >> 8) & 255);
                cfma(acc, tw0[(k0 * i0) % n0], gs[g]);
            }
            a[cell_pos] = acc;
        }
        __syncthreads();
        double2 *r = fft_lines(a, b, pp.K2, n1, 1, pp.ax[1], tw1); // along i1, K2 lines
        double2 *o = (r == a) ? b : a;
        // scatter the K2 columns into full i2 lines: o[i1][i2]
        for (int i = threadIdx.x; i < ns; i += blockDim.x) o[i] = make_double2(0.0, 0.0);
        __syncthreads();
        for (int i = threadIdx.x; i < pp.K2 * n1; i += blockDim.x) {
            int q = i / n1, i1 = i - q * n1;
            o[i1 * n2 + kz[q]] = r[i];
        }
        __syncthreads();
        double2 *t = fft_lines(o, r, n1, n2, 1, pp.ax[2], tw2); // along i2
        for (int i = threadIdx.x; i < ns; i += blockDim.x) {
            double2 z = t[i];
            out[(int64_t)i0 * ns + i] = make_double2(z.x * sc, -z.y * sc);
        }
        __syncthreads();
    }
}

// The same back-projection in two-float arithmetic on the FP32 pipes (bands held in two-float
// form): conj(g_p) converted once per pair, in place over the block's own row of Gb (16 bytes
// an entry either way; Gb is not read again), the i0 sums per cell reading it from L2, both line
// transforms in hi + lo pairs; H is written in two-float form.  Keeping conj(g_p) out of shared
// memory lets four blocks run per SM on 40^3 instead of two.
// N > 0: a cubic N^3 grid, the line transforms and index arithmetic specialised at compile time;
// N = 0: any grid, runtime plans.
template <int N>
__global__ void __launch_bounds__(256) adj_pair_tf_kernel(double2 *__restrict__ Gb, PairPlan pp,
                                                          const int *__restrict__ cell_start,
                                                          const int *__restrict__ cell_g, int ncell, TfConsts kc,
                                                          tf sc, float4 *__restrict__ H)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int n0 = N ? N : pp.n[0], n1 = N ? N : pp.n[1], n2 = N ? N : pp.n[2];
    const int ns = n1 * n2;
    float4 *a = (float4 *)smem, *b = a + ns;
    float4 *tw0 = b + ns, *tw1 = tw0 + n0, *tw2 = tw1 + n1;
    int *kz = (int *)(tw2 + n2);
    for (int i = threadIdx.x; i < n0; i += blockDim.x) tw0[i] = pp.ax[0].twf[i];
    for (int i = threadIdx.x; i < n1; i += blockDim.x) tw1[i] = pp.ax[1].twf[i];
    for (int i = threadIdx.x; i < n2; i += blockDim.x) tw2[i] = pp.ax[2].twf[i];
    for (int i = threadIdx.x; i < pp.K2; i += blockDim.x) kz[i] = pp.kz[i];
    const int64_t p = blockIdx.x;
    float4 *gs = (float4 *)(Gb + p * pp.ng); // [ng] conj(g_p), two-float, over the row
    for (int g = threadIdx.x; g < pp.ng; g += blockDim.x) {
        const double2 x = Gb[p * pp.ng + g];
        const tf re = tf_from(x.x), im = tf_from(-x.y);
        gs[g] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
    __syncthreads();
    float4 *out = H + p * (int64_t)n0 * ns;
    for (int i0 = 0; i0 < n0; ++i0) {
        for (int i = threadIdx.x; i < pp.K2 * n1; i += blockDim.x) a[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        for (int cidx = threadIdx.x; cidx < ncell; cidx += blockDim.x) {
            tcx acc{{0.f, 0.f}, {0.f, 0.f}};
            int cell_pos = 0;
            for (int t = cell_start[cidx]; t < cell_start[cidx + 1]; ++t) {
                const int g = cell_g[t];
                const int pk = pp.gpack[g];
                const int k0 = pk & 255;
                cell_pos = (pk >> 16) * n1 + ((pk >> 8) & 255);
                acc = tc_add(acc, tc_mul(tc_load(gs + g), tc_load(tw0 + (k0 * i0) % n0)));
            }
            tc_store(a + cell_pos, acc);
        }
        __syncthreads();
        float4 *r;
        if constexpr (N > 0) r = tfft_lines_ct<N>(a, b, pp.K2, n1, tw1, kc); // along i1, K2 lines
        else r = tfft_lines(a, b, pp.K2, n1, 1, pp.ax[1], tw1, kc);
        float4 *o = (r == a) ? b : a;
        for (int i = threadIdx.x; i < ns; i += blockDim.x) o[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        for (int i = threadIdx.x; i < pp.K2 * n1; i += blockDim.x) {
            const int q = i / n1, i1 = i - q * n1;
            o[i1 * n2 + kz[q]] = r[i];
        }
        __syncthreads();
        const float4 *t;
        if constexpr (N > 0) t = tfft_lines_ct<N>(o, r, n1, n2, tw2, kc); // along i2
        else t = tfft_lines(o, r, n1, n2, 1, pp.ax[2], tw2, kc);
        for (int i = threadIdx.x; i < ns; i += blockDim.x) {
            const tcx z = tc_load(t + i);
            tc_store(out + (int64_t)i0 * ns + i, tcx{tf_mul(z.re, sc), tf_neg(tf_mul(z.im, sc))});
        }
        __syncthreads();
    }
}

cudaError_t launch_adj_pair(double2 *Gb, int64_t P, const PairPlan &pp, const int *cell_start,
                            const int *cell_g, int ncell, double2 *H, bool twofloat, cudaStream_t st)
{
    if (P == 0) return cudaSuccess;
    if (twofloat) {
        const size_t sm = sizeof(float4) * (2 * (size_t)pp.n[1] * pp.n[2] + pp.n[0] + pp.n[1] + pp.n[2]) +
                          sizeof(int) * pp.K2;
        const double inv = 1.0 / ((double)pp.n[0] * pp.n[1] * pp.n[2]);
        const float hi = (float)inv;
        const tf sc{hi, (float)(inv - (double)hi)};
        const bool cubic = pp.n[0] == pp.n[1] && pp.n[1] == pp.n[2];
        auto run = [&](auto kern) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            kern<<<(unsigned)P, 256, sm, st>>>(Gb, pp, cell_start, cell_g, ncell, tf_consts(), sc, (float4 *)H);
            return cudaGetLastError();
        };
        if (cubic && pp.n[0] == 24) return run(adj_pair_tf_kernel<24>);
        if (cubic && pp.n[0] == 40) return run(adj_pair_tf_kernel<40>);
        if (cubic && pp.n[0] == 48) return run(adj_pair_tf_kernel<48>);
        if (cubic && pp.n[0] == 72) return run(adj_pair_tf_kernel<72>);
        return run(adj_pair_tf_kernel<0>);
    }
    size_t sm = sizeof(double2) * (2 * (size_t)pp.n[1] * pp.n[2] + pp.n[0] + pp.n[1] + pp.n[2] + pp.ng) +
                sizeof(int) * pp.K2;
    cudaError_t e = cudaFuncSetAttribute(adj_pair_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    adj_pair_kernel<false><<<(unsigned)P, 256, sm, st>>>(Gb, P, pp, cell_start, cell_g, ncell, H);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ products into the band adjoints
__device__ __forceinline__ double2 psi_at(const void *psi, int64_t i, bool tf)
{
    if (!tf) return ((const double2 *)psi)[i];
    float4 v = ((const float4 *)psi)[i];
    return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

// psibar_c[c](r) += sum_{v in [v0, v0+nvc)} psi_v(r) H[(v - v0) nc + c](r)
__global__ void adj_cond_kernel(const void *__restrict__ psiv, int v0, int nvc, const double2 *__restrict__ H, int nc,
                                int64_t nr, bool tf, double2 *__restrict__ pbc)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= nr) return;
    double2 acc = pbc[(int64_t)c * nr + i];
    for (int v = 0; v < nvc; ++v) cfma(acc, psi_at(psiv, (int64_t)(v0 + v) * nr + i, tf), H[((int64_t)v * nc + c) * nr + i]);
    pbc[(int64_t)c * nr + i] = acc;
}

// psibar_v[v](r) += sum_c psi_c(r) conj(H[(v - v0) nc + c](r))
__global__ void adj_val_kernel(const void *__restrict__ psic, int v0, const double2 *__restrict__ H, int nc,
                               int64_t nr, bool tf, double2 *__restrict__ pbv)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int vl = blockIdx.y;
    if (i >= nr) return;
    double2 acc = pbv[(int64_t)(v0 + vl) * nr + i];
    for (int c = 0; c < nc; ++c) {
        double2 hh = H[((int64_t)vl * nc + c) * nr + i];
        cfma(acc, psi_at(psic, (int64_t)c * nr + i, tf), make_double2(hh.x, -hh.y));
    }
    pbv[(int64_t)(v0 + vl) * nr + i] = acc;
}

// Two-float forms of the two products (bands, H and the accumulators psibar in two-float form,
// 16 bytes a point as in FP64): everything on the FP32 pipes -- adding into FP64 accumulators
// took eight FP64 instructions a thread, which bounded the conduction product on this GPU.
__global__ void adj_cond_tf_kernel(const float4 *__restrict__ psiv, int v0, int nvc, const float4 *__restrict__ H,
                                   int nc, int64_t nr, float4 *__restrict__ pbc)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= nr) return;
    tcx acc{{0.f, 0.f}, {0.f, 0.f}};
    for (int v = 0; v < nvc; ++v)
        acc = tc_add(acc, tc_mul(tc_load(psiv + (int64_t)(v0 + v) * nr + i), tc_load(H + ((int64_t)v * nc + c) * nr + i)));
    float4 *o = pbc + (int64_t)c * nr + i;
    tc_store(o, tc_add(tc_load(o), acc));
}

__global__ void adj_val_tf_kernel(const float4 *__restrict__ psic, int v0, const float4 *__restrict__ H, int nc,
                                  int64_t nr, float4 *__restrict__ pbv)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int vl = blockIdx.y;
    if (i >= nr) return;
    tcx acc{{0.f, 0.f}, {0.f, 0.f}};
    for (int c = 0; c < nc; ++c) // psi_c conj(H) = conj(conj(psi_c) H)
        acc = tc_add(acc, tc_mulc(tc_load(psic + (int64_t)c * nr + i), tc_load(H + ((int64_t)vl * nc + c) * nr + i)));
    float4 *o = pbv + (int64_t)(v0 + vl) * nr + i;
    tc_store(o, tc_add(tc_load(o), tcx{acc.re, tf_neg(acc.im)}));
}

// Two-float accumulators to FP64, in place (same 16 bytes per point).
__global__ void tf_to_f64_kernel(void *__restrict__ x, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = ((const float4 *)x)[i];
        ((double2 *)x)[i] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
    }
}

cudaError_t launch_tf_to_f64(void *x, int64_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    tf_to_f64_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, n);
    return cudaGetLastError();
}

cudaError_t launch_adj_products(const void *psiv, const void *psic, int v0, int nvc, int nc, const double2 *H,
                                int64_t nr, bool tf, double2 *pbv, double2 *pbc, cudaStream_t st)
{
    if (tf) {
        dim3 gc((unsigned)((nr + 255) / 256), nc);
        adj_cond_tf_kernel<<<gc, 256, 0, st>>>((const float4 *)psiv, v0, nvc, (const float4 *)H, nc, nr,
                                               (float4 *)pbc);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        dim3 gv((unsigned)((nr + 255) / 256), nvc);
        adj_val_tf_kernel<<<gv, 256, 0, st>>>((const float4 *)psic, v0, (const float4 *)H, nc, nr, (float4 *)pbv);
        return cudaGetLastError();
    }
    dim3 gc((unsigned)((nr + 255) / 256), nc);
    adj_cond_kernel<<<gc, 256, 0, st>>>(psiv, v0, nvc, H, nc, nr, tf, pbc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 gv((unsigned)((nr + 255) / 256), nvc);
    adj_val_kernel<<<gv, 256, 0, st>>>(psic, v0, H, nc, nr, tf, pbv);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ band adjoint
__global__ void conj_kernel(double2 *x, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i].y = -x[i].y;
}

// dcoeff[b][k] = 2 conj(F[b][gofs[k]]) where F = FFT_+(conj(psibar)) = conj(FFT_-(psibar))
__global__ void gather_grad_kernel(const double2 *__restrict__ F, const int32_t *__restrict__ gofs, int nb, int ngpsi,
                                   int64_t nr, double2 *__restrict__ dc)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nb * ngpsi) return;
    int b = (int)(i / ngpsi), k = (int)(i - (int64_t)b * ngpsi);
    double2 z = F[(int64_t)b * nr + gofs[k]];
    dc[i] = make_double2(2.0 * z.x, -2.0 * z.y);
}

cudaError_t launch_band_adjoint(double2 *pb, int nb, const int n[3], const FftAxis ax[3], const int32_t *gofs,
                                int ngpsi, double2 *dc, cudaStream_t st)
{
    const int64_t nr = (int64_t)n[0] * n[1] * n[2];
    const int64_t tot = (int64_t)nb * nr;
    if (tot == 0) return cudaSuccess;
    conj_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(pb, tot);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_band_fft(pb, nb, n, ax, st);
    if (e != cudaSuccess) return e;
    const int64_t ng = (int64_t)nb * ngpsi;
    gather_grad_kernel<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(pb, gofs, nb, ngpsi, nr, dc);
    return cudaGetLastError();
}

} // namespace gw
