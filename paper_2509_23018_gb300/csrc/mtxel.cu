// Stage (a) of the chi0 path: band setup and pair matrix elements (the paper's MTXEL step).
//
//   a1  psi_n(r) = sum_K c_n(K) e^{+iK.r}            scatter + 3D FFT, FP64
//   a2  rho_vc(r) = conj(psi_v(r)) psi_c(r)            fused, never stored
//   a3  F_vc(G) = (1/N_r) sum_r rho_vc(r) e^{+iG.r}   output-pruned 3D FFT
//   a4  M[p][g] = F_p(G_g mod N)                       gather onto the caller's sphere
//
// M_mn^G is defined inline after Eq. ff-ch; the FFT route is the one the paper's
// MTXEL kernel takes ("Fourier transformations", Sec. Fast Full-Frequency GW).
#include "internal.h"
#include "fft.cuh"
#include "fft_tf.cuh"
#include "pair_tf_ct.cuh"

namespace gw {

constexpr int kPairThreads = 256; // threads per block of the runtime-shape pair kernels


// ------------------------------------------------------------------ a1: band setup
__global__ void scatter_kernel(const double2 *__restrict__ coeff, const int32_t *__restrict__ gofs, int nb, int ngpsi,
                               int64_t nr, double2 *__restrict__ psi)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t tot = (int64_t)nb * ngpsi;
    if (i >= tot) return;
    int b = (int)(i / ngpsi), k = (int)(i - (int64_t)b * ngpsi);
    psi[(int64_t)b * nr + gofs[k]] = coeff[i];
}

cudaError_t launch_scatter(const double2 *coeff, const int32_t *gofs, int nb, int ngpsi, int64_t nr, double2 *psi,
                           cudaStream_t st)
{
    int64_t tot = (int64_t)nb * ngpsi;
    if (tot == 0) return cudaSuccess;
    scatter_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(coeff, gofs, nb, ngpsi, nr, psi);
    return cudaGetLastError();
}

// One (band, i0) slab of n1 x n2 points: FFT along i2 then along i1, in shared memory.
__global__ void __launch_bounds__(256) band_fft_slab_kernel(double2 *__restrict__ psi, int n0, int n1, int n2,
                                                             FftAxis ax1, FftAxis ax2)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int ns = n1 * n2;
    double2 *a = (double2 *)smem, *b = a + ns, *tw1 = b + ns, *tw2 = tw1 + n1;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) tw1[i] = ax1.tw[i];
    for (int i = threadIdx.x; i < n2; i += blockDim.x) tw2[i] = ax2.tw[i];
    double2 *g = psi + ((int64_t)blockIdx.y * n0 + blockIdx.x) * ns;
    for (int i = threadIdx.x; i < ns; i += blockDim.x) a[i] = g[i];
    __syncthreads();
    double2 *r = fft_lines(a, b, n1, n2, 1, ax2, tw2);      // along i2
    double2 *o = (r == a) ? b : a;
    r = fft_lines(r, o, n2, 1, n2, ax1, tw1);               // along i1 (strided lines)
    for (int i = threadIdx.x; i < ns; i += blockDim.x) g[i] = r[i];
}

// One (band, i1) plane of n0 x n2 points: FFT along i0.
__global__ void __launch_bounds__(256) band_fft_axis0_kernel(double2 *__restrict__ psi, int n0, int n1, int n2,
                                                              FftAxis ax0)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int np = n0 * n2;
    double2 *a = (double2 *)smem, *b = a + np, *tw0 = b + np;
    for (int i = threadIdx.x; i < n0; i += blockDim.x) tw0[i] = ax0.tw[i];
    double2 *g = psi + (int64_t)blockIdx.y * n0 * n1 * n2 + (int64_t)blockIdx.x * n2;
    const int64_t rs = (int64_t)n1 * n2;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        int i0 = i / n2, i2 = i - i0 * n2;
        a[i] = g[i0 * rs + i2];
    }
    __syncthreads();
    double2 *o = b;
    double2 *r = fft_lines(a, o, n2, 1, n2, ax0, tw0);      // lines along i0, stride n2
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        int i0 = i / n2, i2 = i - i0 * n2;
        g[i0 * rs + i2] = r[i];
    }
}

cudaError_t launch_band_fft(double2 *psi, int nb, const int n[3], const FftAxis ax[3], cudaStream_t st)
{
    if (nb == 0) return cudaSuccess;
    size_t sm1 = sizeof(double2) * (2 * (size_t)n[1] * n[2] + n[1] + n[2]);
    size_t sm0 = sizeof(double2) * (2 * (size_t)n[0] * n[2] + n[0]);
    cudaError_t e = cudaFuncSetAttribute(band_fft_slab_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(band_fft_axis0_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm0);
    if (e != cudaSuccess) return e;
    band_fft_slab_kernel<<<dim3(n[0], nb), 256, sm1, st>>>(psi, n[0], n[1], n[2], ax[1], ax[2]);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    band_fft_axis0_kernel<<<dim3(n[1], nb), 256, sm0, st>>>(psi, n[0], n[1], n[2], ax[0]);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ a1 in two-float arithmetic
// Coefficients are split into hi + lo FP32 pairs as they are scattered; the three axes
// are then transformed in two-float arithmetic, in place, with the same kernels' layout.
__global__ void scatter_tf_kernel(const double2 *__restrict__ coeff, const int32_t *__restrict__ gofs, int nb,
                                  int ngpsi, int64_t nr, float4 *__restrict__ psi)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t tot = (int64_t)nb * ngpsi;
    if (i >= tot) return;
    int b = (int)(i / ngpsi), k = (int)(i - (int64_t)b * ngpsi);
    double2 z = coeff[i];
    float rh = __double2float_rn(z.x), ih = __double2float_rn(z.y);
    psi[(int64_t)b * nr + gofs[k]] =
        make_float4(rh, __double2float_rn(z.x - (double)rh), ih, __double2float_rn(z.y - (double)ih));
}

__global__ void __launch_bounds__(256) band_fft_slab_tf_kernel(float4 *__restrict__ psi, int n0, int n1, int n2,
                                                                FftAxis ax1, FftAxis ax2, TfConsts kc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int ns = n1 * n2;
    float4 *a = (float4 *)smem, *b = a + ns, *tw1 = b + ns, *tw2 = tw1 + n1;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) tw1[i] = ax1.twf[i];
    for (int i = threadIdx.x; i < n2; i += blockDim.x) tw2[i] = ax2.twf[i];
    float4 *g = psi + ((int64_t)blockIdx.y * n0 + blockIdx.x) * ns;
    for (int i = threadIdx.x; i < ns; i += blockDim.x) a[i] = g[i];
    __syncthreads();
    float4 *r = tfft_lines(a, b, n1, n2, 1, ax2, tw2, kc);  // along i2
    float4 *o = (r == a) ? b : a;
    r = tfft_lines(r, o, n2, 1, n2, ax1, tw1, kc);          // along i1 (strided lines)
    for (int i = threadIdx.x; i < ns; i += blockDim.x) g[i] = r[i];
}

__global__ void __launch_bounds__(256) band_fft_axis0_tf_kernel(float4 *__restrict__ psi, int n0, int n1, int n2,
                                                                 FftAxis ax0, TfConsts kc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int np = n0 * n2;
    float4 *a = (float4 *)smem, *b = a + np, *tw0 = b + np;
    for (int i = threadIdx.x; i < n0; i += blockDim.x) tw0[i] = ax0.twf[i];
    float4 *g = psi + (int64_t)blockIdx.y * n0 * n1 * n2 + (int64_t)blockIdx.x * n2;
    const int64_t rs = (int64_t)n1 * n2;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        int i0 = i / n2, i2 = i - i0 * n2;
        a[i] = g[i0 * rs + i2];
    }
    __syncthreads();
    float4 *r = tfft_lines(a, b, n2, 1, n2, ax0, tw0, kc);   // lines along i0, stride n2
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        int i0 = i / n2, i2 = i - i0 * n2;
        g[i0 * rs + i2] = r[i];
    }
}

TfConsts tf_consts()
{
    auto from = [](double x) {
        float h = (float)x;
        return tf{h, (float)(x - (double)h)};
    };
    TfConsts kc;
    kc.sin60 = from(kSin60);
    kc.c1 = from(kC1);
    kc.s1 = from(kS1);
    kc.c2 = from(kC2);
    kc.s2 = from(kS2);
    kc.rs2 = from(kRs2);
    return kc;
}

cudaError_t launch_band_setup_tf(const double2 *coeff, const int32_t *gofs, int nb, int ngpsi, void *psi,
                                 const int n[3], const FftAxis ax[3], const int maxabs[3], cudaStream_t st)
{
    const int64_t nr = (int64_t)n[0] * n[1] * n[2];
    const int64_t tot = (int64_t)nb * ngpsi;
    if (tot == 0) return cudaSuccess;
    float4 *p = (float4 *)psi;
    scatter_tf_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(coeff, gofs, nb, ngpsi, nr, p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const TfConsts kc = tf_consts();
    if (n[0] == n[1] && n[1] == n[2]) {
        switch (n[0]) { // grid-specialised transforms for the standard cubic grids
        case 24: return launch_band_fft_tf_g24(p, nb, ax, kc, maxabs[0], maxabs[1], st);
        case 40: return launch_band_fft_tf_g40(p, nb, ax, kc, maxabs[0], maxabs[1], st);
        case 48: return launch_band_fft_tf_g48(p, nb, ax, kc, maxabs[0], maxabs[1], st);
        case 72: return launch_band_fft_tf_g72(p, nb, ax, kc, maxabs[0], maxabs[1], st);
        default: break;
        }
    }
    size_t sm1 = sizeof(float4) * (2 * (size_t)n[1] * n[2] + n[1] + n[2]);
    size_t sm0 = sizeof(float4) * (2 * (size_t)n[0] * n[2] + n[0]);
    if ((e = cudaFuncSetAttribute(band_fft_slab_tf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(band_fft_axis0_tf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm0)) !=
            cudaSuccess)
        return e;
    band_fft_slab_tf_kernel<<<dim3(n[0], nb), 256, sm1, st>>>(p, n[0], n[1], n[2], ax[1], ax[2], kc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    band_fft_axis0_tf_kernel<<<dim3(n[1], nb), 256, sm0, st>>>(p, n[0], n[1], n[2], ax[0], kc);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ a2-a4: fused pair kernel
// One block per pair.  The block walks the n0 slabs of the grid; per slab it forms the
// pair product, transforms along i2 (all lines), keeps the K2 needed i2-frequencies,
// transforms those columns along i1, and adds e^{+2 pi i k0 i0/n0} times the selected
// (k1, k2) values into the per-G accumulators, which live in registers (NPT per thread).
// The i0 axis is thus a direct sum onto the sphere, which also performs the gather.

template <int NPT>
__global__ void __launch_bounds__(kPairThreads) pair_kernel(const double2 *__restrict__ psiv,
                                                             const double2 *__restrict__ psic, int nc, int64_t p0,
                                                             PairPlan pp, double2 *__restrict__ M)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int n0 = pp.n[0], n1 = pp.n[1], n2 = pp.n[2];
    const int ns = n1 * n2;
    double2 *a = (double2 *)smem, *b = a + ns;
    double2 *tw0 = b + ns, *tw1 = tw0 + n0, *tw2 = tw1 + n1;
    int *kz = (int *)(tw2 + n2);
    for (int i = threadIdx.x; i < n0; i += blockDim.x) tw0[i] = pp.ax[0].tw[i];
    for (int i = threadIdx.x; i < n1; i += blockDim.x) tw1[i] = pp.ax[1].tw[i];
    for (int i = threadIdx.x; i < n2; i += blockDim.x) tw2[i] = pp.ax[2].tw[i];
    for (int i = threadIdx.x; i < pp.K2; i += blockDim.x) kz[i] = pp.kz[i];

    const int64_t p = p0 + blockIdx.x;
    const int v = (int)(p / nc), c = (int)(p - (int64_t)v * nc);
    const int64_t nr = (int64_t)n0 * ns;
    const double2 *pv = psiv + (int64_t)v * nr;
    const double2 *pc = psic + (int64_t)c * nr;

    double2 F[NPT];
    int sel[NPT], k0[NPT], e0[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        int g = threadIdx.x + j * kPairThreads;
        F[j] = make_double2(0.0, 0.0);
        int pk = (g < pp.ng) ? pp.gpack[g] : 0;
        k0[j] = pk & 255;
        sel[j] = (pk >> 16) * n1 + ((pk >> 8) & 255); // position in the i1-transformed columns
        e0[j] = 0;                                    // (k0 * i0) mod n0, advanced per slab
    }
    __syncthreads();

    for (int i0 = 0; i0 < n0; ++i0) {
        const double2 *sv = pv + (int64_t)i0 * ns, *sc = pc + (int64_t)i0 * ns;
        for (int i = threadIdx.x; i < ns; i += 3 * blockDim.x) {
            double2 xv[3], xc[3];
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int k = i + u * blockDim.x;
                if (k < ns) {
                    xv[u] = __ldg(sv + k);
                    xc[u] = __ldg(sc + k);
                }
            }
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int k = i + u * blockDim.x;
                if (k < ns) a[k] = cmulc(xv[u], xc[u]);
            }
        }
        __syncthreads();
        double2 *r = fft_lines(a, b, n1, n2, 1, pp.ax[2], tw2); // along i2
        double2 *o = (r == a) ? b : a;
        for (int i = threadIdx.x; i < pp.K2 * n1; i += blockDim.x) {
            int q = i / n1, i1 = i - q * n1;
            o[i] = r[i1 * n2 + kz[q]];
        }
        __syncthreads();
        double2 *t = fft_lines(o, r, pp.K2, n1, 1, pp.ax[1], tw1); // along i1 on the kept columns
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            cfma(F[j], tw0[e0[j]], t[sel[j]]);
            e0[j] += k0[j];
            if (e0[j] >= n0) e0[j] -= n0;
        }
        __syncthreads();
    }
    const double sc = 1.0 / (double)nr;
    double2 *out = M + (int64_t)blockIdx.x * pp.ng;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        int g = threadIdx.x + j * kPairThreads;
        if (g < pp.ng) out[g] = make_double2(F[j].x * sc, F[j].y * sc);
    }
}

int pair_max_ng() { return 32 * kPairThreads; }

// Same algorithm as pair_kernel, in two-float arithmetic on the FP32 pipes.  The band
// grids hold (re.hi, re.lo, im.hi, im.lo) per point (see launch_band_setup_tf); the output
// M is FP64.
template <int NPT>
__global__ void __launch_bounds__(kPairThreads) pair_kernel_tf(const float4 *__restrict__ psiv,
                                                                const float4 *__restrict__ psic, int nc, int64_t p0,
                                                                PairPlan pp, TfConsts kc, tf inv_nr,
                                                                double2 *__restrict__ M)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int n0 = pp.n[0], n1 = pp.n[1], n2 = pp.n[2];
    const int ns = n1 * n2;
    float4 *a = (float4 *)smem, *b = a + ns;
    float4 *tw0 = b + ns, *tw1 = tw0 + n0, *tw2 = tw1 + n1;
    int *kz = (int *)(tw2 + n2);
    for (int i = threadIdx.x; i < n0; i += blockDim.x) tw0[i] = pp.ax[0].twf[i];
    for (int i = threadIdx.x; i < n1; i += blockDim.x) tw1[i] = pp.ax[1].twf[i];
    for (int i = threadIdx.x; i < n2; i += blockDim.x) tw2[i] = pp.ax[2].twf[i];
    for (int i = threadIdx.x; i < pp.K2; i += blockDim.x) kz[i] = pp.kz[i];

    const int64_t p = p0 + blockIdx.x;
    const int v = (int)(p / nc), c = (int)(p - (int64_t)v * nc);
    const int64_t nr = (int64_t)n0 * ns;
    const float4 *pv = psiv + (int64_t)v * nr;
    const float4 *pc = psic + (int64_t)c * nr;

    tcx F[NPT];
    int sel[NPT], k0[NPT], e0[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        int g = threadIdx.x + j * kPairThreads;
        F[j] = {{0.f, 0.f}, {0.f, 0.f}};
        int pk = (g < pp.ng) ? pp.gpack[g] : 0;
        k0[j] = pk & 255;
        sel[j] = (pk >> 16) * n1 + ((pk >> 8) & 255);
        e0[j] = 0;
    }
    __syncthreads();

    for (int i0 = 0; i0 < n0; ++i0) {
        const float4 *sv = pv + (int64_t)i0 * ns, *sc = pc + (int64_t)i0 * ns;
        // three points per thread in flight, so the band loads overlap
        for (int i = threadIdx.x; i < ns; i += 3 * blockDim.x) {
            tcx xv[3], xc[3];
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int k = i + u * blockDim.x;
                if (k < ns) {
                    xv[u] = tc_load(sv + k);
                    xc[u] = tc_load(sc + k);
                }
            }
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int k = i + u * blockDim.x;
                if (k < ns) tc_store(a + k, tc_mulc(xv[u], xc[u]));
            }
        }
        __syncthreads();
        float4 *r = tfft_lines(a, b, n1, n2, 1, pp.ax[2], tw2, kc); // along i2
        float4 *o = (r == a) ? b : a;
        for (int i = threadIdx.x; i < pp.K2 * n1; i += blockDim.x) {
            int q = i / n1, i1 = i - q * n1;
            o[i] = r[i1 * n2 + kz[q]];
        }
        __syncthreads();
        float4 *t = tfft_lines(o, r, pp.K2, n1, 1, pp.ax[1], tw1, kc); // along i1 on the kept columns
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            tcx u = tc_mul(tc_load(t + sel[j]), tc_load(tw0 + e0[j]));
            F[j] = tc_add(F[j], u);
            e0[j] += k0[j];
            if (e0[j] >= n0) e0[j] -= n0;
        }
        __syncthreads();
    }
    double2 *out = M + (int64_t)blockIdx.x * pp.ng;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        int g = threadIdx.x + j * kPairThreads;
        if (g < pp.ng) out[g] = make_double2(tf_to_d(tf_mul(F[j].re, inv_nr)), tf_to_d(tf_mul(F[j].im, inv_nr)));
    }
}

template <int NPT>
static cudaError_t launch_pair_tf_t(const float4 *psiv, const float4 *psic, int nc, int64_t p0, int64_t count,
                                    const PairPlan &pp, const TfConsts &kc, tf inv_nr, double2 *M, cudaStream_t st)
{
    size_t sm = sizeof(float4) * (2 * (size_t)pp.n[1] * pp.n[2] + pp.n[0] + pp.n[1] + pp.n[2]) + sizeof(int) * pp.K2;
    cudaError_t e = cudaFuncSetAttribute(pair_kernel_tf<NPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    pair_kernel_tf<NPT><<<(unsigned)count, kPairThreads, sm, st>>>(psiv, psic, nc, p0, pp, kc, inv_nr, M);
    return cudaGetLastError();
}

size_t pair_tf_ct_smem_bytes(const PairPlan &pp)
{
    if (!pair_tf_ct_fits(pp)) return 0;
    switch (pp.n[0]) {
    case 24: return pair_tf_ct_smem<24>(pp);
    case 40: return pair_tf_ct_smem<40>(pp);
    case 48: return pair_tf_ct_smem<48>(pp);
    case 72: return pair_tf_ct_smem<72>(pp);
    default: return 0;
    }
}

cudaError_t launch_pair_tf_from_f(const CUtensorMap &tmF, const CUtensorMap &tmS, int64_t R, const PairPlan &pp,
                                  double2 *M, cudaStream_t st)
{
    if (R == 0) return cudaSuccess;
    if (pp.n[0] != 48 || pp.n[1] != 48 || pp.n[2] != 48 || !pp.scr || !pp.slot_flags || pp.nslots <= 0)
        return cudaErrorInvalidValue;
    const double invd = 1.0 / ((double)pp.n[0] * pp.n[1] * pp.n[2]);
    const float invh = (float)invd;
    const tf inv{invh, (float)(invd - (double)invh)};
    return launch_pair_tf_from_f_g48(tmF, tmS, R, pp, tf_consts(), inv, M, st);
}

cudaError_t pair_tf_scratch(const PairPlan &pp, int *nslots, size_t *slot_elems)
{
    *nslots = 0;
    *slot_elems = 0;
    if (!pair_tf_ct_fits(pp)) return cudaSuccess;
    cudaError_t e;
    switch (pp.n[0]) {
    case 24: e = pair_tf_slots_g24(pp, nslots); break;
    case 40: e = pair_tf_slots_g40(pp, nslots); break;
    case 48: e = pair_tf_slots_g48(pp, nslots); break;
    case 72: e = pair_tf_slots_g72(pp, nslots); break;
    default: return cudaSuccess;
    }
    if (e == cudaSuccess) *slot_elems = (size_t)pp.n[0] * pp.K12;
    return e;
}

cudaError_t launch_pair_tf(const void *psiv, const void *psic, int nc, int64_t p0, int64_t count, const PairPlan &pp,
                           double2 *M, cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    const TfConsts kc = tf_consts();
    const double invd = 1.0 / ((double)pp.n[0] * pp.n[1] * pp.n[2]);
    const float invh = (float)invd;
    const tf inv{invh, (float)(invd - (double)invh)};
    const float4 *a = (const float4 *)psiv, *b = (const float4 *)psic;
    int need = (pp.ng + kPairThreads - 1) / kPairThreads;
    if (pair_tf_ct_fits(pp) && pp.scr && pp.slot_flags && pp.nslots > 0) {
        // grid-specialised kernels for the cubic grids of the standard workloads
        switch (pp.n[1]) {
        case 24: return launch_pair_tf_g24(a, b, nc, p0, count, pp, kc, inv, M, st);
        case 40: return launch_pair_tf_g40(a, b, nc, p0, count, pp, kc, inv, M, st);
        case 48: return launch_pair_tf_g48(a, b, nc, p0, count, pp, kc, inv, M, st);
        case 72: return launch_pair_tf_g72(a, b, nc, p0, count, pp, kc, inv, M, st);
        default: break;
        }
    }
    if (need <= 2) return launch_pair_tf_t<2>(a, b, nc, p0, count, pp, kc, inv, M, st);
    if (need <= 4) return launch_pair_tf_t<4>(a, b, nc, p0, count, pp, kc, inv, M, st);
    if (need <= 8) return launch_pair_tf_t<8>(a, b, nc, p0, count, pp, kc, inv, M, st);
    if (need <= 12) return launch_pair_tf_t<12>(a, b, nc, p0, count, pp, kc, inv, M, st);
    if (need <= 16) return launch_pair_tf_t<16>(a, b, nc, p0, count, pp, kc, inv, M, st);
    if (need <= 24) return launch_pair_tf_t<24>(a, b, nc, p0, count, pp, kc, inv, M, st);
    if (need <= 32) return launch_pair_tf_t<32>(a, b, nc, p0, count, pp, kc, inv, M, st);
    return cudaErrorInvalidValue;
}


template <int NPT>
static cudaError_t launch_pair_t(const double2 *psiv, const double2 *psic, int nc, int64_t p0, int64_t count,
                                 const PairPlan &pp, double2 *M, cudaStream_t st)
{
    size_t sm = sizeof(double2) * (2 * (size_t)pp.n[1] * pp.n[2] + pp.n[0] + pp.n[1] + pp.n[2]) + sizeof(int) * pp.K2;
    cudaError_t e = cudaFuncSetAttribute(pair_kernel<NPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    for (int64_t off = 0; off < count; off += 65535LL * 1024) {
        int64_t cnt = count - off < 65535LL * 1024 ? count - off : 65535LL * 1024;
        pair_kernel<NPT><<<(unsigned)cnt, kPairThreads, sm, st>>>(psiv, psic, nc, p0 + off, pp,
                                                                  M + off * pp.ng);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_pair(const double2 *psiv, const double2 *psic, int nc, int64_t p0, int64_t count,
                        const PairPlan &pp, double2 *M, cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    int need = (pp.ng + kPairThreads - 1) / kPairThreads;
    if (need <= 2) return launch_pair_t<2>(psiv, psic, nc, p0, count, pp, M, st);
    if (need <= 4) return launch_pair_t<4>(psiv, psic, nc, p0, count, pp, M, st);
    if (need <= 8) return launch_pair_t<8>(psiv, psic, nc, p0, count, pp, M, st);
    if (need <= 12) return launch_pair_t<12>(psiv, psic, nc, p0, count, pp, M, st);
    if (need <= 16) return launch_pair_t<16>(psiv, psic, nc, p0, count, pp, M, st);
    if (need <= 24) return launch_pair_t<24>(psiv, psic, nc, p0, count, pp, M, st);
    if (need <= 32) return launch_pair_t<32>(psiv, psic, nc, p0, count, pp, M, st);
    return cudaErrorInvalidValue;
}

} // namespace gw
