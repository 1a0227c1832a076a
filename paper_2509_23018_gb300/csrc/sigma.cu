// Off-diagonal plasmon-pole self-energy, prep. step (section on the off-diagonal GPP kernel):
// the per-(n, E) matrix P^n_GG'(E) of the Hybertsen-Louie plasmon-pole model, which the paper
// cites for the frequency dependence,
//     P[g][c] = v_c Omega2[g][c] / (2 wt[g][c] (d - sgn wt[g][c])),   d = E - E_n,
// sgn = -1 for an occupied band n (pole at E_n - wt) and +1 for an empty one (E_n + wt).
// gpp_setup_kernel folds the energy-independent residue A = v Omega2 / (2 wt) once per call;
// the FP64 path stores P for its DMMA products, the split path keeps A and wt transposed in
// two-float form and forms P inside the slicing kernel (ozaki.cu, gpp_prep_split_kernel),
// never storing it.
#include "internal.h"

#include <algorithm>

namespace gw {

constexpr int kGppTile = 32;

__device__ __forceinline__ double2 gpp_residue(double2 o, double2 w, double v)
{
    // v Omega2 / (2 w) = v Omega2 conj(w) / (2 |w|^2)
    const double s = v / (2.0 * fma(w.x, w.x, w.y * w.y));
    return make_double2(s * fma(o.x, w.x, o.y * w.y), s * fma(o.y, w.x, -o.x * w.y));
}

__device__ __forceinline__ float4 tf4(double2 x)
{
    const float rh = (float)x.x, ih = (float)x.y;
    return make_float4(rh, (float)(x.x - (double)rh), ih, (float)(x.y - (double)ih));
}

__global__ void __launch_bounds__(256) gpp_setup_kernel(const double2 *__restrict__ omega2,
                                                        const double2 *__restrict__ wtilde,
                                                        const double *__restrict__ vcoul, int64_t n, int ng,
                                                        double2 *__restrict__ A)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        A[i] = gpp_residue(omega2[i], wtilde[i], vcoul[i % ng]);
}

// One 32 x 32 tile of (g, c) per block, transposed through shared memory so that both the reads
// of Omega2 / wt and the writes of At / Wt are row-contiguous.
__global__ void __launch_bounds__(256) gpp_setup_tf_kernel(const double2 *__restrict__ omega2,
                                                           const double2 *__restrict__ wtilde,
                                                           const double *__restrict__ vcoul, int ng,
                                                           float4 *__restrict__ At, float4 *__restrict__ Wt)
{
    __shared__ float4 ta[kGppTile][kGppTile + 1], tw[kGppTile][kGppTile + 1];
    const int g0 = blockIdx.y * kGppTile, c0 = blockIdx.x * kGppTile;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5; // 32 x 8
    for (int r = ty; r < kGppTile; r += 8) {
        const int g = g0 + r, c = c0 + tx;
        if (g < ng && c < ng) {
            const int64_t i = (int64_t)g * ng + c;
            const double2 w = wtilde[i];
            ta[r][tx] = tf4(gpp_residue(omega2[i], w, vcoul[c]));
            tw[r][tx] = tf4(w);
        }
    }
    __syncthreads();
    for (int r = ty; r < kGppTile; r += 8) {
        const int c = c0 + r, g = g0 + tx;
        if (g < ng && c < ng) {
            const int64_t o = (int64_t)c * ng + g;
            At[o] = ta[tx][r];
            Wt[o] = tw[tx][r];
        }
    }
}

__global__ void __launch_bounds__(256) gpp_untranspose_kernel(const double2 *__restrict__ ST, int ne, int nsig,
                                                              double2 *__restrict__ sigma)
{
    // sigma[e][l][m] = ST[m][e nsig + l]; one 32 x 32 (l, m) tile of one energy per block
    __shared__ double2 t[kGppTile][kGppTile + 1];
    const int e = blockIdx.z, l0 = blockIdx.y * kGppTile, m0 = blockIdx.x * kGppTile;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t ld = (int64_t)ne * nsig;
    for (int r = ty; r < kGppTile; r += 8) {
        const int m = m0 + r, l = l0 + tx;
        if (m < nsig && l < nsig) t[r][tx] = ST[(int64_t)m * ld + (int64_t)e * nsig + l];
    }
    __syncthreads();
    for (int r = ty; r < kGppTile; r += 8) {
        const int l = l0 + r, m = m0 + tx;
        if (m < nsig && l < nsig) sigma[((int64_t)e * nsig + l) * nsig + m] = t[tx][r];
    }
}

__global__ void __launch_bounds__(256) gpp_prep_f64_kernel(const double2 *__restrict__ A,
                                                           const double2 *__restrict__ wtilde, int64_t n, double d,
                                                           double sgn, double2 *__restrict__ P)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = A[i], w = wtilde[i];
        const double xr = d - sgn * w.x, xi = -sgn * w.y;
        const double r = 1.0 / fma(xr, xr, xi * xi);
        const double ir = xr * r, ii = -xi * r;
        P[i] = make_double2(fma(a.x, ir, -a.y * ii), fma(a.x, ii, a.y * ir));
    }
}

cudaError_t launch_gpp_setup(const double2 *omega2, const double2 *wtilde, const double *vcoul, int ng, double2 *A,
                             cudaStream_t st)
{
    const int64_t n = (int64_t)ng * ng;
    if (n == 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    gpp_setup_kernel<<<(unsigned)blocks, 256, 0, st>>>(omega2, wtilde, vcoul, n, ng, A);
    return cudaGetLastError();
}

cudaError_t launch_gpp_setup_tf(const double2 *omega2, const double2 *wtilde, const double *vcoul, int ng, float4 *At,
                                float4 *Wt, cudaStream_t st)
{
    if (ng == 0) return cudaSuccess;
    const unsigned nt = (unsigned)((ng + kGppTile - 1) / kGppTile);
    gpp_setup_tf_kernel<<<dim3(nt, nt), 256, 0, st>>>(omega2, wtilde, vcoul, ng, At, Wt);
    return cudaGetLastError();
}

cudaError_t launch_gpp_untranspose(const double2 *ST, int ne, int nsig, double2 *sigma, cudaStream_t st)
{
    if (ne == 0 || nsig == 0) return cudaSuccess;
    const unsigned nt = (unsigned)((nsig + kGppTile - 1) / kGppTile);
    gpp_untranspose_kernel<<<dim3(nt, nt, (unsigned)ne), 256, 0, st>>>(ST, ne, nsig, sigma);
    return cudaGetLastError();
}

cudaError_t launch_gpp_prep_f64(const double2 *A, const double2 *wtilde, int ng, double d, double sgn, double2 *P,
                                cudaStream_t st)
{
    const int64_t n = (int64_t)ng * ng;
    if (n == 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    gpp_prep_f64_kernel<<<(unsigned)blocks, 256, 0, st>>>(A, wtilde, n, d, sgn, P);
    return cudaGetLastError();
}

} // namespace gw
