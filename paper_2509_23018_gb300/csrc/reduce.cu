// Energy factor (a5), diagonal reduction and Hermitian symmetrisation (a7).
#include "internal.h"
#include "ptx.cuh"

namespace gw {

// a5: Delta_vc(iw) = 2/(x - iw) + 2/(x + iw) = 4x / (x^2 + w^2),  x = E_v - E_c.
__global__ void delta_kernel(const double *__restrict__ ev, const double *__restrict__ ec, int nc, int64_t p0,
                             int64_t count, OmegaList om, double *__restrict__ delta)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    int64_t p = p0 + i;
    int v = (int)(p / nc), c = (int)(p - (int64_t)v * nc);
    double x = ev[v] - ec[c];
    for (int w = 0; w < om.nw; ++w) {
        double ww = om.w[w];
        delta[(int64_t)w * count + i] = 4.0 * x / fma(x, x, ww * ww);
    }
}

// The same for a chunk of all valence bands x conduction bands c0 .. c0 + cb - 1, rows in the
// order r = cl nv + v of the tensor-core pair elements.
__global__ void delta_block_kernel(const double *__restrict__ ev, const double *__restrict__ ec, int nv, int c0,
                                   int cb, OmegaList om, double *__restrict__ delta)
{
    const int64_t count = (int64_t)nv * cb;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int cl = (int)(i / nv), v = (int)(i - (int64_t)cl * nv);
    const double x = ev[v] - ec[c0 + cl];
    for (int w = 0; w < om.nw; ++w) {
        const double ww = om.w[w];
        delta[(int64_t)w * count + i] = 4.0 * x / fma(x, x, ww * ww);
    }
}

cudaError_t launch_delta_block(const double *ev, const double *ec, int nv, int c0, int cb, const OmegaList &om,
                               double *delta, cudaStream_t st)
{
    const int64_t count = (int64_t)nv * cb;
    if (count == 0) return cudaSuccess;
    delta_block_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(ev, ec, nv, c0, cb, om, delta);
    return cudaGetLastError();
}

// Real-axis energy factor with broadening: Delta = 2/(x - w - i eta) + 2/(x + w + i eta),
// x = E_v - E_c < 0, split into three non-positive weights per frequency (block 3 w + k):
// k = 0: min(Re Delta, 0); k = 1: -max(Re Delta, 0); k = 2: Im Delta (<= 0 for w >= 0, x < 0).
__global__ void delta_real_kernel(const double *__restrict__ ev, const double *__restrict__ ec, int nc, int64_t p0,
                                  int64_t count, OmegaList om, double eta, double *__restrict__ delta)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    int64_t p = p0 + i;
    int v = (int)(p / nc), c = (int)(p - (int64_t)v * nc);
    const double x = ev[v] - ec[c], e2 = eta * eta;
    for (int w = 0; w < om.nw; ++w) {
        const double a = x - om.w[w], b = x + om.w[w];
        const double da = fma(a, a, e2), db = fma(b, b, e2);
        const double re = 2.0 * a / da + 2.0 * b / db;
        const double im = 2.0 * eta / da - 2.0 * eta / db;
        delta[(int64_t)(3 * w) * count + i] = fmin(re, 0.0);
        delta[(int64_t)(3 * w + 1) * count + i] = -fmax(re, 0.0);
        delta[(int64_t)(3 * w + 2) * count + i] = fmin(im, 0.0);
    }
}

cudaError_t launch_delta_real(const double *ev, const double *ec, int nc, int64_t p0, int64_t count,
                              const OmegaList &om, double eta, double *delta, cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    delta_real_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(ev, ec, nc, p0, count, om, eta, delta);
    return cudaGetLastError();
}

// out[w] = (T[3w] - T[3w+1]) + i T[3w+2] for Hermitian parts T (complex [ng][ng] each)
__global__ void combine_real_kernel(const double2 *__restrict__ T, int64_t nn, int nw, double2 *__restrict__ out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nn * nw) return;
    const int64_t w = e / nn, j = e - w * nn;
    const double2 a = T[(3 * w) * nn + j], b = T[(3 * w + 1) * nn + j], c = T[(3 * w + 2) * nn + j];
    out[e] = make_double2(a.x - b.x - c.y, a.y - b.y + c.x);
}

cudaError_t launch_combine_real(const double2 *T, int64_t nn, int nw, double2 *out, cudaStream_t st)
{
    const int64_t n = nn * nw;
    if (n == 0) return cudaSuccess;
    combine_real_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(T, nn, nw, out);
    return cudaGetLastError();
}

// Forward derivative of Delta(i w) = 4x/(x^2 + w^2) along (dE_v, dE_c): dDelta = 4(w^2 - x^2)/(x^2 +
// w^2)^2 (dE_v - dE_c), split into two non-positive weights: block 2w: min(dDelta, 0), block
// 2w + 1: -max(dDelta, 0).
__global__ void delta_jvp_kernel(const double *__restrict__ ev, const double *__restrict__ ec,
                                 const double *__restrict__ dev, const double *__restrict__ dec, int nc, int64_t p0,
                                 int64_t count, OmegaList om, double *__restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    int64_t p = p0 + i;
    int v = (int)(p / nc), c = (int)(p - (int64_t)v * nc);
    const double x = ev[v] - ec[c], dx = dev[v] - dec[c];
    for (int w = 0; w < om.nw; ++w) {
        const double w2 = om.w[w] * om.w[w], den = fma(x, x, w2);
        const double dd = 4.0 * (w2 - x * x) / (den * den) * dx;
        out[(int64_t)(2 * w) * count + i] = fmin(dd, 0.0);
        out[(int64_t)(2 * w + 1) * count + i] = -fmax(dd, 0.0);
    }
}

cudaError_t launch_delta_jvp(const double *ev, const double *ec, const double *dev, const double *dec, int nc,
                             int64_t p0, int64_t count, const OmegaList &om, double *out, cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    delta_jvp_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(ev, ec, dev, dec, nc, p0, count, om, out);
    return cudaGetLastError();
}

// d = X1 + X2 (the tangent dM); X1 = M + d, X2 = M - d
__global__ void jvp_mix_kernel(const double2 *__restrict__ M, double2 *__restrict__ X1, double2 *__restrict__ X2,
                               int64_t n)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double2 m = M[e], a = X1[e], b = X2[e];
    const double dx = a.x + b.x, dy = a.y + b.y;
    X1[e] = make_double2(m.x + dx, m.y + dy);
    X2[e] = make_double2(m.x - dx, m.y - dy);
}

cudaError_t launch_jvp_mix(const double2 *M, double2 *X1, double2 *X2, int64_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    jvp_mix_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(M, X1, X2, n);
    return cudaGetLastError();
}

// out[w] = (Tp[w] - Tm[w]) / 2 + Tw[2w] - Tw[2w+1]
__global__ void combine_jvp_kernel(const double2 *__restrict__ Tp, const double2 *__restrict__ Tm,
                                   const double2 *__restrict__ Tw, int64_t nn, int nw, double2 *__restrict__ out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nn * nw) return;
    const int64_t w = e / nn, j = e - w * nn;
    const double2 a = Tp[e], b = Tm[e], c = Tw[(2 * w) * nn + j], d = Tw[(2 * w + 1) * nn + j];
    out[e] = make_double2(0.5 * (a.x - b.x) + c.x - d.x, 0.5 * (a.y - b.y) + c.y - d.y);
}

cudaError_t launch_combine_jvp(const double2 *Tp, const double2 *Tm, const double2 *Tw, int64_t nn, int nw,
                               double2 *out, cudaStream_t st)
{
    const int64_t n = nn * nw;
    if (n == 0) return cudaSuccess;
    combine_jvp_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Tp, Tm, Tw, nn, nw, out);
    return cudaGetLastError();
}

cudaError_t launch_delta(const double *ev, const double *ec, int nc, int64_t p0, int64_t count, const OmegaList &om,
                         double *delta, cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    delta_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(ev, ec, nc, p0, count, om, delta);
    return cudaGetLastError();
}

// a7: diag[w][g] += sum_p delta[w][p] |M[p][g]|^2.
// A warp covers 8 consecutive columns (lane & 7) and 4 pair rows at a time (lane >> 3);
// the four row-partial sums of a column are combined with warp shuffles, then one
// lane per column adds the warp's result into diag.
__global__ void diag_kernel(const double2 *__restrict__ M, int64_t P, int ng, const double *__restrict__ delta,
                            int64_t dstride, double *__restrict__ diag, int64_t diag_wstride)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int g = blockIdx.x * 8 + (lane & 7);
    const int w = blockIdx.z;
    const double *dl = delta + (int64_t)w * dstride;
    double acc = 0.0;
    if (g < ng) {
        for (int64_t p = ((int64_t)blockIdx.y * nwarp + wid) * 4 + (lane >> 3); p < P;
             p += (int64_t)gridDim.y * nwarp * 4) {
            double2 m = M[p * ng + g];
            acc = fma(dl[p], fma(m.x, m.x, m.y * m.y), acc);
        }
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 8);
    acc += __shfl_xor_sync(0xffffffffu, acc, 16);
    if (lane < 8 && g < ng) atomicAdd(diag + (int64_t)w * diag_wstride + g, acc);
}

cudaError_t launch_diag(const double2 *M, int64_t P, int ng, const double *delta, int64_t dstride, int nw,
                        double *diag, int64_t diag_wstride, cudaStream_t st)
{
    if (P == 0 || nw == 0) return cudaSuccess;
    int gx = (ng + 7) / 8;
    int64_t rows = (P + 31) / 32;
    int gy = (int)(rows < 64 ? rows : 64);
    diag_kernel<<<dim3(gx, gy, nw), 256, 0, st>>>(M, P, ng, delta, dstride, diag, diag_wstride);
    return cudaGetLastError();
}

// a7: chi[G][G'] = conj(chi[G'][G]) for G > G'; Im chi[G][G] = 0.  32 x 32 tiles through
// shared memory so both the read of the upper tile and the write of the lower tile
// are row-contiguous.
__global__ void symmetrize_kernel(double2 *__restrict__ chi, int ng, int nt)
{
    __shared__ double2 t[32][33];
    int b = blockIdx.x, bi = 0;
    while (b > bi) { b -= bi + 1; ++bi; } // lower-triangle tile (bi, bj), bj <= bi
    const int bj = b;
    double2 *c = chi + (int64_t)blockIdx.z * ng * ng;
    // read upper tile (bj, bi): rows G' in block bj, columns G in block bi
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int Gp = bj * 32 + r, G = bi * 32 + threadIdx.x;
        if (Gp < ng && G < ng) t[r][threadIdx.x] = c[(int64_t)Gp * ng + G];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int G = bi * 32 + r, Gp = bj * 32 + threadIdx.x;
        if (G >= ng || Gp >= ng || Gp > G) continue;
        double2 u = t[threadIdx.x][r]; // chi[Gp][G]
        if (Gp == G) c[(int64_t)G * ng + G] = make_double2(u.x, 0.0);
        else c[(int64_t)G * ng + Gp] = make_double2(u.x, -u.y);
    }
}

cudaError_t launch_symmetrize(double2 *chi, int ng, int nw, cudaStream_t st)
{
    if (ng == 0 || nw == 0) return cudaSuccess;
    int nt = (ng + 31) / 32;
    symmetrize_kernel<<<dim3(nt * (nt + 1) / 2, 1, nw), dim3(32, 8), 0, st>>>(chi, ng, nt);
    return cudaGetLastError();
}

// Hermitian part of a square complex matrix: out[i][j] = (W[i][j] + conj(W[j][i])) / 2.  Tile
// (bi, bj) and its transpose pass through shared memory so reads and writes are row-contiguous.
__global__ void herm_part_kernel(const double2 *__restrict__ W, int n, double2 *__restrict__ out)
{
    __shared__ double2 t[32][33];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) { // the transposed tile W[j0 + r][i0 + x]
        const int j = j0 + r, i = i0 + threadIdx.x;
        if (j < n && i < n) t[r][threadIdx.x] = W[(int64_t)j * n + i];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r, j = j0 + threadIdx.x;
        if (i < n && j < n) {
            const double2 a = W[(int64_t)i * n + j], b = t[threadIdx.x][r]; // W[i][j], W[j][i]
            out[(int64_t)i * n + j] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
        }
    }
}

cudaError_t launch_herm_part(const double2 *W, int n, double2 *out, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    herm_part_kernel<<<dim3((n + 31) / 32, (n + 31) / 32), dim3(32, 8), 0, st>>>(W, n, out);
    return cudaGetLastError();
}

// out[g][b] = conj(V[b n + g]): a column-major n x neig block (an eigensolver's vectors of the
// conjugated matrix) to a row-major [n][neig] basis.  32 x 32 tiles through shared memory.
__global__ void conj_transpose_kernel(const double2 *__restrict__ V, int n, int neig, double2 *__restrict__ out)
{
    __shared__ double2 t[32][33];
    const int g0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int b = b0 + r, g = g0 + threadIdx.x;
        if (b < neig && g < n) t[r][threadIdx.x] = V[(int64_t)b * n + g];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int g = g0 + r, b = b0 + threadIdx.x;
        if (g < n && b < neig) {
            const double2 x = t[threadIdx.x][r];
            out[(int64_t)g * neig + b] = make_double2(x.x, -x.y);
        }
    }
}

cudaError_t launch_conj_transpose(const double2 *V, int n, int neig, double2 *out, cudaStream_t st)
{
    if (n == 0 || neig == 0) return cudaSuccess;
    conj_transpose_kernel<<<dim3((n + 31) / 32, (neig + 31) / 32), dim3(32, 8), 0, st>>>(V, n, neig, out);
    return cudaGetLastError();
}

// Watchdog check: one thread waits, with the given bound, on an mbarrier that nothing
// arrives at, exactly as the contraction kernels wait on their TMA and MMA barriers; when
// the bound runs out it records kStatusTimeout and returns, leaving the context usable.
__global__ void watchdog_kernel(long long iters, int *status)
{
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    bar_init(&bar, 1);
    bar_fence_init();
    const uint32_t a = su32(&bar);
    for (long long it = 0; it < iters; ++it) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok)
                     : "r"(a), "r"(0u)
                     : "memory");
        if (ok) return;
    }
    atomicOr(status, kStatusTimeout);
}

cudaError_t launch_watchdog(long long iters, int *status, cudaStream_t st)
{
    watchdog_kernel<<<1, 32, 0, st>>>(iters, status);
    return cudaGetLastError();
}

} // namespace gw
