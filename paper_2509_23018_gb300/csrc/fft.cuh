// FP64 mixed-radix FFT building blocks (sign +, unnormalised) for lines held in shared memory.
//
// Both transforms of the method use the e^{+i...} kernel: the band transform
// psi(r) = sum_K c(K) e^{+iK.r}, and the forward pair transform
// M(G) = (1/N_r) sum_r rho(r) e^{+iG.r} (the 1/N_r is applied by the caller).
//
// The line transform is the Stockham self-sorting formulation: for each stage of
// radix R, butterfly j (0 <= j < n/R) reads x[j + r n/R], multiplies input r by
// w^{r k} with k = j mod Ns and w = e^{+2 pi i/(Ns R)}, applies an R-point DFT and
// writes y[(j div Ns) Ns R + k + r Ns]; Ns grows by R per stage.  Data ping-pong
// between two shared buffers; every thread of the block takes part.
#pragma once
#include "common.cuh"

namespace gw {

constexpr double kSin60 = 0.86602540378443864676;
constexpr double kC1 = 0.30901699437494742410;   // cos(2 pi/5)
constexpr double kS1 = 0.95105651629515357212;   // sin(2 pi/5)
constexpr double kC2 = -0.80901699437494742410;  // cos(4 pi/5)
constexpr double kS2 = 0.58778525229247312917;   // sin(4 pi/5)
constexpr double kRs2 = 0.70710678118654752440;  // 1/sqrt(2)

__device__ __forceinline__ double2 mul_i(double2 a) { return make_double2(-a.y, a.x); }

__device__ __forceinline__ void dft2(double2 *v)
{
    double2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

__device__ __forceinline__ void dft4(double2 *v)
{
    double2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    double2 c = cadd(v[1], v[3]), d = mul_i(csub(v[1], v[3]));
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
}

__device__ __forceinline__ void dft3(double2 *v)
{
    double2 t = cadd(v[1], v[2]);
    double2 s = csub(v[1], v[2]);
    double2 y0 = cadd(v[0], t);
    double2 m = make_double2(fma(-0.5, t.x, v[0].x), fma(-0.5, t.y, v[0].y));
    double2 is = make_double2(-kSin60 * s.y, kSin60 * s.x);
    v[0] = y0;
    v[1] = cadd(m, is);
    v[2] = csub(m, is);
}

__device__ __forceinline__ void dft5(double2 *v)
{
    double2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    double2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    double2 y0 = cadd(v[0], cadd(t1, t2));
    double2 a1 = make_double2(fma(kC1, t1.x, fma(kC2, t2.x, v[0].x)), fma(kC1, t1.y, fma(kC2, t2.y, v[0].y)));
    double2 a2 = make_double2(fma(kC2, t1.x, fma(kC1, t2.x, v[0].x)), fma(kC2, t1.y, fma(kC1, t2.y, v[0].y)));
    double2 b1 = make_double2(fma(kS1, t3.x, kS2 * t4.x), fma(kS1, t3.y, kS2 * t4.y));
    double2 b2 = make_double2(fma(kS2, t3.x, -kS1 * t4.x), fma(kS2, t3.y, -kS1 * t4.y));
    v[0] = y0;
    v[1] = cadd(a1, mul_i(b1));
    v[4] = csub(a1, mul_i(b1));
    v[2] = cadd(a2, mul_i(b2));
    v[3] = csub(a2, mul_i(b2));
}

__device__ __forceinline__ void dft8(double2 *v)
{
    double2 e[4] = {v[0], v[2], v[4], v[6]};
    double2 o[4] = {v[1], v[3], v[5], v[7]};
    dft4(e);
    dft4(o);
    // o[k] *= e^{+i pi k/4}
    o[1] = make_double2(kRs2 * (o[1].x - o[1].y), kRs2 * (o[1].x + o[1].y));
    o[2] = mul_i(o[2]);
    o[3] = make_double2(-kRs2 * (o[3].x + o[3].y), kRs2 * (o[3].x - o[3].y));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = cadd(e[k], o[k]);
        v[k + 4] = csub(e[k], o[k]);
    }
}

template <int R>
__device__ __forceinline__ void dftR(double2 *v)
{
    if constexpr (R == 2) dft2(v);
    else if constexpr (R == 3) dft3(v);
    else if constexpr (R == 4) dft4(v);
    else if constexpr (R == 5) dft5(v);
    else dft8(v);
}

// One Stockham stage of radix R over nlines lines: element i of line l sits at
// base[l*ls + i*es].  tw: n entries e^{+2 pi i t/n} (shared or global memory).
template <int R>
__device__ __forceinline__ void stockham_stage(const double2 *__restrict__ x, double2 *__restrict__ y, int nlines,
                                               int ls, int es, int n, int Ns, const double2 *__restrict__ tw)
{
    const int nb = n / R;
    const int total = nlines * nb;
    const int tstride = n / (Ns * R);
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
        int l = b / nb, j = b - l * nb;
        int k = j % Ns;
        const double2 *xl = x + l * ls;
        double2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = xl[(j + r * nb) * es];
        if (Ns > 1) {
            int e = k * tstride;
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[(r * e) % n]);
        }
        dftR<R>(v);
        double2 *yl = y + l * ls;
        int o = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) yl[(o + r * Ns) * es] = v[r];
    }
}

// Full line transform; returns the buffer that holds the result (a or b).
// Must be called by every thread of the block (contains __syncthreads).
__device__ inline double2 *fft_lines(double2 *a, double2 *b, int nlines, int ls, int es, const FftAxis &ax,
                                     const double2 *tw)
{
    int Ns = 1;
    double2 *x = a, *y = b;
    for (int s = 0; s < ax.nst; ++s) {
        int R = ax.rad[s];
        switch (R) {
        case 2: stockham_stage<2>(x, y, nlines, ls, es, ax.n, Ns, tw); break;
        case 3: stockham_stage<3>(x, y, nlines, ls, es, ax.n, Ns, tw); break;
        case 4: stockham_stage<4>(x, y, nlines, ls, es, ax.n, Ns, tw); break;
        case 5: stockham_stage<5>(x, y, nlines, ls, es, ax.n, Ns, tw); break;
        default: stockham_stage<8>(x, y, nlines, ls, es, ax.n, Ns, tw); break;
        }
        __syncthreads();
        Ns *= R;
        double2 *t = x;
        x = y;
        y = t;
    }
    return x;
}

} // namespace gw
