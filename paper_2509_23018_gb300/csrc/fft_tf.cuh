// Two-float ("float-float") arithmetic and the matching FFT building blocks.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2,
// i.e. about 48 significand bits.  On this GPU the FP32 pipes are about 60x faster
// than FP64, so transforms in two-float arithmetic run several times faster than in
// FP64 while keeping a relative rounding level near 2^-46.  The error-free building
// blocks are the classical ones: Knuth's two-sum, Dekker's fast two-sum (|a| >= |b|)
// and the FMA-based exact product (the rounding error of a*b is fma(a, b, -a*b)).
// Explicit __f*_rn intrinsics keep the compiler from contracting or reassociating
// the compensation steps.
#pragma once
#include "common.cuh"

namespace gw {

struct tf {
    float hi, lo;
};
struct tcx {
    tf re, im;
};

__device__ __forceinline__ tf tf_fast2sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ tf tf_2sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ tf tf_add(tf x, tf y)
{
    tf s = tf_2sum(x.hi, y.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return tf_fast2sum(s.hi, e);
}
__device__ __forceinline__ tf tf_sub(tf x, tf y)
{
    tf s = tf_2sum(x.hi, -y.hi);
    float e = __fadd_rn(s.lo, __fsub_rn(x.lo, y.lo));
    return tf_fast2sum(s.hi, e);
}
__device__ __forceinline__ tf tf_neg(tf x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ tf tf_mul(tf x, tf y)
{
    float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return tf_fast2sum(p, e);
}
// x*a + y*b without the final renormalisation: hi is the rounded sum of the two leading
// products, lo collects every lower-order term (|lo| stays within a few ulp of hi)
__device__ __forceinline__ tf tf_dot2l(tf x, tf a, tf y, tf b)
{
    float p1 = __fmul_rn(x.hi, a.hi), p2 = __fmul_rn(y.hi, b.hi);
    float e = __fmaf_rn(x.hi, a.hi, -p1);
    e = __fadd_rn(e, __fmaf_rn(y.hi, b.hi, -p2));
    tf s = tf_2sum(p1, p2);
    e = __fadd_rn(e, s.lo);
    e = __fmaf_rn(x.hi, a.lo, e);
    e = __fmaf_rn(x.lo, a.hi, e);
    e = __fmaf_rn(y.hi, b.lo, e);
    e = __fmaf_rn(y.lo, b.hi, e);
    return {s.hi, e};
}
// F += x*a + y*b with F kept lazy: the hi parts are summed exactly (two-sum) and every
// lower-order term goes into F.lo; renormalise F every few updates.
__device__ __forceinline__ void tf_acc2(tf &F, tf x, tf a, tf y, tf b)
{
    float p1 = __fmul_rn(x.hi, a.hi), p2 = __fmul_rn(y.hi, b.hi);
    float e = __fmaf_rn(x.hi, a.hi, -p1);
    e = __fadd_rn(e, __fmaf_rn(y.hi, b.hi, -p2));
    tf s = tf_2sum(p1, p2);
    tf u = tf_2sum(F.hi, s.hi);
    e = __fmaf_rn(x.hi, a.lo, e);
    e = __fmaf_rn(x.lo, a.hi, e);
    e = __fmaf_rn(y.hi, b.lo, e);
    e = __fmaf_rn(y.lo, b.hi, e);
    F = {u.hi, __fadd_rn(F.lo, __fadd_rn(e, __fadd_rn(s.lo, u.lo)))};
}
// x*a + y*b with one final renormalisation
__device__ __forceinline__ tf tf_dot2(tf x, tf a, tf y, tf b)
{
    float p1 = __fmul_rn(x.hi, a.hi), p2 = __fmul_rn(y.hi, b.hi);
    float e = __fmaf_rn(x.hi, a.hi, -p1);
    e = __fadd_rn(e, __fmaf_rn(y.hi, b.hi, -p2));
    tf s = tf_2sum(p1, p2);
    e = __fadd_rn(e, s.lo);
    e = __fmaf_rn(x.hi, a.lo, e);
    e = __fmaf_rn(x.lo, a.hi, e);
    e = __fmaf_rn(y.hi, b.lo, e);
    e = __fmaf_rn(y.lo, b.hi, e);
    return tf_fast2sum(s.hi, e);
}
__device__ __forceinline__ tf tf_scale(tf x, float c) // c a power of two
{
    return {__fmul_rn(x.hi, c), __fmul_rn(x.lo, c)};
}
__device__ __forceinline__ double tf_to_d(tf x) { return (double)x.hi + (double)x.lo; }

// Lazy sums: the exact sum of the hi parts plus every low-order term, without the final
// renormalisation.  Chains of these inside one butterfly keep the ~2^-46 relative level;
// tc_norm renormalises the butterfly's outputs once.
__device__ __forceinline__ tf tf_addl(tf x, tf y)
{
    tf s = tf_2sum(x.hi, y.hi);
    return {s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo))};
}
__device__ __forceinline__ tf tf_subl(tf x, tf y)
{
    tf s = tf_2sum(x.hi, -y.hi);
    return {s.hi, __fadd_rn(s.lo, __fsub_rn(x.lo, y.lo))};
}
__device__ __forceinline__ tf tf_norm(tf x) { return tf_fast2sum(x.hi, x.lo); }

__device__ __forceinline__ tcx tc_add(tcx a, tcx b) { return {tf_add(a.re, b.re), tf_add(a.im, b.im)}; }
__device__ __forceinline__ tcx tc_sub(tcx a, tcx b) { return {tf_sub(a.re, b.re), tf_sub(a.im, b.im)}; }
__device__ __forceinline__ tcx tc_muli(tcx a) { return {tf_neg(a.im), a.re}; }
__device__ __forceinline__ tcx tc_addl(tcx a, tcx b) { return {tf_addl(a.re, b.re), tf_addl(a.im, b.im)}; }
__device__ __forceinline__ tcx tc_subl(tcx a, tcx b) { return {tf_subl(a.re, b.re), tf_subl(a.im, b.im)}; }
__device__ __forceinline__ tcx tc_norm(tcx a) { return {tf_norm(a.re), tf_norm(a.im)}; }
// a * w
__device__ __forceinline__ tcx tc_mul(tcx a, tcx w)
{
    return {tf_dot2(a.re, w.re, tf_neg(a.im), w.im), tf_dot2(a.re, w.im, a.im, w.re)};
}
// a * w, lazy (feeds lazy sums or another renormalising step)
__device__ __forceinline__ tcx tc_mull(tcx a, tcx w)
{
    return {tf_dot2l(a.re, w.re, tf_neg(a.im), w.im), tf_dot2l(a.re, w.im, a.im, w.re)};
}
// F += a * w, F lazy
__device__ __forceinline__ void tc_acc(tcx &F, tcx a, tcx w)
{
    tf_acc2(F.re, a.re, w.re, tf_neg(a.im), w.im);
    tf_acc2(F.im, a.re, w.im, a.im, w.re);
}
// conj(a) * b, lazy (feeds lazy sums)
__device__ __forceinline__ tcx tc_mulcl(tcx a, tcx b)
{
    return {tf_dot2l(a.re, b.re, a.im, b.im), tf_dot2l(a.re, b.im, tf_neg(a.im), b.re)};
}
// conj(a) * b
__device__ __forceinline__ tcx tc_mulc(tcx a, tcx b)
{
    return {tf_dot2(a.re, b.re, a.im, b.im), tf_dot2(a.re, b.im, tf_neg(a.im), b.re)};
}
// real two-float constant times a complex value
__device__ __forceinline__ tcx tc_rmul(tcx a, tf c) { return {tf_mul(a.re, c), tf_mul(a.im, c)}; }

__device__ __forceinline__ tcx tc_load(const float4 *p)
{
    float4 v = *p;
    return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ void tc_store(float4 *p, tcx a) { *p = make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }

// two-float butterfly constants (hi + lo of the FP64 values)
struct TfConsts {
    tf sin60, c1, s1, c2, s2, rs2;
};
TfConsts tf_consts(); // host: the constants above from their FP64 values (mtxel.cu)
__device__ __forceinline__ tf tf_from(double x)
{
    float h = (float)x;
    return {h, (float)(x - (double)h)};
}

__device__ __forceinline__ void tdft2(tcx *v)
{
    tcx a = v[0], b = v[1];
    v[0] = tc_add(a, b);
    v[1] = tc_sub(a, b);
}
template <bool NORM = true>
__device__ __forceinline__ void tdft4(tcx *v)
{
    tcx a = tc_addl(v[0], v[2]), b = tc_subl(v[0], v[2]);
    tcx c = tc_addl(v[1], v[3]), d = tc_muli(tc_subl(v[1], v[3]));
    v[0] = tc_addl(a, c);
    v[2] = tc_subl(a, c);
    v[1] = tc_addl(b, d);
    v[3] = tc_subl(b, d);
    if constexpr (NORM) {
#pragma unroll
        for (int r = 0; r < 4; ++r) v[r] = tc_norm(v[r]);
    }
}
__device__ __forceinline__ void tdft3(tcx *v, const TfConsts &k)
{
    tcx t = tc_addl(v[1], v[2]);
    tcx s = tc_subl(v[1], v[2]);
    tcx y0 = tc_addl(v[0], t);
    tcx m = tc_subl(v[0], {tf_scale(t.re, 0.5f), tf_scale(t.im, 0.5f)});
    tcx is = tc_muli(tc_rmul(s, k.sin60));
    v[0] = tc_norm(y0);
    v[1] = tc_norm(tc_addl(m, is));
    v[2] = tc_norm(tc_subl(m, is));
}
__device__ __forceinline__ void tdft5(tcx *v, const TfConsts &k)
{
    tcx t1 = tc_add(v[1], v[4]), t2 = tc_add(v[2], v[3]);
    tcx t3 = tc_sub(v[1], v[4]), t4 = tc_sub(v[2], v[3]);
    tcx y0 = tc_add(v[0], tc_add(t1, t2));
    tcx a1 = tc_add(v[0], tc_add(tc_rmul(t1, k.c1), tc_rmul(t2, k.c2)));
    tcx a2 = tc_add(v[0], tc_add(tc_rmul(t1, k.c2), tc_rmul(t2, k.c1)));
    tcx b1 = tc_muli(tc_add(tc_rmul(t3, k.s1), tc_rmul(t4, k.s2)));
    tcx b2 = tc_muli(tc_sub(tc_rmul(t3, k.s2), tc_rmul(t4, k.s1)));
    v[0] = y0;
    v[1] = tc_add(a1, b1);
    v[4] = tc_sub(a1, b1);
    v[2] = tc_add(a2, b2);
    v[3] = tc_sub(a2, b2);
}
__device__ __forceinline__ void tdft8(tcx *v, const TfConsts &k)
{
    tcx e[4] = {v[0], v[2], v[4], v[6]};
    tcx o[4] = {v[1], v[3], v[5], v[7]};
    tdft4<false>(e);
    tdft4<false>(o);
    // o[k] *= e^{+i pi k/4}
    o[1] = tc_rmul({tf_subl(o[1].re, o[1].im), tf_addl(o[1].re, o[1].im)}, k.rs2);
    o[2] = tc_muli(o[2]);
    o[3] = tc_rmul({tf_neg(tf_addl(o[3].re, o[3].im)), tf_subl(o[3].re, o[3].im)}, k.rs2);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v[j] = tc_norm(tc_addl(e[j], o[j]));
        v[j + 4] = tc_norm(tc_subl(e[j], o[j]));
    }
}

template <int R>
__device__ __forceinline__ void tdftR(tcx *v, const TfConsts &k)
{
    if constexpr (R == 2) tdft2(v);
    else if constexpr (R == 3) tdft3(v, k);
    else if constexpr (R == 4) tdft4<true>(v);
    else if constexpr (R == 5) tdft5(v, k);
    else tdft8(v, k);
}

// Stockham stage (same index scheme as the FP64 version in fft.cuh), two-float data.
template <int R>
__device__ __forceinline__ void tstockham_stage(const float4 *__restrict__ x, float4 *__restrict__ y, int nlines,
                                                int ls, int es, int n, int Ns, const float4 *__restrict__ tw,
                                                const TfConsts &k)
{
    const int nb = n / R;
    const int total = nlines * nb;
    const int tstride = n / (Ns * R);
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
        int l = b / nb, j = b - l * nb;
        int kk = j % Ns;
        const float4 *xl = x + l * ls;
        tcx v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = tc_load(xl + (j + r * nb) * es);
        if (Ns > 1) {
            int e = kk * tstride;
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = tc_mul(v[r], tc_load(tw + (r * e) % n));
        }
        tdftR<R>(v, k);
        float4 *yl = y + l * ls;
        int o = (j / Ns) * Ns * R + kk;
#pragma unroll
        for (int r = 0; r < R; ++r) tc_store(yl + (o + r * Ns) * es, v[r]);
    }
}

// Full line transform in two-float arithmetic; returns the buffer holding the result.
__device__ inline float4 *tfft_lines(float4 *a, float4 *b, int nlines, int ls, int es, const FftAxis &ax,
                                     const float4 *tw, const TfConsts &k)
{
    int Ns = 1;
    float4 *x = a, *y = b;
    for (int s = 0; s < ax.nst; ++s) {
        int R = ax.rad[s];
        switch (R) {
        case 2: tstockham_stage<2>(x, y, nlines, ls, es, ax.n, Ns, tw, k); break;
        case 3: tstockham_stage<3>(x, y, nlines, ls, es, ax.n, Ns, tw, k); break;
        case 4: tstockham_stage<4>(x, y, nlines, ls, es, ax.n, Ns, tw, k); break;
        case 5: tstockham_stage<5>(x, y, nlines, ls, es, ax.n, Ns, tw, k); break;
        default: tstockham_stage<8>(x, y, nlines, ls, es, ax.n, Ns, tw, k); break;
        }
        __syncthreads();
        Ns *= R;
        float4 *t = x;
        x = y;
        y = t;
    }
    return x;
}

} // namespace gw

namespace gw {

// ------------------------------------------------------------------ compile-time line plans
// The same Stockham scheme with the line length known at compile time: the butterfly
// and twiddle index arithmetic folds into constants, which matters because the two-float
// butterflies leave little issue bandwidth to spare.  Radix order as on the host:
// 3s, 5s, 4s, one 8 (a 2 merged with a 4), 2.
struct RadPlan {
    int nst;
    int r[kMaxStages];
};
constexpr RadPlan make_rad_plan(int n)
{
    RadPlan p{0, {0, 0, 0, 0, 0, 0, 0, 0}};
    int m = n, n4 = 0, n2 = 0, n3 = 0, n5 = 0;
    while (m % 4 == 0) { ++n4; m /= 4; }
    while (m % 2 == 0) { ++n2; m /= 2; }
    while (m % 3 == 0) { ++n3; m /= 3; }
    while (m % 5 == 0) { ++n5; m /= 5; }
    int n8 = 0;
    if (n2 && n4) { n2 = 0; --n4; n8 = 1; }
    for (int i = 0; i < n3; ++i) p.r[p.nst++] = 3;
    for (int i = 0; i < n5; ++i) p.r[p.nst++] = 5;
    for (int i = 0; i < n4; ++i) p.r[p.nst++] = 4;
    for (int i = 0; i < n8; ++i) p.r[p.nst++] = 8;
    for (int i = 0; i < n2; ++i) p.r[p.nst++] = 2;
    return p;
}

// Plan whose last stage is formed output by output (pruned): the smallest available radix
// goes last, so each kept output costs R - 1 twiddle products.
constexpr int prune_radix(int n) { return n % 3 == 0 ? 3 : (n % 2 == 0 ? 2 : 5); }
constexpr RadPlan make_prune_plan(int n)
{
    RadPlan p = make_rad_plan(n / prune_radix(n));
    p.r[p.nst++] = prune_radix(n);
    return p;
}
template <int N, bool PR>
constexpr RadPlan plan_of()
{
    return PR ? make_prune_plan(N) : make_rad_plan(N);
}

// Work split of a block-level stage over its butterflies (line l, index j).  By default j runs
// fastest over the threads: consecutive lanes read consecutive points of a line, right for lines
// at an even stride.  With lines fastest consecutive lanes take consecutive lines, which keeps a
// warp's 16-byte accesses in distinct bank groups when the line stride is odd (N + 1) or the
// lines are contiguous (element stride N); the thread's first butterfly and its step are
// computed once per transform.
struct LMap {
    int j0, l0, dj, dl;
};
__device__ __forceinline__ LMap lmap_lines_fastest(int nlines)
{
    LMap m{1 << 30, 0, 0, 0};
    if (nlines > 0) {
        m.j0 = (int)threadIdx.x / nlines;
        m.l0 = (int)threadIdx.x - m.j0 * nlines;
        m.dj = (int)blockDim.x / nlines;
        m.dl = (int)blockDim.x - m.dj * nlines;
    }
    return m;
}

// lines of N points, line l at x + l * ls, element stride es; LAZY leaves radix-4 outputs
// unrenormalised (for stages whose outputs feed another lazy stage)
// lmax >= 0 skips the lines l whose signed index (l, or l - N above N/2) exceeds lmax in
// magnitude (all-zero lines whose outputs stay zero in both ping-pong buffers).
// LF: lines fastest over the threads, in the split lm (see LMap).
template <int N, int R, int NS, bool LAZY = false, bool LF = false>
__device__ __forceinline__ void tstage_ct(const float4 *__restrict__ x, float4 *__restrict__ y, int nlines, int ls,
                                          const float4 *__restrict__ tw, const TfConsts &k, int es = 1,
                                          int lmax = -1, LMap lm = LMap{})
{
    constexpr int nb = N / R;
    constexpr int tstride = N / (NS * R); // r * kk * tstride < N: no reduction needed
    auto bfly = [&](int l, int j) {
        if (lmax >= 0 && (l <= N / 2 ? l : N - l) > lmax) return;
        const int kk = j % NS;
        const float4 *xl = x + l * ls;
        tcx v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = tc_load(xl + (j + r * nb) * es);
        if constexpr (NS > 1) {
            const int e = kk * tstride;
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = tc_mull(v[r], tc_load(tw + r * e));
        }
        if constexpr (LAZY && R == 4) tdft4<false>(v);
        else tdftR<R>(v, k);
        float4 *yl = y + l * ls;
        const int o = (j / NS) * (NS * R) + kk;
#pragma unroll
        for (int r = 0; r < R; ++r) tc_store(yl + (o + r * NS) * es, v[r]);
    };
    if constexpr (LF) {
        int l = lm.l0, j = lm.j0;
        while (j < nb) {
            bfly(l, j);
            l += lm.dl;
            j += lm.dj;
            if (l >= nlines) {
                l -= nlines;
                ++j;
            }
        }
    } else {
        const int total = nlines * nb;
        for (int b = threadIdx.x; b < total; b += blockDim.x) {
            const int l = b / nb;
            bfly(l, b - l * nb);
        }
    }
}

// Stages S.. of the plan (all of make_rad_plan(N), or all but the pruned last one of
// make_prune_plan(N)), block-wide with a barrier after each; returns the result buffer.
// With PR the stages are lazy: their outputs only feed the pruned stage's lazy sums.
// LF: lines fastest over the threads (see LMap).
template <int N, int S, int NS, bool PR = false, bool LF = false>
__device__ __forceinline__ float4 *tstages_ct(float4 *x, float4 *y, int nlines, int ls, const float4 *tw,
                                              const TfConsts &k, int es, int lmax = -1, LMap lm = LMap{})
{
    constexpr RadPlan P = plan_of<N, PR>();
    if constexpr (S >= P.nst - (PR ? 1 : 0)) {
        return x;
    } else {
        if constexpr (LF && S == 0) lm = lmap_lines_fastest(nlines);
        constexpr int R = P.r[S];
        tstage_ct<N, R, NS, PR, LF>(x, y, nlines, ls, tw, k, es, lmax, lm);
        __syncthreads();
        return tstages_ct<N, S + 1, NS * R, PR, LF>(y, x, nlines, ls, tw, k, es, lmax, lm);
    }
}

// Full two-float transform of nlines lines of length N (line stride ls, element stride es);
// returns the result buffer.  lmax >= 0: lines beyond it are zero and skipped (see tstage_ct).
template <int N, bool LF = false>
__device__ __forceinline__ float4 *tfft_lines_ct(float4 *a, float4 *b, int nlines, int ls, const float4 *tw,
                                                 const TfConsts &k, int es = 1, int lmax = -1)
{
    return tstages_ct<N, 0, 1, false, LF>(a, b, nlines, ls, tw, k, es, lmax);
}

// Warp-level stage over the calling warp's own lines (L lines of N points at x + l * N);
// the warp's stages are separated by __syncwarp only.
template <int N, int R, int NS, int L>
__device__ __forceinline__ void wstage_ct(const float4 *__restrict__ x, float4 *__restrict__ y,
                                          const float4 *__restrict__ tw, const TfConsts &k)
{
    constexpr int nb = N / R, total = L * nb, rounds = (total + 31) / 32;
    constexpr int tstride = N / (NS * R);
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int it = 0; it < rounds; ++it) {
        const int b = lane + 32 * it;
        if (total % 32 == 0 || b < total) {
            const int l = b / nb, j = b - l * nb;
            const int kk = j % NS;
            const float4 *xl = x + l * N;
            tcx v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = tc_load(xl + j + r * nb);
            if constexpr (NS > 1) {
                const int e = kk * tstride;
#pragma unroll
                for (int r = 1; r < R; ++r) v[r] = tc_mull(v[r], tc_load(tw + r * e));
            }
            tdftR<R>(v, k);
            float4 *yl = y + l * N;
            const int o = (j / NS) * (NS * R) + kk;
#pragma unroll
            for (int r = 0; r < R; ++r) tc_store(yl + o + r * NS, v[r]);
        }
    }
}

// Warp-level stages S.. of make_prune_plan(N) except the pruned last one; returns the
// buffer holding their result.
template <int N, int S, int NS, int L>
__device__ __forceinline__ float4 *wstages_ct(float4 *x, float4 *y, const float4 *tw, const TfConsts &k)
{
    constexpr RadPlan P = make_prune_plan(N);
    if constexpr (S + 1 >= P.nst) {
        return x;
    } else {
        constexpr int R = P.r[S];
        wstage_ct<N, R, NS, L>(x, y, tw, k);
        __syncwarp();
        return wstages_ct<N, S + 1, NS * R, L>(y, x, tw, k);
    }
}

// Output k of the pruned last stage of make_prune_plan(N), R its radix: with the earlier
// stages done, x holds the R interleaved (N/R)-point transforms Y_r at x[r N/R + j], and
// X[k] = sum_r W^{r k} Y_r[k mod N/R] (decimation in time; tw[i] = W^i).
template <int N>
__device__ __forceinline__ tcx tprune_ct(const float4 *__restrict__ x, int k, const float4 *__restrict__ tw)
{
    constexpr int R = prune_radix(N), NS = N / R;
    const int j = k % NS;
    tcx acc = tc_load(x + j);
    int e = 0;
#pragma unroll
    for (int r = 1; r < R; ++r) {
        e += k;
        if (e >= N) e -= N;
        acc = tc_addl(acc, tc_mull(tc_load(x + j + r * NS), tc_load(tw + e)));
    }
    return tc_norm(acc);
}

} // namespace gw
