// Digit step of the split (Ozaki) representation in integer arithmetic.
//
// A value x of a row or column with exponent E (E = ilogb of the row's largest magnitude + 2)
// is written as x = 2^E sum_{i=0..s-1} 2^(-6 (i + 1)) d_i with balanced base-64 digits: the
// integer N = round(x 2^(6 s - E)) (to nearest, ties to even) is cut into d_{s-1}, ..., d_1 in
// [-32, 31] from the least significant end and d_0, which keeps the rest.  N is formed from the
// bits of x and the digits are bit fields of N + sum_{k < s-1} 32 64^k (its plain base-64 fields
// are d_k + 32), so no step runs on the FP64 pipe (1/64 of the FP32 rate on this GPU) or on the
// 64-bit conversion units.  Host and device compile the same code.
#pragma once
#include <cstdint>
#include <cstring>

namespace gw {

__host__ __device__ __forceinline__ unsigned long long oz_dbits(double x)
{
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long b;
    std::memcpy(&b, &x, sizeof b);
    return b;
#endif
}

__host__ __device__ __forceinline__ double oz_bits_d(unsigned long long b)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double x;
    std::memcpy(&x, &b, sizeof x);
    return x;
#endif
}

// max(|x|, |y|) by the magnitude bits (the order of non-negative doubles is that of their bits)
__host__ __device__ __forceinline__ unsigned long long oz_absmax_bits(double x, double y)
{
    const unsigned long long a = oz_dbits(x) & 0x7fffffffffffffffull, b = oz_dbits(y) & 0x7fffffffffffffffull;
    return a > b ? a : b;
}

// ilogb(a) + 2 from the bits of a >= 0 (subnormals count as 2^-1023), no_column for a = 0
__host__ __device__ __forceinline__ int oz_expo_bits(unsigned long long a, int no_column)
{
    if (a == 0) return no_column;
    const int be = (int)(a >> 52);
    return (be == 0 ? -1023 : be - 1023) + 2;
}

// ilogb(a) + 2 if a > 0 (positive finite or +inf), no_column otherwise (+0, -0, negative, NaN).
// The column scans use it on a = max(|Re M|, |Im M|) s_p, where s_p = sqrt(-Delta) is -0 for a
// weight that is exactly +0 (the sign-split real-axis weights have many).
__host__ __device__ __forceinline__ int oz_expo_pos(double a, int no_column)
{
    const unsigned long long b = oz_dbits(a);
    return (b - 1ull) < 0x7ff0000000000000ull ? oz_expo_bits(b, no_column) : no_column;
}

// round(x 2^h), ties to even, h = sh clamped to [-1022, 1023].  The split's exponent bounds
// |x 2^h| by 2^47, so N is formed by one right shift of the 53-bit significand (k >= 6).
__host__ __device__ __forceinline__ long long oz_round_scaled(double x, int sh)
{
    const int h = sh < -1022 ? -1022 : (sh > 1023 ? 1023 : sh);
    const unsigned long long b = oz_dbits(x);
    const int be = (int)((b >> 52) & 0x7ff);
    const unsigned long long m = (b & 0xfffffffffffffull) | (be != 0 ? (1ull << 52) : 0ull);
    const int k = 1075 - (be != 0 ? be : 1) - h; // |x| 2^h = m 2^-k
    unsigned long long q;
    if (k <= 0) {
        q = m << (-k < 10 ? -k : 10); // outside the split's range (|x 2^h| >= 2^52); kept defined
    } else if (k > 60) {
        q = 0; // |x| 2^h < 2^-7
    } else {
        q = m >> k;
        const unsigned long long r = m & ((1ull << k) - 1ull), half = 1ull << (k - 1);
        q += (r > half || (r == half && (q & 1ull))) ? 1ull : 0ull;
    }
    return (b >> 63) ? -(long long)q : (long long)q;
}

// sum_{k < s-1} 32 64^k: added to N it turns the balanced digits d_k into the fields d_k + 32
__host__ __device__ __forceinline__ long long oz_digit_bias(int s)
{
    long long b = 0;
    for (int k = 0; k < s - 1; ++k) b |= 32ll << (6 * k);
    return b;
}

// BF16 bit pattern of a small integer v (|v| < 2^22; exact): 1.5 2^23 + v is an FP32 number
// whose significand holds v, and the subtraction is exact
__host__ __device__ __forceinline__ uint16_t oz_small_bf16(int v)
{
#ifdef __CUDA_ARCH__
    const float f = __int_as_float(0x4B400000 + v) - 12582912.0f;
    return (uint16_t)(__float_as_uint(f) >> 16);
#else
    const unsigned u0 = 0x4B400000u + (unsigned)v;
    float f;
    std::memcpy(&f, &u0, sizeof f);
    f -= 12582912.0f;
    unsigned u;
    std::memcpy(&u, &f, sizeof u);
    return (uint16_t)(u >> 16);
#endif
}

// the s digits of N, d_i at out[i plane] (d_0 the most significant); bias = oz_digit_bias(s)
__host__ __device__ __forceinline__ void oz_store_digits(long long N, int s, long long bias, uint16_t *out,
                                                         int64_t plane)
{
    const long long nb = N + bias;
    for (int k = 0; k < s - 1; ++k)
        out[(int64_t)(s - 1 - k) * plane] = oz_small_bf16((int)((nb >> (6 * k)) & 63) - 32);
    out[0] = oz_small_bf16((int)(nb >> (6 * (s - 1))));
}

} // namespace gw
