// Shared device/host helpers of the chi0 CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace gw {

// ----------------------------------------------------------------- complex FP64
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ double2 cmulc(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
// acc += a * b
__device__ __forceinline__ void cfma(double2 &acc, double2 a, double2 b)
{
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}

// ----------------------------------------------------------------- FFT axis plan
// One axis of length n = prod(rad[0..nst)), radices in {2,3,4,5,8}.  tw[t] = e^{+2 pi i t/n}.
constexpr int kMaxStages = 8;
struct FftAxis {
    int n;
    int nst;
    int rad[kMaxStages];
    const double2 *tw;  // device, n entries
    const float4 *twf;  // device, n entries in two-float form (re.hi, re.lo, im.hi, im.lo)
};

// Device-side status word bits (written by bounded waits that gave up).
constexpr int kStatusTimeout = 1;
constexpr int kStatusNoSlot = 2; // a pair block found no free scratch slot
constexpr int kStatusBounds = 4; // an index outside its buffer (bounds-checked build only)

// Bounds checks of the bounds-checked build (compiled with -DGW_DEBUG, see build.py): an index
// outside [0, n) records kStatusBounds in the status word and the access is skipped; in the
// normal build the check compiles to true.
#ifdef GW_DEBUG
__device__ __forceinline__ bool gw_in_range(long long i, long long n, int *status)
{
    if (i >= 0 && i < n) return true;
    if (status) atomicOr(status, kStatusBounds);
    return false;
}
#define GW_IN(i, n, status) ::gw::gw_in_range((long long)(i), (long long)(n), (status))
#else
#define GW_IN(i, n, status) true
#endif

} // namespace gw
