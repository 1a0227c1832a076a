// Dielectric matrix inverse eps^-1 = [I - v chi]^-1 (Eq. epsilon, with the Coulomb
// interaction v_G given by the caller) for each frequency block of chi.
//
// With s_G = sqrt(v_G), eps = s (I - s chi s) s^-1, so eps^-1 = s A^-1 s^-1 with the
// Hermitian A = I - s chi s, whose eigenvalues are >= 1 because chi is negative
// semidefinite.  A^-1 is reached by the Newton-Schulz iteration X <- 2X - X (A X) from
// X0 = a I, a = 2 / (1 + b), b >= lambda_max(A) a Gershgorin bound: the error I - A X
// squares every step, from at most (b - 1)/(b + 1).  The two products per step are dense
// matrix products (split precision on the tensor cores, or FP64 DMMA).  These kernels do
// the elementwise parts.
#include "internal.h"

namespace gw {

// A[i][j] = delta_ij - s_i chi[i][j] s_j
__global__ void eps_sym_kernel(const double2 *__restrict__ chi, const double *__restrict__ sv, int ng,
                               double2 *__restrict__ A)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)ng * ng) return;
    const int i = (int)(e / ng), j = (int)(e - (int64_t)i * ng);
    const double2 c = chi[e];
    const double f = sv[i] * sv[j];
    A[e] = make_double2((i == j ? 1.0 : 0.0) - f * c.x, -f * c.y);
}

// b = max_i sum_j |A[i][j]| (one block per row; the maximum is taken with an integer
// atomic on the bits of a non-negative double, which order like the values)
__global__ void eps_gersh_kernel(const double2 *__restrict__ A, int ng, unsigned long long *__restrict__ bmax)
{
    __shared__ double red[32];
    const double2 *row = A + (int64_t)blockIdx.x * ng;
    double acc = 0.0;
    for (int j = threadIdx.x; j < ng; j += blockDim.x) acc += hypot(row[j].x, row[j].y);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) atomicMax(bmax, (unsigned long long)__double_as_longlong(acc));
    }
}

// X = a I with a = 2 / (1 + b)
__global__ void eps_init_kernel(double2 *__restrict__ X, int ng, const unsigned long long *__restrict__ bmax)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)ng * ng) return;
    const int i = (int)(e / ng), j = (int)(e - (int64_t)i * ng);
    const double a = 2.0 / (1.0 + __longlong_as_double((long long)*bmax));
    X[e] = make_double2(i == j ? a : 0.0, 0.0);
}

// X = 2 X - P  (P = X A X)
__global__ void eps_step_kernel(double2 *__restrict__ X, const double2 *__restrict__ P, int64_t n)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double2 x = X[e], p = P[e];
    X[e] = make_double2(2.0 * x.x - p.x, 2.0 * x.y - p.y);
}

// out[i][j] = s_i X[i][j] / s_j
__global__ void eps_unsym_kernel(const double2 *__restrict__ X, const double *__restrict__ sv, int ng,
                                 double2 *__restrict__ out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)ng * ng) return;
    const int i = (int)(e / ng), j = (int)(e - (int64_t)i * ng);
    const double f = sv[i] / sv[j];
    const double2 x = X[e];
    out[e] = make_double2(f * x.x, f * x.y);
}

__global__ void eps_sqrt_kernel(const double *__restrict__ v, int ng, double *__restrict__ sv)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ng) sv[i] = sqrt(v[i]);
}

static unsigned blocks(int64_t n) { return (unsigned)((n + 255) / 256); }

cudaError_t launch_eps_sqrt(const double *v, int ng, double *sv, cudaStream_t st)
{
    eps_sqrt_kernel<<<blocks(ng), 256, 0, st>>>(v, ng, sv);
    return cudaGetLastError();
}

cudaError_t launch_eps_sym(const double2 *chi, const double *sv, int ng, double2 *A, unsigned long long *bmax,
                           cudaStream_t st)
{
    eps_sym_kernel<<<blocks((int64_t)ng * ng), 256, 0, st>>>(chi, sv, ng, A);
    cudaError_t e = cudaMemsetAsync(bmax, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    eps_gersh_kernel<<<ng, 256, 0, st>>>(A, ng, bmax);
    return cudaGetLastError();
}

cudaError_t launch_eps_init(double2 *X, int ng, const unsigned long long *bmax, cudaStream_t st)
{
    eps_init_kernel<<<blocks((int64_t)ng * ng), 256, 0, st>>>(X, ng, bmax);
    return cudaGetLastError();
}

cudaError_t launch_eps_step(double2 *X, const double2 *P, int64_t n, cudaStream_t st)
{
    eps_step_kernel<<<blocks(n), 256, 0, st>>>(X, P, n);
    return cudaGetLastError();
}

cudaError_t launch_eps_unsym(const double2 *X, const double *sv, int ng, double2 *out, cudaStream_t st)
{
    eps_unsym_kernel<<<blocks((int64_t)ng * ng), 256, 0, st>>>(X, sv, ng, out);
    return cudaGetLastError();
}

} // namespace gw
