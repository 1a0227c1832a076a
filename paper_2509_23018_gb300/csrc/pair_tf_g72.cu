// Two-float pair kernel instantiated for 72 x 72 slabs.
#include "pair_tf_ct.cuh"

namespace gw {

cudaError_t launch_pair_tf_g72(const float4 *a, const float4 *b, int nc, int64_t p0, int64_t count,
                               const PairPlan &pp, const TfConsts &kc, tf inv, double2 *M, cudaStream_t st)
{
    return launch_pair_tf_grid<72, 72>(a, b, nc, p0, count, pp, kc, inv, M, st);
}

cudaError_t launch_band_fft_tf_g72(float4 *psi, int nb, const FftAxis *ax, const TfConsts &kc, cudaStream_t st)
{
    return launch_band_fft_tf_ct<72>(psi, nb, ax, kc, st);
}

} // namespace gw
