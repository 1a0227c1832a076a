// Two-float pair kernel and band setup instantiated for the 48^3 grid.
#include "pair_tf_ct.cuh"

namespace gw {

cudaError_t launch_pair_tf_g48(const float4 *a, const float4 *b, int nc, int64_t p0, int64_t count,
                               const PairPlan &pp, const TfConsts &kc, tf inv, double2 *M, cudaStream_t st)
{
    return launch_pair_tf_cube<48>(a, b, nc, p0, count, pp, kc, inv, M, st);
}

cudaError_t pair_tf_slots_g48(const PairPlan &pp, int *nslots) { return pair_tf_cube_slots<48>(pp, nslots); }

cudaError_t launch_pair_tf_from_f_g48(const CUtensorMap &tmF, const CUtensorMap &tmS, int64_t R, const PairPlan &pp,
                                      const TfConsts &kc, tf inv, double2 *M, cudaStream_t st)
{
    return launch_pair_tf_from_f_cube<48>(tmF, tmS, R, pp, kc, inv, M, st);
}

cudaError_t launch_band_fft_tf_g48(float4 *psi, int nb, const FftAxis *ax, const TfConsts &kc, int m0, int m1,
                                  cudaStream_t st)
{
    return launch_band_fft_tf_ct<48>(psi, nb, ax, kc, m0, m1, st);
}

} // namespace gw
