// lpa_sweep_wide.cu -- sweep kernels of the MG mode with k = 16 and 32 slots.
#include "lpa_sweep_impl.cuh"

namespace lpa {

cudaError_t launch_sweep_mg_wide(int k, bool weighted, const SweepArgs& a, const WarpPlan& p,
                                 cudaStream_t s) {
  switch (k) {
    case 16:
      return weighted ? launch_warp_kernel<MGSketch<16>, true>(a, p, s)
                      : launch_warp_kernel<MGSketch<16>, false>(a, p, s);
    case 32:
      return weighted ? launch_warp_kernel<MGSketch<32>, true>(a, p, s)
                      : launch_warp_kernel<MGSketch<32>, false>(a, p, s);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace lpa
