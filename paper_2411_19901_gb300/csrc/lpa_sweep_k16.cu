// lpa_sweep_k16.cu -- sweep kernels of the MG mode with k = 16 slots.
#include "lpa_sweep_impl.cuh"

namespace lpa {

cudaError_t launch_sweep_mg16(const SweepArgs& a, const WarpPlan& p, cudaStream_t s,
                              cudaStream_t s_hub) {
  return launch_warp_variants<MGSketch<16>>(a, p, s, s_hub);
}

}  // namespace lpa
