// lpa_sweep_k32.cu -- sweep kernels of the MG mode with k = 32 slots.
#include "lpa_sweep_impl.cuh"

namespace lpa {

cudaError_t launch_sweep_mg32(const SweepArgs& a, const WarpPlan& p, cudaStream_t s,
                              cudaStream_t s_hub) {
  return launch_warp_variants<MGSketch<32>>(a, p, s, s_hub);
}

}  // namespace lpa
