// lpa_sweep.cu -- sweep kernels of the sketch modes: MG with k = 1, 2, 4, 8 and BM.
// (k = 16 and k = 32 live in lpa_sweep_k16.cu / lpa_sweep_k32.cu so they compile in
// parallel.)
#include "lpa_sweep_impl.cuh"

namespace lpa {

cudaError_t launch_sweep_warp(int mode, int k, const SweepArgs& a, const WarpPlan& p,
                              cudaStream_t s, cudaStream_t s_hub) {
  if (mode == kBM) return launch_warp_variants<BMState, true>(a, p, s, s_hub);
  switch (k) {
    case 1: return launch_warp_variants<MGSketch<1>>(a, p, s, s_hub);
    case 2: return launch_warp_variants<MGSketch<2>>(a, p, s, s_hub);
    case 4: return launch_warp_variants<MGSketch<4>>(a, p, s, s_hub);
    case 8: return launch_warp_variants<MGSketch<8>, true>(a, p, s, s_hub);
    case 16: return launch_sweep_mg16(a, p, s, s_hub);
    case 32: return launch_sweep_mg32(a, p, s, s_hub);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lpa
