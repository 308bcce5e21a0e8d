// lpa_sweep.cu -- sweep kernels of the sketch modes: MG with k = 1, 2, 4, 8 and BM.
// (k = 16 and 32 live in lpa_sweep_wide.cu so the two compile in parallel.)
#include "lpa_sweep_impl.cuh"

namespace lpa {

cudaError_t launch_sweep_warp(int mode, int k, bool weighted, const SweepArgs& a,
                              const WarpPlan& p, cudaStream_t s) {
  if (mode == kBM)
    return weighted ? launch_warp_kernel<BMState, true>(a, p, s)
                    : launch_warp_kernel<BMState, false>(a, p, s);
  switch (k) {
    case 1:
      return weighted ? launch_warp_kernel<MGSketch<1>, true>(a, p, s)
                      : launch_warp_kernel<MGSketch<1>, false>(a, p, s);
    case 2:
      return weighted ? launch_warp_kernel<MGSketch<2>, true>(a, p, s)
                      : launch_warp_kernel<MGSketch<2>, false>(a, p, s);
    case 4:
      return weighted ? launch_warp_kernel<MGSketch<4>, true>(a, p, s)
                      : launch_warp_kernel<MGSketch<4>, false>(a, p, s);
    case 8:
      return weighted ? launch_warp_kernel<MGSketch<8>, true>(a, p, s)
                      : launch_warp_kernel<MGSketch<8>, false>(a, p, s);
    default:
      return launch_sweep_mg_wide(k, weighted, a, p, s);
  }
}

}  // namespace lpa
