// lpa_sweep_variants_k16.cu -- the MG ablation variants (paper-literal accumulate, double
// scan) with k = 16 slots.
#include "lpa_sweep_impl.cuh"

namespace lpa {

cudaError_t launch_sweep_mg16_variant(bool literal, bool rescan, const SweepArgs& a,
                                     const WarpPlan& p, cudaStream_t s, cudaStream_t s_hub) {
  return launch_mg_variant<16>(literal, rescan, a, p, s, s_hub);
}

}  // namespace lpa
