// lpa_sweep_variants.cu -- the MG ablation axes of the paper: the paper-literal
// accumulate of Alg. 2 (LPA_MG_UNCLAMPED) and the double scan of Sec. 4.4 (LPA_RESCAN),
// for k <= 8 here and k = 16, 32 in lpa_sweep_variants_k16.cu / _k32.cu (translation
// units of their own so they compile in parallel beside the main sweep).
#include "lpa_sweep_impl.cuh"

namespace lpa {

cudaError_t launch_sweep_mg_variant(int k, bool literal, bool rescan, const SweepArgs& a,
                                    const WarpPlan& p, cudaStream_t s, cudaStream_t s_hub) {
  switch (k) {
    case 1: return launch_mg_variant<1>(literal, rescan, a, p, s, s_hub);
    case 2: return launch_mg_variant<2>(literal, rescan, a, p, s, s_hub);
    case 4: return launch_mg_variant<4>(literal, rescan, a, p, s, s_hub);
    case 8: return launch_mg_variant<8>(literal, rescan, a, p, s, s_hub);
    case 16: return launch_sweep_mg16_variant(literal, rescan, a, p, s, s_hub);
    case 32: return launch_sweep_mg32_variant(literal, rescan, a, p, s, s_hub);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lpa
