// Expansion kernels instantiated for order p = 5.
#include "gen/exp_p5.cuh"
#include "expansion_impl.cuh"

namespace gbfmm {
GBFMM_INSTANTIATE(5)
}  // namespace gbfmm
