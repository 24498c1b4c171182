// Expansion kernels instantiated for order p = 2.
#include "gen/exp_p2.cuh"
#include "expansion_impl.cuh"

namespace gbfmm {
GBFMM_INSTANTIATE(2)
}  // namespace gbfmm
