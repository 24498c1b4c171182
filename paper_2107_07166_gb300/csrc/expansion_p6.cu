// Expansion kernels instantiated for order p = 6.
#include "gen/exp_p6.cuh"
#include "expansion_impl.cuh"

namespace gbfmm {
GBFMM_INSTANTIATE(6)
}  // namespace gbfmm
