// Expansion kernels instantiated for order p = 1.
#include "gen/exp_p1.cuh"
#include "expansion_impl.cuh"

namespace gbfmm {
GBFMM_INSTANTIATE(1)
}  // namespace gbfmm
