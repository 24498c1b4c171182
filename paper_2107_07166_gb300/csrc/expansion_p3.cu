// Expansion kernels instantiated for order p = 3.
#include "gen/exp_p3.cuh"
#include "expansion_impl.cuh"

namespace gbfmm {
GBFMM_INSTANTIATE(3)
}  // namespace gbfmm
