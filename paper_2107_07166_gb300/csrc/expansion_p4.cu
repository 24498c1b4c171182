// Expansion kernels instantiated for order p = 4.
#include "gen/exp_p4.cuh"
#include "expansion_impl.cuh"

namespace gbfmm {
GBFMM_INSTANTIATE(4)
}  // namespace gbfmm
