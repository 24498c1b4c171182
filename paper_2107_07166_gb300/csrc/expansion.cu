// Dispatch of the expansion stages to the order-specialised kernels (expansion_p*.cu).
#include "fmm_internal.h"

namespace gbfmm {

template <int P>
void run_moments_p(fmm_ctx* c);
template <int P>
void run_far_field_p(fmm_ctx* c, int variant, bool want_pot);
template <int P>
void run_finish_p(fmm_ctx* c, int variant, bool want_pot, double* acc, double* pot);

#define GB_DISPATCH(p, call)                                            \
    switch (p) {                                                        \
        case 1: call(1); break;                                         \
        case 2: call(2); break;                                         \
        case 3: call(3); break;                                         \
        case 4: call(4); break;                                         \
        case 5: call(5); break;                                         \
        case 6: call(6); break;                                         \
        case 7: call(7); break;                                         \
        case 8: call(8); break;                                         \
        default: throw FmmError{FMM_ERR_INVALID, "order p out of range"}; \
    }

void run_moments_dispatch(fmm_ctx* c, int p) {
#define CALL(P) run_moments_p<P>(c)
    GB_DISPATCH(p, CALL)
#undef CALL
}

void run_far_field_dispatch(fmm_ctx* c, int p, int variant, bool want_pot) {
#define CALL(P) run_far_field_p<P>(c, variant, want_pot)
    GB_DISPATCH(p, CALL)
#undef CALL
}

void run_finish_dispatch(fmm_ctx* c, int p, int variant, bool want_pot, double* acc, double* pot) {
#define CALL(P) run_finish_p<P>(c, variant, want_pot, acc, pot)
    GB_DISPATCH(p, CALL)
#undef CALL
}

}  // namespace gbfmm
