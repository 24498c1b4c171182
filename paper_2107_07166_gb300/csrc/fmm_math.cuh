// Arithmetic helpers shared by the generated expansion operators.
#pragma once
#include <cuda_runtime.h>

namespace gbfmm {

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }

// Expansion operators of order P; specialisations are generated (gen/exp_p{P}.cuh).
template <int P>
struct Exp;

}  // namespace gbfmm
