// Arithmetic helpers shared by the generated expansion operators.
#pragma once
#include <cuda_runtime.h>

namespace gbfmm {

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
// multiplication by a power of two f (exact unless the result leaves the format's range)
__device__ __forceinline__ double scale_t(double a, float f) { return a * (double)f; }
__device__ __forceinline__ float scale_t(float a, float f) { return a * f; }
// a * f * c for a power of two f and a small integer c (f c is exact)
__device__ __forceinline__ double scale_c_t(double a, float f, float c) { return a * ((double)f * (double)c); }
__device__ __forceinline__ float scale_c_t(float a, float f, float c) { return a * (f * c); }

// Expansion operators of order P; specialisations are generated (gen/exp_p{P}.cuh).
template <int P>
struct Exp;

}  // namespace gbfmm
