// Arithmetic types of the pair kernels (M2L and P2P) and their storage.
//
//   T = double : binary64 throughout (FMM_FP64)
//   T = df64   : double-float on the FP32 units, binary64-accurate (FMM_DF64)
//   T = float  : binary32 pair arithmetic with binary64 translations and accumulators
//                (FMM_MIXED)
//
// Positions and cell centres are stored as binary64 in FMM_FP64 and as double-float
// otherwise ("storage type" S).  Differences X_a - X_b are formed from the S operands to
// the accuracy of T (sep), so binary32 pair kernels still see separations accurate to
// their own rounding.  The pair kernel's per-(leaf pair, particle) partials are stored in
// T; the per-item sums over them are kept in G (binary64 for binary64, double-float
// otherwise, so that no binary64 conversion sits in the binary32 kernels) and reduced in a
// fixed order; the per-particle totals are binary64.
#pragma once
#include <cuda_runtime.h>

#include "df64.cuh"

namespace gbfmm {

// fin(v): a finished value of type T (double-float normalised) for storage
template <class T>
struct Prec;

template <>
struct Prec<double> {
    using S = double;  // storage of positions, masses and centres
    using G = double;  // item-level partial sums
    __device__ static double sep(double a, double b) { return a - b; }
    __device__ static double fin(double v) { return v; }
    __device__ static double mass(double m) { return m; }
};

template <>
struct Prec<df64> {
    using S = df64;
    using G = df64;
    __device__ static df64 sep(df64 a, df64 b) { return a - b; }
    __device__ static df64 fin(df64 v) { return norm(v); }
    __device__ static df64 mass(df64 m) { return m; }
};

template <>
struct Prec<float> {
    using S = df64;
    using G = df64;  // item-level sums of the binary32 pair partials kept as double-float
    // a - b rounded to binary32 from double-float operands: (a.hi - b.hi) + (a.lo - b.lo).
    // When a and b are close the high-word difference is exact (Sterbenz); otherwise its
    // rounding is within binary32's own 2^-24 of the result.
    __device__ static float sep(df64 a, df64 b) { return __fadd_rn(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo)); }
    __device__ static float fin(float v) { return v; }
    __device__ static float mass(df64 m) { return m.hi; }  // hi is m rounded to binary32
};

__device__ __forceinline__ double to_storage(double v, double) { return v; }
__device__ __forceinline__ df64 to_storage(double v, df64) { return to_df(v); }
__device__ __forceinline__ float to_kernel(double v, float) { return (float)v; }
__device__ __forceinline__ double to_kernel(double v, double) { return v; }
__device__ __forceinline__ df64 to_kernel(double v, df64) { return to_df(v); }

__device__ __forceinline__ bool is_zero(double v) { return v == 0.0; }
__device__ __forceinline__ bool is_zero(float v) { return v == 0.f; }
__device__ __forceinline__ bool is_zero(df64 v) { return v.hi == 0.f; }

// four partial sums (a_x, a_y, a_z, phi)
template <class G>
struct Quad {
    G x, y, z, w;
};

}  // namespace gbfmm
