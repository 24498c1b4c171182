// Arithmetic types of the pair kernels (M2L and P2P) and their storage.
//
//   T = double : binary64 throughout (FMM_FP64)
//   T = df64   : double-float on the FP32 units, binary64-accurate (FMM_DF64)
//   T = float  : binary32 pair arithmetic with binary64 translations and accumulators
//                (FMM_MIXED)
//
// Positions and cell centres are stored as binary64 in FMM_FP64 and as double-float
// otherwise ("storage type" S).  Differences X_a - X_b and Z_A - Z_B are formed in S and
// only then narrowed to T, so binary32 pair kernels still see separations accurate to
// their own rounding.  Per-pair and per-chunk partial sums are kept in G (binary64 for
// binary64, double-float otherwise, so that no binary64 conversion sits in the binary32
// pair kernels) and reduced in a fixed order; the per-particle totals are binary64.
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
    using G = double;  // partial sums
    __device__ static double fin(double v) { return v; }
    __device__ static double narrow(double v) { return v; }
    __device__ static double mass(double m) { return m; }
    __device__ static double to_g(double v) { return v; }
    __device__ static double g_to_double(double v) { return v; }
    __device__ static double g_add(double a, double b) { return a + b; }
};

template <>
struct Prec<df64> {
    using S = df64;
    using G = df64;
    __device__ static df64 fin(df64 v) { return norm(v); }
    __device__ static df64 narrow(df64 v) { return v; }
    __device__ static df64 mass(df64 m) { return m; }
    __device__ static df64 to_g(df64 v) { return norm(v); }
    __device__ static double g_to_double(df64 v) { return to_double(v); }
    __device__ static df64 g_add(df64 a, df64 b) { return a + b; }
};

template <>
struct Prec<float> {
    using S = df64;
    using G = df64;  // per-pair partials kept as double-float: no binary64 converts in the pair kernel
    __device__ static float fin(float v) { return v; }
    __device__ static float narrow(df64 v) { return __fadd_rn(v.hi, v.lo); }
    __device__ static float mass(df64 m) { return __fadd_rn(m.hi, m.lo); }
    __device__ static df64 to_g(float v) { return df64(v, 0.f); }
    __device__ static double g_to_double(df64 v) { return to_double(v); }
    __device__ static df64 g_add(df64 a, df64 b) { return a + b; }
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
