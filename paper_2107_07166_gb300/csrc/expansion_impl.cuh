// Expansion kernels of order P (included once per P by the generated expansion_p*.cu):
// P2M, M2M (upward pass), target-major M2L, L2L (downward pass) and the final
// per-particle kernel (L2P + P2P partial reduction + return to input order).
//
// Layouts (device, node ids breadth-first):
//   mom[n * NM + k]     raw moments M_alpha about Z_n, alpha in generated order
//   loc[n * NM + k]     standard locals L_gamma                       (variant 0)
//   loc[n * NSU + k]    conserving locals [S | Ux | Uy | Uz]          (variants 1 and 2)
//   m2l_dir[e]          source id of entry e; m2l_seg[n] = first entry of target n (sources increase)
//
// Range scaling of the binary32 and double-float M2L (their exponent range is binary32's).
// A tensor of order n at separation R grows like R^-(n+1) (R^-(n+3) for the conserving
// kernel), which leaves the binary32 range for close, small cells (R ~ 1e-5 at p = 6),
// and the moments of small cells underflow.  These modes therefore work in powers of two:
//   * node n stores its moments in units of s_n = 2^k_n, k_n = floor(log2 r_max,n):
//     Mt_beta = M_beta s_n^-|beta| (exact power-of-two scaling in binary64, then narrowed);
//   * an M2L item (one target, up to M2L_CHUNK sources) works in units of
//     s_I = 2^k_I <= its nearest source separation;
//   * each entry takes its tensor at R' = R / 2^k_e with k_e = floor(log2 |R|_inf), so
//     |R'|_inf is in [1, 2) and no monomial of the tensor leaves the range, and moves it to
//     item units by homogeneity, T_alpha(R / s_I) = v^(|alpha|+1) T_alpha(R') (v^(|alpha|+3)
//     for the conserving kernel), v = 2^(k_I - k_e) <= 1;
//   * a source's moments are multiplied on load by (s_n / s_I)^|beta| (saturated at 2^100:
//     a source that far beyond the item's nearest one contributes below binary32 resolution);
//   * the item's partial locals carry s_I^(|gamma|+1) (standard), s_I^(|gamma|+3) (S) or
//     s_I^(|gamma|+2) (U); the binary64 reduction removes the factor exactly.
// Every factor is a power of two, so the scaling itself adds no rounding.  binary64 (FMM_FP64)
// is unscaled.  The binary32 separation is formed from double-float centres (two binary32
// words per coordinate) with an error-free subtraction, so no binary64 arithmetic sits in the
// binary32 kernel.
#pragma once
#include <type_traits>

#include "fmm_device.cuh"
#include "fmm_internal.h"
#include "fmm_math.cuh"
#include "fused_traverse.cuh"
#include "prec.cuh"

namespace gbfmm {

constexpr int EB = 128;

// a5 P2M: moments of every leaf from its particles (y = X - Z), one thread per leaf, leaves
// taken in order of size so that a warp's lanes finish together.  (A warp
// per leaf with a butterfly reduction was 4x slower: every lane then runs the reduction's
// binary64 adds, and binary64 warp instructions cost the same with idle lanes.)
template <int P>
__global__ void __launch_bounds__(EB) p2m_k(int nn, const uint32_t* __restrict__ order,
                                            const int* __restrict__ nfirst, const int* __restrict__ ncount,
                                            const int* __restrict__ nnchild, const double* __restrict__ xs,
                                            const double* __restrict__ ys, const double* __restrict__ zs,
                                            const double* __restrict__ ms, const double* __restrict__ Zx,
                                            const double* __restrict__ Zy, const double* __restrict__ Zz,
                                            double* __restrict__ mom) {
    using E = Exp<P>;
    int t = blockIdx.x * EB + threadIdx.x;
    if (t >= nn) return;
    int nd = (int)order[t];  // nodes by leaf size: a warp's leaves hold equal counts
    if (nnchild[nd] != 0) return;
    double M[E::NM];
#pragma unroll
    for (int k = 0; k < E::NM; k++) M[k] = 0.0;
    double zx = Zx[nd], zy = Zy[nd], zz = Zz[nd];
    int f = nfirst[nd], e = f + ncount[nd];
    for (int i = f; i < e; i++) E::p2m(ms[i], xs[i] - zx, ys[i] - zy, zs[i] - zz, M);
#pragma unroll
    for (int k = 0; k < E::NM; k++) mom[(int64_t)nd * E::NM + k] = M[k];
}

// ---- range scaling helpers (binary32 and double-float kernels)

// floor(log2(max(|x|, |y|, |z|))) from the binary32 exponent, clamped to [-100, 100]
__device__ __forceinline__ int sep_exp(float x, float y, float z) {
    float m = fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z)));
    int e = (int)((__float_as_uint(m) >> 23) & 0xffu) - 127;
    return min(100, max(-100, e));
}

// 2^e as binary32, e in [-126, 127]
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((unsigned)(e + 127) << 23); }

// Z_a - Z_b from double-float centres, rounded to binary32: (ah - bh) + (al - bl).  When
// the centres are close (the case that cancels), ah - bh is exact by Sterbenz's lemma;
// otherwise its rounding is within binary32's own 2^-24 of |Z_a - Z_b|
__device__ __forceinline__ float dsep(float ah, float al, float bh, float bl) {
    return __fadd_rn(__fsub_rn(ah, bh), __fsub_rn(al, bl));
}

// The double-float centre words hold a centre to about 2^-48 |Z| (the rounding of the low
// word), so (hi - hi) + (lo - lo) carries an absolute error of up to ~2^-47 |Z|.  Below
// |R|_inf = 2^-20 max(|Z_a|, |Z_b|) that is more than 2^-27 of R, and R is formed again
// from the binary64 centres (rounded once to binary32).  Only cells that nearly coincide
// take this branch.
// (al.w and bl.w hold max_i |hi(Z_i)| of the two centres.)  The binary64 path is a call
// that is not inlined, so that its loads are not hoisted into every entry.
static __device__ __noinline__ float3 close_sep_slow(const double* __restrict__ Zx, const double* __restrict__ Zy,
                                              const double* __restrict__ Zz, int t, int s) {
    return make_float3((float)(Zx[t] - Zx[s]), (float)(Zy[t] - Zy[s]), (float)(Zz[t] - Zz[s]));
}
__device__ __forceinline__ void close_sep_fix(float4 al, float4 bl, const double* __restrict__ Zx,
                                              const double* __restrict__ Zy, const double* __restrict__ Zz, int t,
                                              int s, float& rx, float& ry, float& rz) {
    float r = fmaxf(fabsf(rx), fmaxf(fabsf(ry), fabsf(rz)));
    if (r < 0x1p-20f * fmaxf(al.w, bl.w)) {
        float3 v = close_sep_slow(Zx, Zy, Zz, t, s);
        rx = v.x;
        ry = v.y;
        rz = v.z;
    }
}

// 2^e as binary64 for |e| <= 1022
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

// the item unit exponent: min over the item's sources of floor(log2 |R|_inf), with R formed
// as the M2L kernels form it (close_sep_fix included)
__device__ __forceinline__ int item_exp(int tgt, int e0, int e1, const uint32_t* __restrict__ dir,
                                        const float4* __restrict__ zh, const float4* __restrict__ zl,
                                        const double* __restrict__ Zx, const double* __restrict__ Zy,
                                        const double* __restrict__ Zz) {
    float4 ah = zh[tgt], al = zl[tgt];
    int k = 100;
    // four entries per round with all loads first: the id -> centre chains overlap (an index
    // past the end repeats the last entry, which leaves the minimum unchanged)
    for (int e = e0; e < e1; e += 4) {
        int s[4];
#pragma unroll
        for (int j = 0; j < 4; j++) s[j] = (int)dir[min(e + j, e1 - 1)];
        float4 bh[4], bl[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            bh[j] = zh[s[j]];
            bl[j] = zl[s[j]];
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            float rx = dsep(ah.x, al.x, bh[j].x, bl[j].x), ry = dsep(ah.y, al.y, bh[j].y, bl[j].y);
            float rz = dsep(ah.z, al.z, bh[j].z, bl[j].z);
            close_sep_fix(al, bl[j], Zx, Zy, Zz, tgt, s[j], rx, ry, rz);
            k = min(k, sep_exp(rx, ry, rz));
        }
    }
    return k;
}

// degree of multi-index number j in the generated order (by degree)
__host__ __device__ constexpr int mi_deg(int j) {
    int n = 0;
    while (j >= (n + 1) * (n + 2) * (n + 3) / 6) n++;
    return n;
}

// v^n for n < NF (v a power of two <= 1; underflow to zero is harmless here)
template <int NF>
__device__ __forceinline__ void pow_table(float v, float* w) {
    w[0] = 1.f;
#pragma unroll
    for (int n = 1; n < NF; n++) w[n] = w[n - 1] * v;
}

// f[n] = 2^(e n), n < NF, saturated at 2^100
template <int NF>
__device__ __forceinline__ void moment_factors(int e, float* f) {
    float t = pow2f(min(100, max(-126, e)));
    f[0] = 1.f;
#pragma unroll
    for (int n = 1; n < NF; n++) f[n] = fminf(f[n - 1] * t, 0x1p100f);
}

// R = Z_tgt - Z_src in the kernel type: binary64 from the binary64 centres; double-float
// from the binary64 difference; binary32 from the double-float centres
template <class T>
struct SepOf;
template <>
struct SepOf<double> {
    __device__ static void get(const double* Zx, const double* Zy, const double* Zz, const float4*, const float4*,
                               int tgt, int src, double& rx, double& ry, double& rz) {
        rx = Zx[tgt] - Zx[src];
        ry = Zy[tgt] - Zy[src];
        rz = Zz[tgt] - Zz[src];
    }
    __device__ static float approx(double v) { return (float)v; }
};
template <>
struct SepOf<df64> {
    __device__ static void get(const double* Zx, const double* Zy, const double* Zz, const float4*, const float4*,
                               int tgt, int src, df64& rx, df64& ry, df64& rz) {
        rx = to_df(Zx[tgt] - Zx[src]);
        ry = to_df(Zy[tgt] - Zy[src]);
        rz = to_df(Zz[tgt] - Zz[src]);
    }
    __device__ static float approx(df64 v) { return v.hi; }
};
template <>
struct SepOf<float> {
    __device__ static void get(const double* Zx, const double* Zy, const double* Zz, const float4* zh,
                               const float4* zl, int tgt, int src, float& rx, float& ry, float& rz) {
        float4 ah = zh[tgt], al = zl[tgt], bh = zh[src], bl = zl[src];
        rx = dsep(ah.x, al.x, bh.x, bl.x);
        ry = dsep(ah.y, al.y, bh.y, bl.y);
        rz = dsep(ah.z, al.z, bh.z, bl.z);
        close_sep_fix(al, bl, Zx, Zy, Zz, tgt, src, rx, ry, rz);
    }
    __device__ static float approx(float v) { return v; }
};

// one M2L entry's geometry in the scaled modes: R' = R 2^-k_e (|R'|_inf in [1, 2)), the
// item-unit separation R'' = R' 2^(k_e - k_I), v = 2^(k_I - k_e); returns k_e
template <class T>
__device__ __forceinline__ int entry_units(T& rx, T& ry, T& rz, int kI, T& ux, T& uy, T& uz, float& v) {
    int ke = sep_exp(SepOf<T>::approx(rx), SepOf<T>::approx(ry), SepOf<T>::approx(rz));
    float se = pow2f(-ke);
    rx = scale_t(rx, se);
    ry = scale_t(ry, se);
    rz = scale_t(rz, se);
    int d = ke - kI;  // >= 0 by the choice of k_I
    v = pow2f(-min(d, 126));
    float up = pow2f(min(d, 100));
    ux = scale_t(rx, up);
    uy = scale_t(ry, up);
    uz = scale_t(rz, up);
    return ke;
}

// N (a multiple of 8) binary32 values of a 32-byte aligned row in 32-byte loads: one
// load per thread then fills whole 32-byte sectors (a 16-byte load per thread, to rows of
// different threads, moves twice the sectors it uses); the rows are read-only in the
// kernels that read them
template <int N>
__device__ __forceinline__ void load_f8(const float* __restrict__ src, float* dst) {
    static_assert(N % 8 == 0, "load_f8: rows of whole 32-byte sectors");
#pragma unroll
    for (int k = 0; k < N / 8; k++)
        asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=f"(dst[8 * k]), "=f"(dst[8 * k + 1]), "=f"(dst[8 * k + 2]), "=f"(dst[8 * k + 3]),
                       "=f"(dst[8 * k + 4]), "=f"(dst[8 * k + 5]), "=f"(dst[8 * k + 6]), "=f"(dst[8 * k + 7])
                     : "l"(src + 8 * k));
}

// geometry of the M2L kernels
// a5 in the double-float and binary32 modes: y = X - Z in binary64, in units of the leaf
// 2^k (k = floor(log2 r_max), so |y| 2^-k < 2 and no monomial leaves binary32's range), then
// the monomials and their sums in double-float (about 2^-44 relative) on the binary32
// units; moment alpha is stored in binary64 times 2^(k |alpha|) (exact) for the binary64
// M2M.  Leaves in order of size, as above.
template <int P>
__global__ void __launch_bounds__(EB) p2m_df_k(int nn, const uint32_t* __restrict__ order,
                                               const int* __restrict__ nfirst, const int* __restrict__ ncount,
                                               const int* __restrict__ nnchild, const double* __restrict__ rmax,
                                               const double* __restrict__ xs,
                                               const double* __restrict__ ys, const double* __restrict__ zs,
                                               const double* __restrict__ ms, const double* __restrict__ Zx,
                                               const double* __restrict__ Zy, const double* __restrict__ Zz,
                                               double* __restrict__ mom) {
    using E = Exp<P>;
    int t = blockIdx.x * EB + threadIdx.x;
    if (t >= nn) return;
    int nd = (int)order[t];
    if (nnchild[nd] != 0) return;
    df64 M[E::NM];
#pragma unroll
    for (int k = 0; k < E::NM; k++) M[k] = df64();
    double r = rmax[nd];
    int kn = r > 0.0 ? max(-120, min(120, ilogb(r))) : 0;
    double sc = pow2d(-kn);
    double zx = Zx[nd], zy = Zy[nd], zz = Zz[nd];
    int f = nfirst[nd], e = f + ncount[nd];
    for (int i = f; i < e; i++)
        E::p2m(to_df(ms[i]), to_df((xs[i] - zx) * sc), to_df((ys[i] - zy) * sc), to_df((zs[i] - zz) * sc), M);
#pragma unroll
    for (int k = 0; k < E::NM; k++) mom[(int64_t)nd * E::NM + k] = to_double(M[k]) * pow2d(kn * mi_deg(k));
}

struct M2LGeom {
    const double *Zx, *Zy, *Zz;  // binary64 centres
    const float4 *zh, *zl;       // double-float centres (scaled modes)
    const int* nk;               // per-node moment unit exponent (scaled modes)
};

// An M2L entry's source geometry (centre, and moment unit in the scaled modes), fetched one
// entry ahead of its use so that the id -> centre load chain of the next entry overlaps
// this entry's arithmetic; the target's is loaded once per item.
template <class T>
struct SrcGeo {  // binary64 and double-float: binary64 centres
    double x, y, z;
    int nk;
    __device__ void load(const M2LGeom& g, int s) {
        x = g.Zx[s];
        y = g.Zy[s];
        z = g.Zz[s];
        nk = std::is_same<T, double>::value ? 0 : g.nk[s];
    }
};
template <>
struct SrcGeo<float> {
    float4 h, l;
    int nk;
    __device__ void load(const M2LGeom& g, int s) {
        h = g.zh[s];
        l = g.zl[s];
        nk = g.nk[s];
    }
};
template <class T>
struct TgtGeo {
    double x, y, z;
    __device__ void load(const M2LGeom& g, int t) {
        x = g.Zx[t];
        y = g.Zy[t];
        z = g.Zz[t];
    }
    // R = Z_tgt - Z_src, formed in binary64 and rounded to T
    __device__ void sep(const SrcGeo<T>& s, T& rx, T& ry, T& rz, const M2LGeom&, int, int) const {
        rx = to_kernel(x - s.x, T());
        ry = to_kernel(y - s.y, T());
        rz = to_kernel(z - s.z, T());
    }
};
template <>
struct TgtGeo<float> {
    float4 h, l;
    __device__ void load(const M2LGeom& g, int t) {
        h = g.zh[t];
        l = g.zl[t];
    }
    // R from the double-float centre words: (hi - hi) + (lo - lo), or from the binary64
    // centres for nearly coincident cells (close_sep_fix)
    __device__ void sep(const SrcGeo<float>& s, float& rx, float& ry, float& rz, const M2LGeom& g, int t,
                        int src) const {
        rx = dsep(h.x, l.x, s.h.x, s.l.x);
        ry = dsep(h.y, l.y, s.h.y, s.l.y);
        rz = dsep(h.z, l.z, s.h.z, s.l.z);
        close_sep_fix(l, s.l, g.Zx, g.Zy, g.Zz, t, src, rx, ry, rz);
    }
};

// a8 M2L, standard, one work item = up to M2L_CHUNK directed entries of one target cell
// (sources in list order): L_gamma += sum_beta M_beta D_{beta+gamma}(Z_tgt - Z_src),
// in the pair-kernel type T.  The item's partial local goes to part[item] (and its unit
// exponent to kpart[item] in the scaled modes); m2l_reduce_k sums a cell's items in order.
template <int P, class T>
__global__ void __launch_bounds__(EB) m2l_std_k(int64_t nitems, const int4* __restrict__ items,
                                                const uint32_t* __restrict__ dir, M2LGeom g,
                                                const T* __restrict__ mom, T* __restrict__ part,
                                                int* __restrict__ kpart) {
    using E = Exp<P>;
    constexpr bool SC = !std::is_same<T, double>::value;
    int64_t it = (int64_t)blockIdx.x * EB + threadIdx.x;
    if (it >= nitems) return;
    int4 w = items[it];
    T L[E::NM];
#pragma unroll
    for (int k = 0; k < E::NM; k++) L[k] = T(0);
    int kI = 0;
    if constexpr (SC) {
        kI = item_exp(w.x, w.y, w.z, dir, g.zh, g.zl, g.Zx, g.Zy, g.Zz);
        kpart[it] = kI;
    }
    TgtGeo<T> tg;
    tg.load(g, w.x);
    int src = (int)dir[w.y];  // an item holds at least one entry
    SrcGeo<T> sg;
    sg.load(g, src);
    for (int e = w.y; e < w.z; e++) {
        int nsrc = e + 1 < w.z ? (int)dir[e + 1] : src;
        T rx, ry, rz;
        tg.sep(sg, rx, ry, rz, g, w.x, src);
        T D[E::NM];
        if constexpr (SC) {
            T ux, uy, uz;
            float v;
            entry_units(rx, ry, rz, kI, ux, uy, uz, v);
            E::dtensor(rx, ry, rz, D);
            float vp[P + 2];
            pow_table<P + 2>(v, vp);
#pragma unroll
            for (int k = 0; k < E::NM; k++) D[k] = scale_t(D[k], vp[mi_deg(k) + 1]);
            float f[P + 1];
            moment_factors<P + 1>(sg.nk - kI, f);
            if constexpr (sizeof(T) == 4) {
                T Ms[E::NMP];
                load_f8<E::NMP>(mom + (int64_t)src * E::NMP, Ms);
                E::m2l_std_s(Ms, f, D, L);
            } else {
                E::m2l_std_s(mom + (int64_t)src * E::NMP, f, D, L);
            }
        } else {
            E::dtensor(rx, ry, rz, D);
            E::m2l_std(mom + (int64_t)src * E::NM, D, L);
        }
        src = nsrc;
        sg.load(g, src);
    }
#pragma unroll
    for (int k = 0; k < E::NM; k++) part[it * E::NM + k] = Prec<T>::fin(L[k]);
}

// a8' M2L, conserving: S and U of the realigned pair forces; binary64 reads the conserving
// moments of con_moments_k, the scaled modes read the raw moments (padded, range-scaled)
// and form the conserving ones on load
template <int P, class T>
__global__ void __launch_bounds__(EB) m2l_con_k(int64_t nitems, const int4* __restrict__ items,
                                                const uint32_t* __restrict__ dir, M2LGeom g,
                                                const T* __restrict__ cmom, T* __restrict__ part,
                                                int* __restrict__ kpart) {
    using E = Exp<P>;
    constexpr bool SC = !std::is_same<T, double>::value;
    int64_t it = (int64_t)blockIdx.x * EB + threadIdx.x;
    if (it >= nitems) return;
    int4 w = items[it];
    T SU[E::NSU];
#pragma unroll
    for (int k = 0; k < E::NSU; k++) SU[k] = T(0);
    int kI = 0;
    if constexpr (SC) {
        kI = item_exp(w.x, w.y, w.z, dir, g.zh, g.zl, g.Zx, g.Zy, g.Zz);
        kpart[it] = kI;
    }
    TgtGeo<T> tg;
    tg.load(g, w.x);
    int src = (int)dir[w.y];  // an item holds at least one entry
    SrcGeo<T> sg;
    sg.load(g, src);
    for (int e = w.y; e < w.z; e++) {
        int nsrc = e + 1 < w.z ? (int)dir[e + 1] : src;
        T rx, ry, rz;
        tg.sep(sg, rx, ry, rz, g, w.x, src);
        T H[E::NQ];
        if constexpr (SC) {
            T ux, uy, uz;
            float v;
            entry_units(rx, ry, rz, kI, ux, uy, uz, v);
            E::htensor(rx, ry, rz, H);
            float vp[P + 3];
            pow_table<P + 3>(v, vp);
#pragma unroll
            for (int k = 0; k < E::NQ; k++) H[k] = scale_t(H[k], vp[mi_deg(k) + 3]);
            rx = ux;
            ry = uy;
            rz = uz;
        } else {
            E::htensor(rx, ry, rz, H);
        }
        if constexpr (sizeof(T) == 4) {
            // binary32: the raw moments (padded to a multiple of 8 floats) in 32-byte loads;
            // the conserving moments are formed from them on load
            T Ms[E::NMP];
            load_f8<E::NMP>(cmom + (int64_t)src * E::NMP, Ms);
            float f[P + 1];
            moment_factors<P + 1>(sg.nk - kI, f);
            E::m2l_con_m(Ms, f, H, rx, ry, rz, SU);
        } else if constexpr (SC) {
            float f[P + 1];
            moment_factors<P + 1>(sg.nk - kI, f);
            E::m2l_con_m(cmom + (int64_t)src * E::NMP, f, H, rx, ry, rz, SU);
        } else {
            E::m2l_con(cmom + (int64_t)src * E::NSU, H, rx, ry, rz, SU);
        }
        src = nsrc;
        sg.load(g, src);
    }
#pragma unroll
    for (int k = 0; k < E::NSU; k++) part[it * E::NSU + k] = Prec<T>::fin(SU[k]);
}

// row stride of the stored pair tensors: NT doubles padded to whole 32-byte sectors
__host__ __device__ constexpr int pair_tensor_stride(int nt) { return (nt + 3) / 4 * 4; }

// Binary64 M2L with shared pair tensors.  The tensor of R = Z_A - Z_B (D for the standard
// form, h for the conserving one) is formed once per mutual pair; the entry of cell A
// (side 0) uses it as it is, the entry of cell B (side 1) sees R' = -R, whose tensor is the
// same with the odd degrees negated.  That is exact: every term of a component of degree n
// carries n factors of R, and binary64 rounding is symmetric, so the result is the one
// the per-entry tensor gives.  It halves the tensor work of the binary64-bound M2L; the
// tensors come from memory, whose latency the binary64 pipe hides.
template <int P, int V>
__global__ void __launch_bounds__(EB) m2l_ptensor_k(int64_t npairs, const int2* __restrict__ pairs,
                                                    const double* __restrict__ Zx, const double* __restrict__ Zy,
                                                    const double* __restrict__ Zz, double* __restrict__ T) {
    using E = Exp<P>;
    constexpr int NT = V == 0 ? E::NM : E::NQ, NTP = pair_tensor_stride(NT);
    int64_t k = (int64_t)blockIdx.x * EB + threadIdx.x;
    if (k >= npairs) return;
    int2 pr = pairs[k];
    double rx = Zx[pr.x] - Zx[pr.y], ry = Zy[pr.x] - Zy[pr.y], rz = Zz[pr.x] - Zz[pr.y];
    double H[NTP];
    if constexpr (V == 0)
        E::dtensor(rx, ry, rz, H);
    else
        E::htensor(rx, ry, rz, H);
#pragma unroll
    for (int j = NT; j < NTP; j++) H[j] = 0.0;
    // whole 32-byte sectors per store: one row per thread, rows 32-byte aligned
    double* Tk = T + k * NTP;
#pragma unroll
    for (int j = 0; j < NTP; j += 4)
        asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(Tk + j), "d"(H[j]), "d"(H[j + 1]),
                     "d"(H[j + 2]), "d"(H[j + 3])
                     : "memory");
}

// the pair tensor of entry v = pair << 1 | side, as seen from the entry's target, read in
// 32-byte loads from its padded row (the tensors are read-only in the M2L kernels)
template <int NT>
__device__ __forceinline__ void load_pair_tensor(const double* __restrict__ T, uint32_t v, double* __restrict__ H) {
    constexpr int NTP = pair_tensor_stride(NT);
    const double* Tp = T + (int64_t)(v >> 1) * NTP;
    double R[NTP];
#pragma unroll
    for (int j = 0; j < NTP; j += 4)
        asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];"
            : "=d"(R[j]), "=d"(R[j + 1]), "=d"(R[j + 2]), "=d"(R[j + 3])
            : "l"(Tp + j));
    unsigned long long flip = (v & 1u) ? 0x8000000000000000ull : 0ull;
#pragma unroll
    for (int j = 0; j < NT; j++) {
        unsigned long long b = (unsigned long long)__double_as_longlong(R[j]);
        if (mi_deg(j) & 1) b ^= flip;
        H[j] = __longlong_as_double((long long)b);
    }
}

template <int P>
__global__ void __launch_bounds__(EB) m2l_std_t_k(int64_t nitems, const int4* __restrict__ items,
                                                  const uint32_t* __restrict__ dir, const uint32_t* __restrict__ dirp,
                                                  const double* __restrict__ T, const double* __restrict__ mom,
                                                  double* __restrict__ part) {
    using E = Exp<P>;
    int64_t it = (int64_t)blockIdx.x * EB + threadIdx.x;
    if (it >= nitems) return;
    int4 w = items[it];
    double L[E::NM];
#pragma unroll
    for (int k = 0; k < E::NM; k++) L[k] = 0.0;
    for (int e = w.y; e < w.z; e++) {
        int src = (int)dir[e];
        double D[E::NM];
        load_pair_tensor<E::NM>(T, dirp[e], D);
        E::m2l_std(mom + (int64_t)src * E::NM, D, L);
    }
#pragma unroll
    for (int k = 0; k < E::NM; k++) part[it * E::NM + k] = L[k];
}

// conserving, on the root-relative source moments of con_moments_k: 4 nmi(p-1)-term
// contractions per entry and no per-pair geometry (con_origin_k adds the target term)
template <int P>
__global__ void __launch_bounds__(EB) m2l_con_t_k(int64_t nitems, const int4* __restrict__ items,
                                                  const uint32_t* __restrict__ dir, const uint32_t* __restrict__ dirp,
                                                  const double* __restrict__ T, const double* __restrict__ cmom,
                                                  double* __restrict__ part) {
    using E = Exp<P>;
    int64_t it = (int64_t)blockIdx.x * EB + threadIdx.x;
    if (it >= nitems) return;
    int4 w = items[it];
    double SU[E::NSU];
#pragma unroll
    for (int k = 0; k < E::NSU; k++) SU[k] = 0.0;
    for (int e = w.y; e < w.z; e++) {
        int src = (int)dir[e];
        double H[E::NQ];
        load_pair_tensor<E::NQ>(T, dirp[e], H);
        E::m2l_con_o(cmom + (int64_t)src * E::NSU, H, SU);
    }
#pragma unroll
    for (int k = 0; k < E::NSU; k++) part[it * E::NSU + k] = SU[k];
}

// a8'' M2L, literal order-0 realigned form (eq. aaB0), run at expansion order 2: from the
// raw moments of the source (M = M_0, Qbar_ii = 2 M_{2e_i}, Qbar_ij = M_{e_i+e_j}) the
// degree-1 conserving locals of
//   a(x) = -(M/R^2) [n + x/R - (n.x) n/R - (n.x) x/R^2] + Qbar n / R^4 = x S(x) + U(x):
//   S_0 = -M/R^3, S_{e_j} = M n_j/R^4, U_{i,0} = -M n_i/R^2 + (Qbar n)_i/R^4,
//   U_{i,e_j} = M n_i n_j/R^3.
// Moment order (10 entries): 1 | x y z | xx xy xz yy yz zz; locals [S | Ux | Uy | Uz], 4 each.
template <class T>
__global__ void __launch_bounds__(EB) m2l_p0_k(int64_t nitems, const int4* __restrict__ items,
                                               const uint32_t* __restrict__ dir, M2LGeom g,
                                               const T* __restrict__ mom, T* __restrict__ part,
                                               int* __restrict__ kpart) {
    constexpr bool SC = !std::is_same<T, double>::value;
    constexpr int NM = SC ? 16 : 10, NQ = 4, NSU = 16;  // moment stride (Exp<2>::NMP, ::NM): padded in the scaled modes
    int64_t it = (int64_t)blockIdx.x * EB + threadIdx.x;
    if (it >= nitems) return;
    int4 w = items[it];
    T SU[NSU];
#pragma unroll
    for (int k = 0; k < NSU; k++) SU[k] = T(0);
    int kI = 0;
    if constexpr (SC) {
        kI = item_exp(w.x, w.y, w.z, dir, g.zh, g.zl, g.Zx, g.Zy, g.Zz);
        kpart[it] = kI;
    }
    for (int e = w.y; e < w.z; e++) {
        int src = (int)dir[e];
        T r[3];
        SepOf<T>::get(g.Zx, g.Zy, g.Zz, g.zh, g.zl, w.x, src, r[0], r[1], r[2]);
        // scaled modes: the terms are formed in entry units (|R'| ~ 1) and moved to item
        // units by v^(length power): S_0 ~ R^-3, S_ej ~ R^-4, U_i0 ~ R^-2, U_iej ~ R^-3
        float w2 = 1.f, w3 = 1.f, w4 = 1.f, f2 = 1.f;
        if constexpr (SC) {
            T ux, uy, uz;
            float v;
            int ke = entry_units(r[0], r[1], r[2], kI, ux, uy, uz, v);
            w2 = v * v;
            w3 = w2 * v;
            w4 = w2 * w2;
            float f[3];
            moment_factors<3>(g.nk[src] - ke, f);  // Qbar in entry units
            f2 = f[2];
        }
        T ir = rsqrt_t(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        T n[3] = {r[0] * ir, r[1] * ir, r[2] * ir};
        const T* Ms = mom + (int64_t)src * NM;
        T M = Ms[0];
        T q[6];
#pragma unroll
        for (int k = 0; k < 6; k++) q[k] = scale_t(Ms[4 + k], f2);
        T two = T(2);
        T Q[3][3] = {{two * q[0], q[1], q[2]}, {q[1], two * q[3], q[4]}, {q[2], q[4], two * q[5]}};
        T ir2 = ir * ir;
        T mi3 = M * (ir2 * ir), mi4 = M * (ir2 * ir2), ir4 = ir2 * ir2;
        SU[0] = SU[0] - scale_t(mi3, w3);
#pragma unroll
        for (int j = 0; j < 3; j++) SU[1 + j] = SU[1 + j] + scale_t(mi4 * n[j], w4);
#pragma unroll
        for (int i = 0; i < 3; i++) {
            T Qn = Q[i][0] * n[0] + Q[i][1] * n[1] + Q[i][2] * n[2];
            SU[NQ * (i + 1)] = SU[NQ * (i + 1)] + scale_t(Qn * ir4 - (M * ir2) * n[i], w2);
            T mn = mi3 * n[i];
#pragma unroll
            for (int j = 0; j < 3; j++) SU[NQ * (i + 1) + 1 + j] = SU[NQ * (i + 1) + 1 + j] + scale_t(mn * n[j], w3);
        }
    }
#pragma unroll
    for (int k = 0; k < NSU; k++) part[it * NSU + k] = Prec<T>::fin(SU[k]);
}

// a9: loc[x][k] = sum over the cell's items (full chunks in order, then the partial one),
// accumulated in binary64; in the scaled modes each item's unit 2^k_I is removed exactly
// (coefficient k carries 2^(k_I d(k)), d from out_deg)
__device__ __forceinline__ double as_double(double v) { return v; }
__device__ __forceinline__ double as_double(float v) { return (double)v; }
__device__ __forceinline__ double as_double(df64 v) { return to_double(v); }

// power of the length unit carried by local coefficient k: standard L_gamma ~ length^-(|gamma|+1);
// conserving S_gamma ~ length^-(|gamma|+3), U_gamma ~ length^-(|gamma|+2)
template <int KIND, int NQ>
__device__ __forceinline__ int out_deg(int k) {
    if (KIND == 0) return mi_deg(k) + 1;
    return k < NQ ? mi_deg(k) + 3 : mi_deg(k % NQ) + 2;
}

template <int NL, int NQ, int KIND, class T>
__global__ void m2l_reduce_k(int nn, const long long* __restrict__ fo, const long long* __restrict__ po,
                             long long nfull, const T* __restrict__ part, const int* __restrict__ kpart,
                             double* __restrict__ loc) {
    constexpr bool SC = !std::is_same<T, double>::value;
    int64_t t = (int64_t)blockIdx.x * EB + threadIdx.x;
    if (t >= (int64_t)nn * NL) return;
    int x = (int)(t / NL), k = (int)(t - (int64_t)x * NL);
    int d = SC ? out_deg<KIND, NQ>(k) : 0;
    double acc = 0.0;
    for (long long i = fo[x]; i < fo[x + 1]; i++) {
        double v = as_double(part[i * NL + k]);
        acc += SC ? v * pow2d(-kpart[i] * d) : v;
    }
    if (po[x + 1] > po[x]) {
        long long i = nfull + po[x];
        double v = as_double(part[i * NL + k]);
        acc += SC ? v * pow2d(-kpart[i] * d) : v;
    }
    loc[t] = acc;
}

// moments of every node in the pair-kernel type, in units of 2^k_n (k_n = floor(log2 r_max)
// for r_max > 0; a node with r_max = 0 has all particles at its centre, so its moments
// beyond the mass vanish and any unit serves), padded to NMP per node: one thread per
// (node, padded coefficient)
template <int P, class T>
__global__ void scale_moments_k(int nn, const double* __restrict__ mom, const double* __restrict__ rmax,
                                T* __restrict__ momT, int* __restrict__ nk) {
    using E = Exp<P>;
    int64_t t = (int64_t)blockIdx.x * EB + threadIdx.x;
    if (t >= (int64_t)nn * E::NMP) return;
    int n = (int)(t / E::NMP), k = (int)(t - (int64_t)n * E::NMP);
    double r = rmax[n];
    int kn = r > 0.0 ? max(-120, min(120, ilogb(r))) : 0;
    momT[t] = k < E::NM ? to_kernel(mom[(int64_t)n * E::NM + k] * pow2d(-kn * mi_deg(k)), T()) : T(0);
    if (k == 0) nk[n] = kn;
}

// the root of node nd's system (roots are nodes 0 .. nsys-1; systems are contiguous in
// particle order, so the node's first particle decides)
__device__ __forceinline__ int root_of(const long long* __restrict__ off, int nsys, int first) {
    int lo = 0, hi = nsys;  // off[lo] <= first < off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= first)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// conserving source moments of every cell (formed once per moment build), about the
// centre of the cell's system root: Q = [M_b | (b_i+1) M_{b+e_i} - z_i M_b], z = Z - Z_root.
// The binary64 M2L then needs no per-pair work on them: with R = z_tgt - z_src,
// sum_b (C_{i,b} + R_i M_b) h_{b+g} = sum_b Q_{i,b} h_{b+g} + z_tgt,i S_g, and the last term
// is added once per target (con_origin_k).  The rounding it adds is about 2^-53 |z| / R
// of the U locals, R the pair separation: 1e-15 for the cells of a Plummer sphere.
template <int P>
__global__ void __launch_bounds__(EB) con_moments_k(int nn, const double* __restrict__ mom,
                                                    const double* __restrict__ Zx, const double* __restrict__ Zy,
                                                    const double* __restrict__ Zz, const int* __restrict__ nfirst,
                                                    const long long* __restrict__ off, int nsys,
                                                    double* __restrict__ cmom) {
    using E = Exp<P>;
    int nd = blockIdx.x * EB + threadIdx.x;
    if (nd >= nn) return;
    int r = root_of(off, nsys, nfirst[nd]);
    double C[E::NSU];
    E::con_moments_o(mom + (int64_t)nd * E::NM, Zx[nd] - Zx[r], Zy[nd] - Zy[r], Zz[nd] - Zz[r], C);
#pragma unroll
    for (int k = 0; k < E::NSU; k++) cmom[(int64_t)nd * E::NSU + k] = C[k];
}

// the target-side term of the root-relative conserving M2L: U_{i,g} += z_i S_g, z = Z - Z_root,
// on the M2L sums of every node (before L2L); one thread per (node, U coefficient)
template <int NQ>
__global__ void con_origin_k(int nn, const double* __restrict__ Zx, const double* __restrict__ Zy,
                             const double* __restrict__ Zz, const int* __restrict__ nfirst,
                             const long long* __restrict__ off, int nsys, double* __restrict__ loc) {
    int64_t t = (int64_t)blockIdx.x * EB + threadIdx.x;
    if (t >= (int64_t)nn * 3 * NQ) return;
    int nd = (int)(t / (3 * NQ)), k = (int)(t - (int64_t)nd * 3 * NQ);
    int i = k / NQ, g = k - i * NQ;
    int r = root_of(off, nsys, nfirst[nd]);
    double z = i == 0 ? Zx[nd] - Zx[r] : (i == 1 ? Zy[nd] - Zy[r] : Zz[nd] - Zz[r]);
    double* L = loc + (int64_t)nd * 4 * NQ;
    L[NQ + k] = fma(z, L[g], L[NQ + k]);
}

// a6 M2M in two steps per level: one thread per (parent, child) shifts the child's
// moments to the parent centre (straight-line, independent accumulators), then one thread
// per (parent, coefficient) adds the children's shifted moments in child order.  A single
// thread per parent would run one long binary64 chain per level, which on GB300 sets the
// level's time.
template <int P>
__global__ void __launch_bounds__(EB) m2m_child_k(int lo, int hi, int cfirst, const int* __restrict__ nparent,
                                                  const double* __restrict__ Zx, const double* __restrict__ Zy,
                                                  const double* __restrict__ Zz, const double* __restrict__ mom,
                                                  double* __restrict__ shifted) {
    using E = Exp<P>;
    // children of the parents in [lo, hi) are the nodes [cfirst, cfirst + gridDim-covered)
    int ch = cfirst + blockIdx.x * EB + threadIdx.x;
    if (ch >= hi) return;
    int par = nparent[ch];
    double M[E::NM];
#pragma unroll
    for (int k = 0; k < E::NM; k++) M[k] = 0.0;
    E::m2m(mom + (int64_t)ch * E::NM, Zx[ch] - Zx[par], Zy[ch] - Zy[par], Zz[ch] - Zz[par], M);
#pragma unroll
    for (int k = 0; k < E::NM; k++) shifted[(int64_t)(ch - cfirst) * E::NM + k] = M[k];
    (void)lo;
}

template <int P>
__global__ void m2m_sum_k(int lo, int hi, int cfirst, const int* __restrict__ nchildf, const int* __restrict__ nnchild,
                          const double* __restrict__ shifted, double* __restrict__ mom) {
    using E = Exp<P>;
    int64_t t = (int64_t)blockIdx.x * EB + threadIdx.x;
    if (t >= (int64_t)(hi - lo) * E::NM) return;
    int nd = lo + (int)(t / E::NM), k = (int)(t - (int64_t)(nd - lo) * E::NM);
    int nc = nnchild[nd];
    if (nc == 0) return;
    int c0 = nchildf[nd] - cfirst;
    double s = 0.0;
    for (int c = 0; c < nc; c++) s += shifted[(int64_t)(c0 + c) * E::NM + k];
    mom[(int64_t)nd * E::NM + k] = s;
}

// a10 L2L, one level: child += shift(parent) by s = Z_child - Z_parent
template <int P>
__global__ void __launch_bounds__(EB) l2l_std_k(int lo, int hi, const int* __restrict__ nparent,
                                                const double* __restrict__ Zx, const double* __restrict__ Zy,
                                                const double* __restrict__ Zz, double* __restrict__ loc) {
    using E = Exp<P>;
    int nd = lo + blockIdx.x * EB + threadIdx.x;
    if (nd >= hi) return;
    int par = nparent[nd];
    double L[E::NM];
#pragma unroll
    for (int k = 0; k < E::NM; k++) L[k] = loc[(int64_t)nd * E::NM + k];
    E::l2l(loc + (int64_t)par * E::NM, Zx[nd] - Zx[par], Zy[nd] - Zy[par], Zz[nd] - Zz[par], L);
#pragma unroll
    for (int k = 0; k < E::NM; k++) loc[(int64_t)nd * E::NM + k] = L[k];
}

template <int P>
__global__ void __launch_bounds__(EB) l2l_con_k(int lo, int hi, const int* __restrict__ nparent,
                                                const double* __restrict__ Zx, const double* __restrict__ Zy,
                                                const double* __restrict__ Zz, double* __restrict__ loc) {
    using E = Exp<P>;
    constexpr int NQ = E::NQ;
    int nd = lo + blockIdx.x * EB + threadIdx.x;
    if (nd >= hi) return;
    int par = nparent[nd];
    double sx = Zx[nd] - Zx[par], sy = Zy[nd] - Zy[par], sz = Zz[nd] - Zz[par];
    const double* Lp = loc + (int64_t)par * E::NSU;
    double* Lc = loc + (int64_t)nd * E::NSU;
    double sh[NQ];
#pragma unroll
    for (int k = 0; k < NQ; k++) sh[k] = 0.0;
    E::l2l_q(Lp, sx, sy, sz, sh);  // shifted parent S
    double t[NQ];
#pragma unroll
    for (int k = 0; k < NQ; k++) t[k] = Lc[k] + sh[k];
#pragma unroll
    for (int k = 0; k < NQ; k++) Lc[k] = t[k];
    const double s3[3] = {sx, sy, sz};
#pragma unroll
    for (int d = 0; d < 3; d++) {
#pragma unroll
        for (int k = 0; k < NQ; k++) t[k] = Lc[(d + 1) * NQ + k];
        E::l2l_q(Lp + (d + 1) * NQ, sx, sy, sz, t);
#pragma unroll
        for (int k = 0; k < NQ; k++) Lc[(d + 1) * NQ + k] = fma(s3[d], sh[k], t[k]);
    }
}

// a11 in the scaled modes: the L2P runs in the pair-kernel type X on every leaf's locals
// expressed in the leaf's unit 2^k (k = nk, the moments' unit exponent, so |x| 2^-k < 2 for
// its particles): with u = x 2^-k, a standard coefficient L_g becomes L_g 2^(k|g|) (the
// acceleration then carries 2^-k), a conserving S_g becomes S_g 2^(k(|g|+1)) and U_g
// becomes U_g 2^(k|g|), so that a = u S''(u) + U'(u) needs no factor.  Every factor is a
// power of two applied in binary64.  The acceptance test bounds a leaf's coefficients of
// degree d by about (M/R) theta^d in these units, so no term leaves binary32's range.  A
// leaf with r_max = 0 has no such bound (single particles can meet in M2L at any
// separation), but all its particles sit at its centre: the L2P there keeps only the
// degree-0 terms, read in binary64 (finish_k), and the leaf is skipped here.  One thread
// per (node, coefficient).
template <int P, int V, class X>
__global__ void scale_locals_k(int nn, const int* __restrict__ nnchild, const double* __restrict__ rmax,
                               const int* __restrict__ nk, const double* __restrict__ loc,
                               const double* __restrict__ locp, X* __restrict__ locT, X* __restrict__ locpT) {
    using E = Exp<P>;
    constexpr int NL = V == 0 ? E::NM : E::NSU, NQ = E::NSU / 4;
    int64_t t = (int64_t)blockIdx.x * EB + threadIdx.x;
    if (t >= (int64_t)nn * NL) return;
    int n = (int)(t / NL), k = (int)(t - (int64_t)n * NL);
    if (nnchild[n] != 0 || rmax[n] == 0.0) return;
    int kn = nk[n];
    int e = V == 0 ? kn * mi_deg(k) : (k < NQ ? kn * (mi_deg(k) + 1) : kn * mi_deg(k % NQ));
    locT[t] = to_kernel(loc[t] * pow2d(e), X());
    if (V != 0 && locp && k < E::NM)
        locpT[(int64_t)n * E::NM + k] = to_kernel(locp[(int64_t)n * E::NM + k] * pow2d(kn * mi_deg(k)), X());
}

// a11 + a13: far field at every particle from its leaf's locals, plus the leaf's P2P item
// sums (full chunks in order, then the partial one), written in input order.  X is the
// L2P arithmetic: binary64, or the pair-kernel type on the scaled locals above.
template <int P, int V, class G, class X>
__global__ void __launch_bounds__(EB) finish_k(int n, const int* __restrict__ leaf_of, const int* __restrict__ nfirst,
                                               const double* __restrict__ xs, const double* __restrict__ ys,
                                               const double* __restrict__ zs, const double* __restrict__ Zx,
                                               const double* __restrict__ Zy, const double* __restrict__ Zz,
                                               const double* __restrict__ rmax, const int* __restrict__ nk,
                                               const double* __restrict__ loc64, const double* __restrict__ locp64,
                                               const X* __restrict__ loc, const X* __restrict__ locp,
                                               const long long* __restrict__ fo,
                                               const long long* __restrict__ po, long long nfull,
                                               const long long* __restrict__ islot, const Quad<G>* __restrict__ ipart,
                                               const Quad<double>* __restrict__ pdirect,
                                               const uint32_t* __restrict__ perm, double* __restrict__ acc_s,
                                               double* __restrict__ pot_s, double* __restrict__ acc_out,
                                               double* __restrict__ pot_out) {
    using E = Exp<P>;
    constexpr bool SC = !std::is_same<X, double>::value;
    int i = blockIdx.x * EB + threadIdx.x;
    if (i >= n) return;
    int lf = leaf_of[i];
    int slot = i - nfirst[lf];
    double x = xs[i] - Zx[lf], y = ys[i] - Zy[lf], z = zs[i] - Zz[lf];
    double sc = 1.0;  // 2^-k in the scaled modes
    if constexpr (SC) {
        sc = pow2d(-nk[lf]);
        x *= sc;
        y *= sc;
        z *= sc;
    }
    X ux = to_kernel(x, X()), uy = to_kernel(y, X()), uz = to_kernel(z, X());
    X bx, by, bz, bp = X(0);
    double ax, ay, az, ph = 0.0;
    if (SC && rmax[lf] == 0.0) {
        // every particle of the leaf is at its centre (x = 0): the degree-0 terms, in binary64
        // (multi-index order 1 | x y z | ...; conserving rows [S | Ux | Uy | Uz])
        if (V == 0) {
            const double* L = loc64 + (int64_t)lf * E::NM;
            ax = -L[1];
            ay = -L[2];
            az = -L[3];
            ph = L[0];
        } else {
            const double* SU = loc64 + (int64_t)lf * E::NSU;
            constexpr int NQ = E::NSU / 4;
            ax = SU[NQ];
            ay = SU[2 * NQ];
            az = SU[3 * NQ];
            if (locp64) ph = locp64[(int64_t)lf * E::NM];
        }
    } else if (V == 0) {
        E::l2p_std(loc + (int64_t)lf * E::NM, ux, uy, uz, bx, by, bz, bp);
        ax = as_double(bx) * sc;
        ay = as_double(by) * sc;
        az = as_double(bz) * sc;
        ph = as_double(bp);
    } else {
        E::l2p_con(loc + (int64_t)lf * E::NSU, ux, uy, uz, bx, by, bz);
        ax = as_double(bx);
        ay = as_double(by);
        az = as_double(bz);
        if (locp) {
            X cx, cy, cz;
            E::l2p_std(locp + (int64_t)lf * E::NM, ux, uy, uz, cx, cy, cz, bp);
            ph = as_double(bp);
        }
    }
    double px = 0.0, py = 0.0, pz = 0.0, pp = 0.0;
    if (pdirect) {  // the fused schedule's per-particle sums
        Quad<double> q = pdirect[i];
        px = q.x;
        py = q.y;
        pz = q.z;
        pp = q.w;
    }
    for (long long k = pdirect ? 0 : fo[lf]; k < (pdirect ? 0 : fo[lf + 1]); k++) {
        Quad<G> q = ipart[islot[k] + slot];
        px += as_double(q.x);
        py += as_double(q.y);
        pz += as_double(q.z);
        pp += as_double(q.w);
    }
    if (!pdirect && po[lf + 1] > po[lf]) {
        Quad<G> q = ipart[islot[nfull + po[lf]] + slot];
        px += as_double(q.x);
        py += as_double(q.y);
        pz += as_double(q.z);
        pp += as_double(q.w);
    }
    ax += px;
    ay += py;
    az += pz;
    ph += pp;
    acc_s[i] = ax;
    acc_s[n + i] = ay;
    acc_s[2 * (int64_t)n + i] = az;
    int64_t j = perm[i];
    acc_out[3 * j] = ax;
    acc_out[3 * j + 1] = ay;
    acc_out[3 * j + 2] = az;
    if (pot_out) {
        pot_s[i] = ph;
        pot_out[j] = ph;
    }
}

// host side, one order P
template <int P>
void run_moments_p(fmm_ctx* c) {
    using E = Exp<P>;
    cudaStream_t s = c->stream;
    int nn = (int)c->n_nodes;
    ensure(c->mom, sizeof(double) * (size_t)nn * E::NM);
    auto p2m64 = [&]() {
        p2m_k<P><<<grid_for(nn, EB), EB, 0, s>>>(nn, c->leaf_order.as<uint32_t>(), c->nfirst.as<int>(),
                                                 c->ncount.as<int>(), c->nnchild.as<int>(), c->xs.as<double>(),
                                                 c->ys.as<double>(), c->zs.as<double>(), c->ms.as<double>(),
                                                 c->nZx.as<double>(), c->nZy.as<double>(), c->nZz.as<double>(),
                                                 c->mom.as<double>());
    };
    if constexpr (P > FMM_MIXED_P_MAX) {  // binary64 only at these orders
        p2m64();
    } else {
        if (c->precision == FMM_FP64)
            p2m64();
        else
            p2m_df_k<P><<<grid_for(nn, EB), EB, 0, s>>>(
                nn, c->leaf_order.as<uint32_t>(), c->nfirst.as<int>(), c->ncount.as<int>(), c->nnchild.as<int>(),
                c->nrmax.as<double>(), c->xs.as<double>(), c->ys.as<double>(), c->zs.as<double>(),
                c->ms.as<double>(), c->nZx.as<double>(), c->nZy.as<double>(), c->nZz.as<double>(),
                c->mom.as<double>());
    }
    GB_LAUNCH("p2m_k");
    for (int l = c->n_levels - 2; l >= 0; l--) {
        int lo = c->level_start[l], hi = c->level_start[l + 1];
        // the children of level l are exactly level l + 1
        int c_lo = c->level_start[l + 1], c_hi = c->level_start[l + 2];
        ensure(c->m2m_tmp, sizeof(double) * (size_t)(c_hi - c_lo) * E::NM);
        m2m_child_k<P><<<grid_for(c_hi - c_lo, EB), EB, 0, s>>>(lo, c_hi, c_lo, c->nparent.as<int>(),
                                                                c->nZx.as<double>(), c->nZy.as<double>(),
                                                                c->nZz.as<double>(), c->mom.as<double>(),
                                                                c->m2m_tmp.as<double>());
        GB_LAUNCH("m2m_child_k");
        m2m_sum_k<P><<<grid_for((int64_t)(hi - lo) * E::NM, EB), EB, 0, s>>>(
            lo, hi, c_lo, c->nchildf.as<int>(), c->nnchild.as<int>(), c->m2m_tmp.as<double>(), c->mom.as<double>());
        GB_LAUNCH("m2m_sum_k");
    }
    if (c->precision == FMM_FP64) {
        if constexpr (P <= 6) {  // the shared-tensor M2L (p = 7, 8 read the raw moments)
            ensure(c->cmom, sizeof(double) * (size_t)nn * E::NSU);
            con_moments_k<P><<<grid_for(nn, EB), EB, 0, s>>>(nn, c->mom.as<double>(), c->nZx.as<double>(),
                                                             c->nZy.as<double>(), c->nZz.as<double>(),
                                                             c->nfirst.as<int>(), c->sys_off.as<long long>(),
                                                             c->n_sys, c->cmom.as<double>());
            GB_LAUNCH("con_moments_k");
        }
        return;
    }
    // the scaled modes: raw moments in the pair-kernel type, range-scaled and padded
    int64_t nmp = (int64_t)nn * E::NMP;
    ensure(c->nk, sizeof(int) * (size_t)nn);
    auto launch = [&](auto* mT) {
        scale_moments_k<P><<<grid_for(nmp, EB), EB, 0, s>>>(nn, c->mom.as<double>(), c->nrmax.as<double>(), mT,
                                                            c->nk.as<int>());
    };
    if (c->precision == FMM_DF64) {
        ensure(c->momT, sizeof(df64) * (size_t)nmp);
        launch(c->momT.as<df64>());
    } else {
        ensure(c->momT, sizeof(float) * (size_t)nmp);
        launch(c->momT.as<float>());
    }
    GB_LAUNCH("scale_moments_k");
}

// the binary64 pair tensors of the current lists at order P (V = 0: D, V = 1: h), formed
// once per walk and order
template <int P, int V>
static const double* pair_tensors(fmm_ctx* c, DevBuf& buf, int64_t& gen, int& order) {
    using E = Exp<P>;
    constexpr int NT = V == 0 ? E::NM : E::NQ, NTP = pair_tensor_stride(NT);
    int64_t np = c->n_m2l;
    if (gen != c->walk_gen || order != P) {
        ensure(buf, sizeof(double) * (size_t)NTP * (size_t)(np > 0 ? np : 1));
        if (np > 0) {
            m2l_ptensor_k<P, V><<<grid_for(np, EB), EB, 0, c->stream>>>(
                np, c->m2l_pairs.as<int2>(), c->nZx.as<double>(), c->nZy.as<double>(), c->nZz.as<double>(),
                buf.as<double>());
            GB_LAUNCH("m2l_ptensor_k");
        }
        gen = c->walk_gen;
        order = P;
    }
    return buf.as<double>();
}

template <int P, class T>
void m2l_launch(fmm_ctx* c, int variant, bool std_locals) {
    using E = Exp<P>;
    cudaStream_t s = c->stream;
    int nn = (int)c->n_nodes;
    const uint32_t* dir = c->m2l_dir.as<uint32_t>();
    const ItemSet& it = c->m2l_items;
    int64_t ni = it.n_items;
    bool native = c->precision == FMM_FP64;
    const T* mom = native ? c->mom.as<T>() : c->momT.as<T>();
    const T* cmom = native ? c->cmom.as<T>() : c->momT.as<T>();  // scaled modes: raw moments
    M2LGeom g{c->nZx.as<double>(), c->nZy.as<double>(), c->nZz.as<double>(), nullptr, nullptr, nullptr};
    if (!native) {
        g.zh = c->zhl.as<float4>();
        g.zl = g.zh + nn;
        g.nk = c->nk.as<int>();
    }
    int nl_max = E::NSU > E::NM ? E::NSU : E::NM;
    ensure(c->m2l_part, sizeof(T) * (size_t)(ni > 0 ? ni : 1) * nl_max);
    ensure(c->m2l_kpart, sizeof(int) * (size_t)(ni > 0 ? ni : 1));
    T* part = c->m2l_part.as<T>();
    int* kpart = c->m2l_kpart.as<int>();
    auto reduce = [&](auto kern, int NL, double* out) {
        kern<<<grid_for((int64_t)nn * NL, EB), EB, 0, s>>>(nn, it.fo.as<long long>(), it.po.as<long long>(), it.n_full,
                                                          part, kpart, out);
        GB_LAUNCH("m2l_reduce_k");
    };
    if (variant == 2) {
        // the literal order-0 realigned form runs at expansion order 2 only
        if constexpr (P == 2) {
            static_assert(E::NMP == 16 && E::NM == 10, "m2l_p0_k: moment strides of order 2");
            ensure(c->loc, sizeof(double) * (size_t)nn * E::NSU);
            if (ni > 0) {
                m2l_p0_k<T><<<grid_for(ni, EB), EB, 0, s>>>(ni, it.items.as<int4>(), dir, g, mom, part,
                                                            kpart);
                GB_LAUNCH("m2l_p0_k");
            }
            reduce(m2l_reduce_k<E::NSU, E::NQ, 1, T>, E::NSU, c->loc.as<double>());
        }
    }
    if constexpr (std::is_same<T, double>::value && P <= 6) {
        if (c->schedule == FMM_SCHEDULE_FUSED) {  // no lists: one traversal per target node
            if (variant == 1) {
                ensure(c->loc, sizeof(double) * (size_t)nn * E::NSU);
                fused_m2l_launch<P>(c, 1, c->fused_theta, c->loc.as<double>());
                con_origin_k<E::NQ><<<grid_for((int64_t)nn * 3 * E::NQ, EB), EB, 0, s>>>(
                    nn, c->nZx.as<double>(), c->nZy.as<double>(), c->nZz.as<double>(), c->nfirst.as<int>(),
                    c->sys_off.as<long long>(), c->n_sys, c->loc.as<double>());
                GB_LAUNCH("con_origin_k");
            }
            if (std_locals) {
                DevBuf& L = variant == 0 ? c->loc : c->locp;
                ensure(L, sizeof(double) * (size_t)nn * E::NM);
                fused_m2l_launch<P>(c, 0, c->fused_theta, L.as<double>());
            }
            return;
        }
    }
    if (variant == 1) {
        ensure(c->loc, sizeof(double) * (size_t)nn * E::NSU);
        if (ni > 0) {
            if constexpr (P >= 7) {
                m2l_generic_launch(c, P, 1, reinterpret_cast<double*>(part));
            } else if constexpr (std::is_same<T, double>::value) {
                const double* pt = pair_tensors<P, 1>(c, c->m2l_pth, c->pth_gen, c->pth_p);
                m2l_con_t_k<P><<<grid_for(ni, EB), EB, 0, s>>>(ni, it.items.as<int4>(), dir,
                                                               c->m2l_dirp.as<uint32_t>(), pt, cmom, part);
                GB_LAUNCH("m2l_con_t_k");
            } else {
                m2l_con_k<P, T><<<grid_for(ni, EB), EB, 0, s>>>(ni, it.items.as<int4>(), dir, g, cmom, part,
                                                                kpart);
                GB_LAUNCH("m2l_con_k");
            }
        }
        reduce(m2l_reduce_k<E::NSU, E::NQ, 1, T>, E::NSU, c->loc.as<double>());
        if constexpr (P <= 6 && std::is_same<T, double>::value) {
            con_origin_k<E::NQ><<<grid_for((int64_t)nn * 3 * E::NQ, EB), EB, 0, s>>>(
                nn, c->nZx.as<double>(), c->nZy.as<double>(), c->nZz.as<double>(), c->nfirst.as<int>(),
                c->sys_off.as<long long>(), c->n_sys, c->loc.as<double>());
            GB_LAUNCH("con_origin_k");
        }
    }
    if (std_locals) {
        DevBuf& L = variant == 0 ? c->loc : c->locp;
        ensure(L, sizeof(double) * (size_t)nn * E::NM);
        if (ni > 0) {
            if constexpr (P >= 7) {
                m2l_generic_launch(c, P, 0, reinterpret_cast<double*>(part));
            } else if constexpr (std::is_same<T, double>::value) {
                const double* pt = pair_tensors<P, 0>(c, c->m2l_ptd, c->ptd_gen, c->ptd_p);
                m2l_std_t_k<P><<<grid_for(ni, EB), EB, 0, s>>>(ni, it.items.as<int4>(), dir,
                                                               c->m2l_dirp.as<uint32_t>(), pt, mom, part);
                GB_LAUNCH("m2l_std_t_k");
            } else {
                m2l_std_k<P, T><<<grid_for(ni, EB), EB, 0, s>>>(ni, it.items.as<int4>(), dir, g, mom, part,
                                                                kpart);
                GB_LAUNCH("m2l_std_k");
            }
        }
        reduce(m2l_reduce_k<E::NM, E::NQ, 0, T>, E::NM, L.as<double>());
    }
}

template <int P>
void run_far_field_p(fmm_ctx* c, int variant, bool want_pot) {
    cudaStream_t s = c->stream;
    bool std_locals = (variant == 0) || want_pot;
    stage_begin(c, ST_M2L);
    if (c->precision == FMM_FP64)
        m2l_launch<P, double>(c, variant, std_locals);
    else if (c->precision == FMM_DF64) {
        if constexpr (P <= FMM_DF64_P_MAX) m2l_launch<P, df64>(c, variant, std_locals);
    } else {
        if constexpr (P <= FMM_MIXED_P_MAX) m2l_launch<P, float>(c, variant, std_locals);
    }
    stage_end(c, ST_M2L);
    stage_begin(c, ST_L2L);
    for (int l = 1; l < c->n_levels; l++) {
        int lo = c->level_start[l], hi = c->level_start[l + 1];
        if constexpr (P >= 7) {
            // table-driven at the high orders (straight-line shifts take minutes to compile)
            if (variant != 0) l2l_generic_launch(c, P, 1, lo, hi, c->loc.as<double>());
            if (std_locals) l2l_generic_launch(c, P, 0, lo, hi, (variant == 0 ? c->loc : c->locp).as<double>());
        } else {
            if (variant != 0) {
                l2l_con_k<P><<<grid_for(hi - lo, EB), EB, 0, s>>>(lo, hi, c->nparent.as<int>(), c->nZx.as<double>(),
                                                                  c->nZy.as<double>(), c->nZz.as<double>(),
                                                                  c->loc.as<double>());
                GB_LAUNCH("l2l_con_k");
            }
            if (std_locals) {
                DevBuf& L = variant == 0 ? c->loc : c->locp;
                l2l_std_k<P><<<grid_for(hi - lo, EB), EB, 0, s>>>(lo, hi, c->nparent.as<int>(),
                                                                  c->nZx.as<double>(), c->nZy.as<double>(),
                                                                  c->nZz.as<double>(), L.as<double>());
                GB_LAUNCH("l2l_std_k");
            }
        }
    }
    stage_end(c, ST_L2L);
}

template <int P, class G, class X>
static void finish_launch(fmm_ctx* c, int variant, bool want_pot, double* acc_out, double* pot_out) {
    using E = Exp<P>;
    cudaStream_t s = c->stream;
    int n = (int)c->N;
    int nn = (int)c->n_nodes;
    const ItemSet& it = c->p2p_items;
    bool pot_con = variant != 0 && want_pot;  // potentials of the realigned forms: standard locals
    const X* locX = nullptr;
    const X* locpX = nullptr;
    if constexpr (std::is_same<X, double>::value) {
        locX = c->loc.as<double>();
        locpX = pot_con ? c->locp.as<double>() : nullptr;
    } else {
        int NL = variant == 0 ? E::NM : E::NSU;
        ensure(c->locT, sizeof(X) * (size_t)nn * NL);
        if (pot_con) ensure(c->locpT, sizeof(X) * (size_t)nn * E::NM);
        auto sl = [&](auto kern) {
            kern<<<grid_for((int64_t)nn * NL, EB), EB, 0, s>>>(
                nn, c->nnchild.as<int>(), c->nrmax.as<double>(), c->nk.as<int>(), c->loc.as<double>(),
                pot_con ? c->locp.as<double>() : nullptr, c->locT.as<X>(), pot_con ? c->locpT.as<X>() : nullptr);
        };
        if (variant == 0)
            sl(scale_locals_k<P, 0, X>);
        else
            sl(scale_locals_k<P, 1, X>);
        GB_LAUNCH("scale_locals_k");
        locX = c->locT.as<X>();
        locpX = pot_con ? c->locpT.as<X>() : nullptr;
    }
    auto args = [&](auto kern) {
        kern<<<grid_for(n, EB), EB, 0, s>>>(
            n, c->leaf_of.as<int>(), c->nfirst.as<int>(), c->xs.as<double>(), c->ys.as<double>(), c->zs.as<double>(),
            c->nZx.as<double>(), c->nZy.as<double>(), c->nZz.as<double>(), c->nrmax.as<double>(), c->nk.as<int>(),
            c->loc.as<double>(), pot_con ? c->locp.as<double>() : nullptr, locX, locpX,
            it.fo.as<long long>(), it.po.as<long long>(), it.n_full, c->p2p_islot.as<long long>(),
            c->p2p_ipart.as<Quad<G>>(),
            c->schedule == FMM_SCHEDULE_FUSED ? c->p2p_direct.as<Quad<double>>() : nullptr,
            c->perm.as<uint32_t>(), c->acc_s.as<double>(), c->pot_s.as<double>(), acc_out,
            want_pot ? pot_out : nullptr);
    };
    if (variant == 0)
        args(finish_k<P, 0, G, X>);
    else
        args(finish_k<P, 1, G, X>);
    GB_LAUNCH("finish_k");
}

// the L2P arithmetic follows the pair kernels': binary64, or double-float / binary32 on
// leaf-scaled locals (the modes' order limits are checked at the API)
template <int P>
void run_finish_p(fmm_ctx* c, int variant, bool want_pot, double* acc_out, double* pot_out) {
    if (c->precision == FMM_FP64) {
        finish_launch<P, double, double>(c, variant, want_pot, acc_out, pot_out);
    } else if (c->precision == FMM_DF64) {
        if constexpr (P <= FMM_DF64_P_MAX)
            finish_launch<P, df64, df64>(c, variant, want_pot, acc_out, pot_out);
        else
            throw FmmError{FMM_ERR_INVALID, "double-float mode: order above FMM_DF64_P_MAX"};
    } else {
        if constexpr (P <= FMM_MIXED_P_MAX)
            finish_launch<P, df64, float>(c, variant, want_pot, acc_out, pot_out);
        else
            throw FmmError{FMM_ERR_INVALID, "mixed mode: order above FMM_MIXED_P_MAX"};
    }
}

// One translation unit per order instantiates the order's stages; the M2L launches of
// each arithmetic type get translation units of their own (compiled in parallel).
#define GBFMM_INSTANTIATE(P)                                                                             \
    extern template void m2l_launch<P, double>(fmm_ctx*, int, bool);                                    \
    extern template void m2l_launch<P, float>(fmm_ctx*, int, bool);                                     \
    extern template void m2l_launch<P, df64>(fmm_ctx*, int, bool);                                      \
    template void run_moments_p<P>(fmm_ctx*);                                                           \
    template void run_far_field_p<P>(fmm_ctx*, int, bool);                                              \
    template void run_finish_p<P>(fmm_ctx*, int, bool, double*, double*);

#define GBFMM_INSTANTIATE_M2L(P, T) template void m2l_launch<P, T>(fmm_ctx*, int, bool);

}  // namespace gbfmm
