// The decision rule of the mutual dual-tree walk (Sec. 2, eq. mac_criterion), shared by the
// level-synchronous walk (walk.cu) and the fused per-target traversal (fused.cu), so that
// both take exactly the same decisions.
#pragma once
#include "fmm_device.cuh"
#include "fmm_internal.h"

namespace gbfmm {

__device__ __forceinline__ bool mac_accept(const NodeView& nv, int A, int B, double theta) {
    double dx = __dsub_rn(nv.Zx[A], nv.Zx[B]);
    double dy = __dsub_rn(nv.Zy[A], nv.Zy[B]);
    double dz = __dsub_rn(nv.Zz[A], nv.Zz[B]);
    double R = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
    return R > 0.0 && __dadd_rn(nv.rmax[A], nv.rmax[B]) <= __dmul_rn(theta, R);
}

// binary32 prefilter of mac_accept: 1 accept, 0 reject, -1 too close to call.  The
// separation comes from the double-float centre words ((hi - hi) + (lo - lo): exact high
// difference when the centres are close, else within 2^-23), r_max is rounded up, and the
// squared test (r_A + r_B)^2 vs theta^2 R^2 carries a relative error below 2^-18 while
// max|Z| / R <= 2^20 and nothing under- or overflows; a 2^-12 margin on either side is
// therefore decided exactly as the binary64 test decides it, and the rest (ties within
// the margin, extreme ranges) falls through to that test.
__device__ __forceinline__ int mac_fast(const NodeView& nv, int A, int B, float th2) {
    float4 ah = nv.zh[A], bh = nv.zh[B], al = nv.zl[A], bl = nv.zl[B];
    float dx = __fadd_rn(__fsub_rn(ah.x, bh.x), __fsub_rn(al.x, bl.x));
    float dy = __fadd_rn(__fsub_rn(ah.y, bh.y), __fsub_rn(al.y, bl.y));
    float dz = __fadd_rn(__fsub_rn(ah.z, bh.z), __fsub_rn(al.z, bl.z));
    float R2 = dx * dx + dy * dy + dz * dz;
    float z2 = fmaxf(ah.x * ah.x + ah.y * ah.y + ah.z * ah.z, bh.x * bh.x + bh.y * bh.y + bh.z * bh.z);
    if (!(R2 >= 0x1p-100f && R2 <= 0x1p100f) || R2 < 0x1p-40f * z2 || !(ah.w + bh.w <= 0x1p50f)) return -1;
    float rs = ah.w + bh.w;
    float lhs = rs * rs, rhs = th2 * R2;
    if (lhs <= rhs * (1.f - 0x1p-12f)) return 1;
    if (lhs >= rhs * (1.f + 0x1p-12f)) return 0;
    return -1;
}

// true: split A; false: split B (neither is a leaf here)
__device__ __forceinline__ bool split_a(const NodeView& nv, int A, int B) {
    double ra = nv.rmax[A], rb = nv.rmax[B];
    if (ra != rb) return ra > rb;
    int ca = nv.count[A], cb = nv.count[B];
    if (ca != cb) return ca > cb;
    return A < B;
}

// decision: 0 = split, 1 = M2L, 2 = P2P; *split_node / *nnew for splits
__device__ __forceinline__ int decide(const NodeView& nv, int2 it, double theta, float th2, int* nnew, bool* sa) {
    int A = it.x, B = it.y;
    if (A == B) {
        int nc = nv.nchild[A];
        if (nc == 0) return 2;
        *nnew = nc * (nc + 1) / 2;
        return 0;
    }
    int f = mac_fast(nv, A, B, th2);
    if (f == 1 || (f < 0 && mac_accept(nv, A, B, theta))) return 1;
    bool la = nv.nchild[A] == 0, lb = nv.nchild[B] == 0;
    if (la && lb) return 2;
    bool s = lb ? true : (la ? false : split_a(nv, A, B));
    *sa = s;
    *nnew = nv.nchild[s ? A : B];
    return 0;
}

}  // namespace gbfmm
