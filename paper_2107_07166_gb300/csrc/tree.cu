// Tree build: bounding cube, Morton keys, radix sort, breadth-first octree, centres of
// mass and exact r_max (Sec. 2: nodes with COM Z and r_max of eq. mac_criterion).
//
// Every geometric quantity is computed with explicitly rounded IEEE operations
// (__dadd_rn, __dmul_rn, __ddiv_rn, __dsqrt_rn) in a fixed order, so that keys, tree,
// centres of mass, radii and the acceptance decisions of the walk are reproducible bit
// for bit by any binary64 implementation using the same order:
//   cube:  lo = per-axis minimum, side = max extent (1 if zero), scale = 2^21 / side
//   key:   q_d = min(floor((x_d - lo_d) * scale), 2^21 - 1), bits interleaved x,y,z
//   COM:   leaves sum m and m*X sequentially in sorted order; parents sum their
//          children's sums in child order; Z = (sum m X) / M
//   r_max: sqrt of the maximum over the node's particles of (dx*dx + dy*dy) + dz*dz
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include <cooperative_groups.h>

#include "fmm_device.cuh"
#include "fmm_internal.h"

namespace gbfmm {

namespace cg = cooperative_groups;

constexpr int MAX_LEVEL = 21;
constexpr int TB = 256;

// ------------------------------------------------------------------ cube + validation

// Per-block min/max of each axis plus a flag for non-finite coordinates or bad masses.
__global__ void bbox_partial_k(const double* __restrict__ x, const double* __restrict__ m, int64_t n,
                               double* __restrict__ part, int* __restrict__ bad) {
    __shared__ double smn[3][TB], smx[3][TB];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    int b = 0;
    for (int64_t i = (int64_t)blockIdx.x * TB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TB) {
        for (int d = 0; d < 3; d++) {
            double v = x[3 * i + d];
            if (!isfinite(v)) b = 1;
            mn[d] = fmin(mn[d], v);
            mx[d] = fmax(mx[d], v);
        }
        double mm = m[i];
        if (!(mm >= 0.0) || !isfinite(mm)) b = 1;
    }
    if (b) atomicOr(bad, 1);
    for (int d = 0; d < 3; d++) {
        smn[d][threadIdx.x] = mn[d];
        smx[d][threadIdx.x] = mx[d];
    }
    __syncthreads();
    for (int s = TB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int d = 0; d < 3; d++) {
                smn[d][threadIdx.x] = fmin(smn[d][threadIdx.x], smn[d][threadIdx.x + s]);
                smx[d][threadIdx.x] = fmax(smx[d][threadIdx.x], smx[d][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < 3; d++) {
            part[6 * blockIdx.x + d] = smn[d][0];
            part[6 * blockIdx.x + 3 + d] = smx[d][0];
        }
}

// geom[0..2] = lo, geom[3] = side, geom[4] = scale.  One block, a tree over the partials
// (min and max are exact, so the grouping does not matter).
constexpr int BFB = 512;
__global__ void __launch_bounds__(BFB) bbox_final_k(const double* __restrict__ part, int nb, double* __restrict__ geom) {
    __shared__ double smn[3][BFB], smx[3][BFB];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = threadIdx.x; b < nb; b += BFB)
        for (int d = 0; d < 3; d++) {
            mn[d] = fmin(mn[d], part[6 * b + d]);
            mx[d] = fmax(mx[d], part[6 * b + 3 + d]);
        }
    for (int d = 0; d < 3; d++) {
        smn[d][threadIdx.x] = mn[d];
        smx[d][threadIdx.x] = mx[d];
    }
    __syncthreads();
    for (int st = BFB / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            for (int d = 0; d < 3; d++) {
                smn[d][threadIdx.x] = fmin(smn[d][threadIdx.x], smn[d][threadIdx.x + st]);
                smx[d][threadIdx.x] = fmax(smx[d][threadIdx.x], smx[d][threadIdx.x + st]);
            }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    double side = 0.0;
    for (int d = 0; d < 3; d++) {
        geom[d] = smn[d][0];
        double e = __dsub_rn(smx[d][0], smn[d][0]);
        if (e > side) side = e;
    }
    if (side == 0.0) side = 1.0;
    geom[3] = side;
    geom[4] = __ddiv_rn(2097152.0, side);
}

// ------------------------------------------------------------------ keys

__device__ __forceinline__ uint64_t spread_bits3(uint64_t v) {
    // place bit b of a 21-bit value at bit 3b
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x001f00000000ffffull;
    v = (v | (v << 16)) & 0x001f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__device__ __forceinline__ uint64_t quantise(double x, double lo, double scale) {
    double t = __dmul_rn(__dsub_rn(x, lo), scale);
    double f = floor(t);
    uint64_t q = (f <= 0.0) ? 0ull : (uint64_t)f;
    return q > 2097151ull ? 2097151ull : q;
}

// The block's TB particles are 3 TB consecutive doubles of x: they are read as 16-byte
// double2 loads (coalesced; the block's span starts on a 16-byte boundary because 3 TB is
// even, when x itself is 16-byte aligned, checked here) into shared memory, and each
// thread then takes its own three coordinates.  The block at the end of the array, or an
// x not 16-byte aligned, reads doubles one by one.
__global__ void keys_k(const double* __restrict__ x, int64_t n, const double* __restrict__ geom,
                       uint64_t* __restrict__ keys, uint32_t* __restrict__ idx) {
    __shared__ double sx[3 * TB];
    int64_t b0 = (int64_t)blockIdx.x * TB;
    int64_t i = b0 + threadIdx.x;
    int cnt = (int)min((int64_t)TB, n - b0);  // particles of this block
    const double* xb = x + 3 * b0;
    if (cnt == TB && (reinterpret_cast<uintptr_t>(xb) & 15u) == 0) {
        const double2* x2 = reinterpret_cast<const double2*>(xb);
        for (int k = threadIdx.x; k < 3 * TB / 2; k += TB) {
            double2 v = x2[k];
            sx[2 * k] = v.x;
            sx[2 * k + 1] = v.y;
        }
    } else {
        for (int k = threadIdx.x; k < 3 * cnt; k += TB) sx[k] = xb[k];
    }
    __syncthreads();
    if (i >= n) return;
    double lo0 = geom[0], lo1 = geom[1], lo2 = geom[2], sc = geom[4];
    int t = threadIdx.x;
    uint64_t qx = quantise(sx[3 * t], lo0, sc);
    uint64_t qy = quantise(sx[3 * t + 1], lo1, sc);
    uint64_t qz = quantise(sx[3 * t + 2], lo2, sc);
    keys[i] = (spread_bits3(qx) << 2) | (spread_bits3(qy) << 1) | spread_bits3(qz);
    idx[i] = (uint32_t)i;
}

__global__ void gather_k(const double* __restrict__ x, const double* __restrict__ m,
                         const uint32_t* __restrict__ perm, int64_t n, double* __restrict__ xs,
                         double* __restrict__ ys, double* __restrict__ zs, double* __restrict__ ms) {
    int64_t i = (int64_t)blockIdx.x * TB + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm[i];
    xs[i] = x[3 * j];
    ys[i] = x[3 * j + 1];
    zs[i] = x[3 * j + 2];
    ms[i] = m[j];
}

// ------------------------------------------------------------------ octree, level by level

// A node at `level` splits when it holds more than `leaf` particles and level < MAX_LEVEL.
// Its particles' keys are sorted and share the node's prefix, so the level+1 octant
// digit never decreases over [f, e): child o starts at the first particle whose digit is
// at least o, and octants with no particle are omitted.  One thread per (node, octant)
// finds that bound by binary search (lanes 8t .. 8t + 7 of a warp hold node t's octants),
// so a level costs one search depth of latency and work proportional to its nodes.
struct Octant {
    int b, next;  // octant range [b, next)
    bool split;   // the node splits
    unsigned grp; // non-empty octants of the node, bit o
};

__device__ __forceinline__ Octant octant_of(const uint64_t* __restrict__ keys, bool in, int f, int cn, int level,
                                            int leaf, int o) {
    Octant r;
    r.split = in && cn > leaf && level < MAX_LEVEL;
    int e = f + cn, lo = f;
    if (r.split && o > 0) {
        int hi = e, shift = 60 - 3 * level;
        while (lo < hi) {
            int mid = lo + ((hi - lo) >> 1);
            if ((int)((keys[mid] >> shift) & 7ull) < o)
                lo = mid + 1;
            else
                hi = mid;
        }
    }
    r.b = lo;
    int nb = __shfl_down_sync(FULL, lo, 1, 8);
    r.next = o == 7 ? e : nb;
    unsigned bal = __ballot_sync(FULL, r.split && r.next > r.b);
    r.grp = (bal >> (threadIdx.x & 24)) & 0xffu;
    return r;
}

// number of children of the m nodes lo .. lo + m - 1 of `level`
__global__ void split_count_k(const uint64_t* __restrict__ keys, int lo, int m, int level, int leaf,
                              const int* __restrict__ nfirst, const int* __restrict__ ncount, int* __restrict__ nch) {
    int64_t g = (int64_t)blockIdx.x * TB + threadIdx.x;
    int t = (int)(g >> 3), o = (int)(g & 7);
    bool in = t < m;  // groups of 8 are whole: all in or all out
    int f = in ? nfirst[lo + t] : 0, cn = in ? ncount[lo + t] : 0;
    Octant q = octant_of(keys, in, f, cn, level, leaf, o);
    if (in && o == 0) nch[t] = __popc(q.grp);
}

// children of the level's nodes get breadth-first ids new_base + pos[t] + (rank among the
// node's non-empty octants); pos is the exclusive scan of nch
__global__ void split_emit_k(const uint64_t* __restrict__ keys, int lo, int m, int level, int leaf, int new_base,
                             const int* __restrict__ pos, int* __restrict__ nfirst, int* __restrict__ ncount,
                             int* __restrict__ nlevel, int* __restrict__ nparent, int* __restrict__ nchildf,
                             int* __restrict__ nnchild) {
    int64_t g = (int64_t)blockIdx.x * TB + threadIdx.x;
    int t = (int)(g >> 3), o = (int)(g & 7);
    bool in = t < m;
    int nd = lo + t;
    int f = in ? nfirst[nd] : 0, cn = in ? ncount[nd] : 0;
    Octant q = octant_of(keys, in, f, cn, level, leaf, o);
    if (!in || q.grp == 0u) return;  // a leaf keeps nchildf = -1, nnchild = 0 from its creation
    int base = new_base + pos[t];
    if (o == 0) {
        nchildf[nd] = base;
        nnchild[nd] = __popc(q.grp);
    }
    if ((q.grp >> o) & 1u) {
        int id = base + __popc(q.grp & ((1u << o) - 1u));
        nfirst[id] = q.b;
        ncount[id] = q.next - q.b;
        nlevel[id] = level + 1;
        nparent[id] = nd;
        nchildf[id] = -1;
        nnchild[id] = 0;
    }
}

// The octree level by level without host round trips.  Each level fuses the child count,
// its prefix over the level and the emission of the children: blocks take tiles of
// LV_NODES consecutive nodes in ticket order, the node's 8 lanes find its octant bounds
// (octant_of), a block scan places the children inside the tile, and the tile's place
// among the level's children comes from a decoupled look-back over the tiles before it.
// The level's bounds live in device memory (LevelCtl::start); the last tile of level L
// writes start[L + 2].  All levels run in one cooperative launch with a grid barrier
// between levels, and the host reads the table once.  Children beyond the node capacity
// are counted but not stored (the host grows the arrays and builds the levels again).
constexpr int LV_NODES = TB / 8;
constexpr long long LEVEL_SPIN_LIMIT = 1ll << 22;  // polls of one status word (~0.1-1 s)

struct LevelCtl {
    int start[MAX_LEVEL + 2];  // first node id of level L; start[L + 1] - start[L] nodes at level L
    int ticket[MAX_LEVEL];     // tile tickets of level L's launch
    int overflow;              // a level did not fit the node arrays
    int err;                   // a look-back wait ran out
};

// The tiles of one level (all blocks of the grid take part)
__device__ __forceinline__ void split_level_tiles(const uint64_t* __restrict__ keys, int level, int leaf, int lo,
                                                  int hi, LevelCtl* __restrict__ ctl,
                                                  unsigned long long* __restrict__ status, int* __restrict__ nfirst,
                                                  int* __restrict__ ncount, int* __restrict__ nlevel,
                                                  int* __restrict__ nparent, int* __restrict__ nchildf,
                                                  int* __restrict__ nnchild, int cap_nodes) {
    __shared__ int s_tile, s_base;
    int m = hi - lo;
    int ntiles = (m + LV_NODES - 1) / LV_NODES;
    const unsigned tag_agg = 2u * (unsigned)level + 1u, tag_pre = 2u * (unsigned)level + 2u;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&ctl->ticket[level], 1);
        __syncthreads();
        int tile = s_tile;
        if (tile >= ntiles) break;
        int t = tile * LV_NODES + (threadIdx.x >> 3), o = threadIdx.x & 7;
        bool in = t < m;  // groups of 8 lanes are whole: all in or all out
        int nd = lo + t;
        int f = in ? nfirst[nd] : 0, cn = in ? ncount[nd] : 0;
        Octant q = octant_of(keys, in, f, cn, level, leaf, o);
        int cnt = __popc(q.grp);
        int tot;
        int ex = block_exclusive_scan((in && o == 0) ? cnt : 0, &tot);
        int pos = __shfl_sync(FULL, ex, (threadIdx.x & 31) & ~7);  // the node's offset in the tile
        if (threadIdx.x < 32) {
            // publish the tile's count before looking back (tiles behind it need not wait
            // for its prefix), then its inclusive prefix; one thread writes both, in order
            if (threadIdx.x == 0 && tile > 0) st_status(status + tile, tag_agg, tot);
            int pre = lookback_prefix(status, tile, tag_agg, tag_pre, LEVEL_SPIN_LIMIT, &ctl->err);
            if (threadIdx.x == 0) {
                st_status(status + tile, tag_pre, pre + tot);
                if (tile == ntiles - 1) ctl->start[level + 2] = hi + pre + tot;
                s_base = hi + pre;
            }
        }
        __syncthreads();
        if (in && q.grp != 0u) {
            int base = s_base + pos;
            if (o == 0) {
                nchildf[nd] = base;
                nnchild[nd] = cnt;
            }
            int id = base + __popc(q.grp & ((1u << o) - 1u));
            if (((q.grp >> o) & 1u) && id < cap_nodes) {
                nfirst[id] = q.b;
                ncount[id] = q.next - q.b;
                nlevel[id] = level + 1;
                nparent[id] = nd;
                nchildf[id] = -1;
                nnchild[id] = 0;
            }
        }
        __syncthreads();  // s_tile and s_base are reused by the next tile
    }
}

// All levels in one cooperative launch: the blocks stay resident, take the level's tiles,
// meet at a grid barrier, and read the next level's bounds, which the last tile wrote
// before the barrier; every block reads the same bounds and flags, so every block leaves
// the level loop at the same level (the first empty one, or on an error or overflow).
__global__ void __launch_bounds__(TB) split_levels_k(const uint64_t* __restrict__ keys, int leaf, int cap_nodes,
                                                     LevelCtl* __restrict__ ctl,
                                                     unsigned long long* __restrict__ status,
                                                     int* __restrict__ nfirst, int* __restrict__ ncount,
                                                     int* __restrict__ nlevel, int* __restrict__ nparent,
                                                     int* __restrict__ nchildf, int* __restrict__ nnchild) {
    cg::grid_group grid = cg::this_grid();
    for (int level = 0; level < MAX_LEVEL; level++) {
        volatile LevelCtl* vc = ctl;
        int lo = vc->start[level], hi = vc->start[level + 1];
        if (hi <= lo || vc->err || vc->overflow) break;
        if (hi > cap_nodes) {  // the level's nodes were not stored: the host grows the arrays
            if (blockIdx.x == 0 && threadIdx.x == 0) ctl->overflow = 1;
            break;
        }
        split_level_tiles(keys, level, leaf, lo, hi, ctl, status, nfirst, ncount, nlevel, nparent, nchildf, nnchild,
                          cap_nodes);
        grid.sync();
    }
}

// leaf of every particle
__global__ void leaf_of_k(int nn, const int* __restrict__ nfirst, const int* __restrict__ ncount,
                          const int* __restrict__ nnchild, int* __restrict__ leaf_of) {
    int nd = blockIdx.x * TB + threadIdx.x;
    if (nd >= nn || nnchild[nd] != 0) return;
    int f = nfirst[nd], e = f + ncount[nd];
    for (int i = f; i < e; i++) leaf_of[i] = nd;
}

// ------------------------------------------------------------------ centres of mass

__global__ void com_leaf_k(int nn, const int* __restrict__ nfirst, const int* __restrict__ ncount,
                           const int* __restrict__ nnchild, const double* __restrict__ xs,
                           const double* __restrict__ ys, const double* __restrict__ zs,
                           const double* __restrict__ ms, double* __restrict__ M, double* __restrict__ Sx,
                           double* __restrict__ Sy, double* __restrict__ Sz, double* __restrict__ Zx,
                           double* __restrict__ Zy, double* __restrict__ Zz) {
    int nd = blockIdx.x * TB + threadIdx.x;
    if (nd >= nn || nnchild[nd] != 0) return;
    int f = nfirst[nd], e = f + ncount[nd];
    double m = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    for (int i = f; i < e; i++) {
        double mi = ms[i];
        m = __dadd_rn(m, mi);
        sx = __dadd_rn(sx, __dmul_rn(mi, xs[i]));
        sy = __dadd_rn(sy, __dmul_rn(mi, ys[i]));
        sz = __dadd_rn(sz, __dmul_rn(mi, zs[i]));
    }
    M[nd] = m;
    Sx[nd] = sx;
    Sy[nd] = sy;
    Sz[nd] = sz;
    bool ok = m > 0.0;
    Zx[nd] = ok ? __ddiv_rn(sx, m) : xs[f];
    Zy[nd] = ok ? __ddiv_rn(sy, m) : ys[f];
    Zz[nd] = ok ? __ddiv_rn(sz, m) : zs[f];
}

__global__ void com_inner_k(int lo, int hi, const int* __restrict__ nfirst, const int* __restrict__ nchildf,
                            const int* __restrict__ nnchild, const double* __restrict__ xs,
                            const double* __restrict__ ys, const double* __restrict__ zs, double* __restrict__ M,
                            double* __restrict__ Sx, double* __restrict__ Sy, double* __restrict__ Sz,
                            double* __restrict__ Zx, double* __restrict__ Zy, double* __restrict__ Zz) {
    int nd = lo + blockIdx.x * TB + threadIdx.x;
    if (nd >= hi || nnchild[nd] == 0) return;
    int c0 = nchildf[nd], c1 = c0 + nnchild[nd];
    double m = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    for (int c = c0; c < c1; c++) {
        m = __dadd_rn(m, M[c]);
        sx = __dadd_rn(sx, Sx[c]);
        sy = __dadd_rn(sy, Sy[c]);
        sz = __dadd_rn(sz, Sz[c]);
    }
    M[nd] = m;
    Sx[nd] = sx;
    Sy[nd] = sy;
    Sz[nd] = sz;
    int f = nfirst[nd];
    bool ok = m > 0.0;
    Zx[nd] = ok ? __ddiv_rn(sx, m) : xs[f];
    Zy[nd] = ok ? __ddiv_rn(sy, m) : ys[f];
    Zz[nd] = ok ? __ddiv_rn(sz, m) : zs[f];
}

// ------------------------------------------------------------------ r_max

// Every node's centre as double-float words: zh = (hi(Z), 0), zl = (lo(Z), max_i |hi(Z_i)|);
// rmax_k fills zh.w with r_max rounded up.  The walk's binary32 acceptance prefilter, the binary32 M2L
// separations and the r_max prefilter below read these.
__global__ void centre_words_k(int nn, const double* __restrict__ Zx, const double* __restrict__ Zy,
                               const double* __restrict__ Zz, float4* __restrict__ zh, float4* __restrict__ zl) {
    int nd = blockIdx.x * TB + threadIdx.x;
    if (nd >= nn) return;
    double z[3] = {Zx[nd], Zy[nd], Zz[nd]};
    float h[3], l[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        h[i] = (float)z[i];
        l[i] = (float)(z[i] - (double)h[i]);
    }
    zh[nd] = make_float4(h[0], h[1], h[2], 0.f);
    zl[nd] = make_float4(l[0], l[1], l[2], fmaxf(fmaxf(fabsf(h[0]), fabsf(h[1])), fabsf(h[2])));
}

// r_max^2 = max over the node's particles of |X - Z|^2 for every node, exact in binary64
// (A11), in two passes over (particle, level); a particle's node at each level comes from
// the parent chain of its leaf, deepest level first.  Equal nodes are contiguous in sorted order,
// so a segmented warp maximum leaves one integer atomicMax per node and warp (on the bit
// pattern of a non-negative number, which orders like the value); max is order
// independent, so the result is bit exact.
//  * Pass 1 (binary32): |X - Z|^2 from the double-float words of X and Z, (hi - hi) +
//    (lo - lo) per axis; its relative error is below 2^-20 while r_max >= 2^-20 |Z| and
//    nothing under- or overflows.  The node's maximum m goes to r2f.
//  * Pass 2: a particle whose binary32 estimate is within 2^-16 of m, or of a node outside
//    that range, forms |X - Z|^2 in binary64 (the formula of the oracle) for the exact max.
//    The binary64 work falls from every (particle, level) to the few near the maximum.
__device__ __forceinline__ void split_df(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

__device__ __forceinline__ float d2_words(float xh, float xl, float yh, float yl, float zh_, float zl_, float4 ch,
                                          float4 cl) {
    float dx = __fadd_rn(__fsub_rn(xh, ch.x), __fsub_rn(xl, cl.x));
    float dy = __fadd_rn(__fsub_rn(yh, ch.y), __fsub_rn(yl, cl.y));
    float dz = __fadd_rn(__fsub_rn(zh_, ch.z), __fsub_rn(zl_, cl.z));
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__global__ void rmax2f_k(int n, int nlev, const int* __restrict__ leaf_of, const int* __restrict__ nlevel,
                         const int* __restrict__ nparent, const double* __restrict__ xs,
                         const double* __restrict__ ys, const double* __restrict__ zs, const float4* __restrict__ zh,
                         const float4* __restrict__ zl, unsigned* __restrict__ r2f) {
    int i = blockIdx.x * TB + threadIdx.x;
    int lane = threadIdx.x & 31;
    bool in = i < n;
    float xh = 0.f, xl = 0.f, yh = 0.f, yl = 0.f, zh_ = 0.f, zl_ = 0.f;
    int up = -1, dl = -1;  // the particle's ancestor at the current level, and its leaf's level
    if (in) {
        split_df(xs[i], xh, xl);
        split_df(ys[i], yh, yl);
        split_df(zs[i], zh_, zl_);
        up = leaf_of[i];
        dl = nlevel[up];
    }
    for (int l = nlev - 1; l >= 0; l--) {
        int nd = l <= dl ? up : -1;
        if (nd >= 0 && l > 0) up = nparent[nd];
        unsigned v = 0u;
        if (nd >= 0) v = __float_as_uint(d2_words(xh, xl, yh, yl, zh_, zl_, zh[nd], zl[nd]));
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            unsigned u = __shfl_down_sync(FULL, v, off);
            int no = __shfl_down_sync(FULL, nd, off);
            if (lane + off < 32 && no == nd && u > v) v = u;
        }
        int prev = __shfl_up_sync(FULL, nd, 1);
        bool head = (lane == 0) || (prev != nd);
        if (head && nd >= 0 && v != 0u) atomicMax(&r2f[nd], v);
    }
}

__global__ void rmax2_k(int n, int nlev, const int* __restrict__ leaf_of, const int* __restrict__ nlevel,
                        const int* __restrict__ nparent, const double* __restrict__ xs,
                        const double* __restrict__ ys, const double* __restrict__ zs,
                        const double* __restrict__ Zx, const double* __restrict__ Zy,
                        const double* __restrict__ Zz, const float4* __restrict__ zh, const float4* __restrict__ zl,
                        const unsigned* __restrict__ r2f, unsigned long long* __restrict__ r2bits) {
    int i = blockIdx.x * TB + threadIdx.x;
    int lane = threadIdx.x & 31;
    bool in = i < n;
    double px = in ? xs[i] : 0.0, py = in ? ys[i] : 0.0, pz = in ? zs[i] : 0.0;
    float xh = 0.f, xl = 0.f, yh = 0.f, yl = 0.f, zh_ = 0.f, zl_ = 0.f;
    int up = -1, dl = -1;
    if (in) {
        split_df(px, xh, xl);
        split_df(py, yh, yl);
        split_df(pz, zh_, zl_);
        up = leaf_of[i];
        dl = nlevel[up];
    }
    for (int l = nlev - 1; l >= 0; l--) {
        int nd = l <= dl ? up : -1;
        if (nd >= 0 && l > 0) up = nparent[nd];
        unsigned long long v = 0ull;
        if (nd >= 0) {
            float4 ch = zh[nd], cl = zl[nd];
            float m = __uint_as_float(r2f[nd]);
            float z2 = ch.x * ch.x + ch.y * ch.y + ch.z * ch.z;
            bool ranged = m >= 0x1p-100f && m <= 0x1p100f && m >= 0x1p-40f * z2;
            bool cand = !ranged || d2_words(xh, xl, yh, yl, zh_, zl_, ch, cl) >= m * (1.f - 0x1p-16f);
            if (cand) {
                double dx = __dsub_rn(px, Zx[nd]);
                double dy = __dsub_rn(py, Zy[nd]);
                double dz = __dsub_rn(pz, Zz[nd]);
                double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                v = (unsigned long long)__double_as_longlong(d2);
            }
        }
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            unsigned long long u = __shfl_down_sync(FULL, v, off);
            int no = __shfl_down_sync(FULL, nd, off);
            if (lane + off < 32 && no == nd && u > v) v = u;
        }
        int prev = __shfl_up_sync(FULL, nd, 1);
        bool head = (lane == 0) || (prev != nd);
        if (head && nd >= 0 && v != 0ull) atomicMax(&r2bits[nd], v);
    }
}

// r_max from its square; zh.w = r_max rounded up to binary32 (the centre words are set)
__global__ void rmax_k(int nn, const unsigned long long* __restrict__ r2bits, double* __restrict__ rmax,
                       float4* __restrict__ zh) {
    int nd = blockIdx.x * TB + threadIdx.x;
    if (nd >= nn) return;
    double r = __dsqrt_rn(__longlong_as_double((long long)r2bits[nd]));
    rmax[nd] = r;
    zh[nd].w = __double2float_ru(r);
}

// ------------------------------------------------------------------ batches of systems
// A batch is a forest: every system keeps its own bounding cube and keys (as if it were
// built alone), particles are ordered by (system, key), and system s owns root node s.

__device__ __forceinline__ int system_of(const long long* __restrict__ off, int nsys, int64_t i) {
    int lo = 0, hi = nsys;  // off[lo] <= i < off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= i)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// one block per system: cube [lo(3), side, scale] into geom[8 s ..] and input validation
__global__ void bbox_sys_k(const double* __restrict__ x, const double* __restrict__ m,
                           const long long* __restrict__ off, double* __restrict__ geom, int* __restrict__ bad) {
    __shared__ double smn[3][TB], smx[3][TB];
    int sys = blockIdx.x;
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    int b = 0;
    for (int64_t i = off[sys] + threadIdx.x; i < off[sys + 1]; i += TB) {
        for (int d = 0; d < 3; d++) {
            double v = x[3 * i + d];
            if (!isfinite(v)) b = 1;
            mn[d] = fmin(mn[d], v);
            mx[d] = fmax(mx[d], v);
        }
        double mm = m[i];
        if (!(mm >= 0.0) || !isfinite(mm)) b = 1;
    }
    if (b) atomicOr(bad, 1);
    for (int d = 0; d < 3; d++) {
        smn[d][threadIdx.x] = mn[d];
        smx[d][threadIdx.x] = mx[d];
    }
    __syncthreads();
    for (int st = TB / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            for (int d = 0; d < 3; d++) {
                smn[d][threadIdx.x] = fmin(smn[d][threadIdx.x], smn[d][threadIdx.x + st]);
                smx[d][threadIdx.x] = fmax(smx[d][threadIdx.x], smx[d][threadIdx.x + st]);
            }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    double side = 0.0;
    for (int d = 0; d < 3; d++) {
        geom[8 * sys + d] = smn[d][0];
        double e = __dsub_rn(smx[d][0], smn[d][0]);
        if (e > side) side = e;
    }
    if (side == 0.0) side = 1.0;
    geom[8 * sys + 3] = side;
    geom[8 * sys + 4] = __ddiv_rn(2097152.0, side);
}

__global__ void keys_sys_k(const double* __restrict__ x, int64_t n, const long long* __restrict__ off, int nsys,
                           const double* __restrict__ geom, uint64_t* __restrict__ keys, uint32_t* __restrict__ idx) {
    int64_t i = (int64_t)blockIdx.x * TB + threadIdx.x;
    if (i >= n) return;
    const double* g = geom + 8 * system_of(off, nsys, i);
    uint64_t qx = quantise(x[3 * i], g[0], g[4]);
    uint64_t qy = quantise(x[3 * i + 1], g[1], g[4]);
    uint64_t qz = quantise(x[3 * i + 2], g[2], g[4]);
    keys[i] = (spread_bits3(qx) << 2) | (spread_bits3(qy) << 1) | spread_bits3(qz);
    idx[i] = (uint32_t)i;
}

// after the key sort: the system of every sorted particle, with its position as payload
__global__ void sys_keys_k(const uint32_t* __restrict__ perm, int64_t n, const long long* __restrict__ off, int nsys,
                           uint64_t* __restrict__ sk, uint32_t* __restrict__ pos) {
    int64_t i = (int64_t)blockIdx.x * TB + threadIdx.x;
    if (i >= n) return;
    sk[i] = (uint64_t)system_of(off, nsys, perm[i]);
    pos[i] = (uint32_t)i;
}

// reorder keys and permutation by q (sorted by system, stable in key order)
__global__ void regather_k(const uint32_t* __restrict__ q, int64_t n, const uint64_t* __restrict__ kin,
                           const uint32_t* __restrict__ pin, uint64_t* __restrict__ kout, uint32_t* __restrict__ pout) {
    int64_t i = (int64_t)blockIdx.x * TB + threadIdx.x;
    if (i >= n) return;
    uint32_t j = q[i];
    kout[i] = kin[j];
    pout[i] = pin[j];
}

__global__ void roots_k(const long long* __restrict__ off, int nsys, int* nfirst, int* ncount, int* nlevel,
                        int* nparent, int* nchildf, int* nnchild) {
    int sys = blockIdx.x * TB + threadIdx.x;
    if (sys >= nsys) return;
    nfirst[sys] = (int)off[sys];
    ncount[sys] = (int)(off[sys + 1] - off[sys]);
    nlevel[sys] = 0;
    nparent[sys] = -1;
    nchildf[sys] = -1;
    nnchild[sys] = 0;
}

// ------------------------------------------------------------------ host driver

// Per-leaf work (P2M) runs one thread per leaf, so a warp lasts as long as its largest
// leaf.  Nodes ordered by this key (leaf size, capped at 510; inner nodes 511, last) give
// warps leaves of equal size.
__global__ void leaf_key_k(int nn, const int* __restrict__ ncount, const int* __restrict__ nnchild,
                           uint32_t* __restrict__ key, uint32_t* __restrict__ order) {
    int nd = blockIdx.x * TB + threadIdx.x;
    if (nd >= nn) return;
    key[nd] = nnchild[nd] != 0 ? 511u : (uint32_t)min(ncount[nd], 510);
    order[nd] = (uint32_t)nd;
}

static void ensure_nodes(fmm_ctx* c, int64_t need) {
    if (need <= c->cap_nodes) return;
    int64_t cap = need + need / 2 + 1024;
    size_t b = sizeof(int) * (size_t)cap;
    ensure_keep(c->nfirst, b, c->stream);
    ensure_keep(c->ncount, b, c->stream);
    ensure_keep(c->nlevel, b, c->stream);
    ensure_keep(c->nparent, b, c->stream);
    ensure_keep(c->nchildf, b, c->stream);
    ensure_keep(c->nnchild, b, c->stream);
    c->cap_nodes = cap;
}

int build_tree(fmm_ctx* c, const double* x, const double* m) {
    cudaStream_t s = c->stream;
    int n = (int)c->N;
    int nsys = c->n_sys;
    const long long* off = c->sys_off.as<long long>();
    // a1: bounding cube(s) and validation
    int nb = (int)((c->N + TB - 1) / TB);
    if (nb > 1024) nb = 1024;
    ensure(c->geom, sizeof(double) * (size_t)(8 * nsys + 6 * nb));
    ensure(c->errflag, sizeof(int) * 4);
    double* geom = c->geom.as<double>();
    double* part = geom + 8 * nsys;
    GB_CUDA(cudaMemsetAsync(c->errflag.p, 0, sizeof(int) * 4, s));
    if (nsys == 1) {
        bbox_partial_k<<<nb, TB, 0, s>>>(x, m, c->N, part, c->errflag.as<int>());
        GB_LAUNCH("bbox_partial_k");
        bbox_final_k<<<1, BFB, 0, s>>>(part, nb, geom);
        GB_LAUNCH("bbox_final_k");
    } else {
        bbox_sys_k<<<nsys, TB, 0, s>>>(x, m, off, geom, c->errflag.as<int>());
        GB_LAUNCH("bbox_sys_k");
    }
    // (the input check is read with the level table below: every step of the build is
    // index-safe on any values, so invalid input costs one build and returns FMM_ERR_INVALID)
    // a2: keys; a3: sort
    ensure(c->keys0, sizeof(uint64_t) * (size_t)n);
    ensure(c->vals0, sizeof(uint32_t) * (size_t)n);
    if (nsys == 1)
        keys_k<<<grid_for(n, TB), TB, 0, s>>>(x, n, geom, c->keys0.as<uint64_t>(), c->vals0.as<uint32_t>());
    else
        keys_sys_k<<<grid_for(n, TB), TB, 0, s>>>(x, n, off, nsys, geom, c->keys0.as<uint64_t>(),
                                                  c->vals0.as<uint32_t>());
    GB_LAUNCH("keys_k");
    radix_sort(c, c->keys0, c->keys1, &c->vals0, &c->vals1, n, 63);
    ensure(c->perm, sizeof(uint32_t) * (size_t)n);
    if (nsys == 1) {
        GB_CUDA(cudaMemcpyAsync(c->perm.p, c->vals0.p, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    } else {
        // stable sort by system on top of the key order: (system, key) order
        ensure(c->sys_k, sizeof(uint64_t) * (size_t)n);
        ensure(c->sys_v, sizeof(uint32_t) * (size_t)n);
        sys_keys_k<<<grid_for(n, TB), TB, 0, s>>>(c->vals0.as<uint32_t>(), n, off, nsys, c->sys_k.as<uint64_t>(),
                                                  c->sys_v.as<uint32_t>());
        GB_LAUNCH("sys_keys_k");
        int sbits = 1;
        while ((1 << sbits) < nsys) sbits++;
        radix_sort(c, c->sys_k, c->keys1, &c->sys_v, &c->vals1, n, sbits);
        regather_k<<<grid_for(n, TB), TB, 0, s>>>(c->sys_v.as<uint32_t>(), n, c->keys0.as<uint64_t>(),
                                                  c->vals0.as<uint32_t>(), c->keys1.as<uint64_t>(),
                                                  c->perm.as<uint32_t>());
        GB_LAUNCH("regather_k");
        GB_CUDA(cudaMemcpyAsync(c->keys0.p, c->keys1.p, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    }
    ensure(c->xs, sizeof(double) * (size_t)n);
    ensure(c->ys, sizeof(double) * (size_t)n);
    ensure(c->zs, sizeof(double) * (size_t)n);
    ensure(c->ms, sizeof(double) * (size_t)n);
    gather_k<<<grid_for(n, TB), TB, 0, s>>>(x, m, c->perm.as<uint32_t>(), n, c->xs.as<double>(),
                                            c->ys.as<double>(), c->zs.as<double>(), c->ms.as<double>());
    GB_LAUNCH("gather_k");
    // a4: octree, level by level (breadth-first ids)
    const uint64_t* keys = c->keys0.as<uint64_t>();
    ensure_nodes(c, (int64_t)n / 4 + 64);
    ensure(c->leaf_of, sizeof(int) * (size_t)n);
    ensure_nodes(c, (int64_t)nsys + 64);
    roots_k<<<grid_for(nsys, TB), TB, 0, s>>>(off, nsys, c->nfirst.as<int>(), c->ncount.as<int>(), c->nlevel.as<int>(),
                                              c->nparent.as<int>(), c->nchildf.as<int>(), c->nnchild.as<int>());
    GB_LAUNCH("roots_k");
    // levels 1 .. MAX_LEVEL in one cooperative launch (split_levels_k), bounds and counts on
    // the device, one read of the level table (and of the input check) at the end; a tree
    // that outgrows the node arrays is built again with arrays of the size it reported
    int dev_sms = 0;
    GB_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c->device));
    ensure(c->lvl_ctl, sizeof(LevelCtl));
    LevelCtl* ctl = c->lvl_ctl.as<LevelCtl>();
    LevelCtl h;
    int bad = 0;
    int64_t n_nodes = nsys;
    for (int attempt = 0;; attempt++) {
        int cap = (int)std::min<int64_t>(c->cap_nodes, INT32_MAX);
        size_t nstat = (size_t)cap / LV_NODES + 2;
        ensure(c->lvl_status, sizeof(unsigned long long) * nstat);
        memset(&h, 0, sizeof(h));
        h.start[1] = nsys;
        GB_CUDA(cudaMemcpyAsync(ctl, &h, sizeof(LevelCtl), cudaMemcpyHostToDevice, s));
        GB_CUDA(cudaMemsetAsync(c->lvl_status.p, 0, sizeof(unsigned long long) * nstat, s));
        {
            int per_sm = 0;
            GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, split_levels_k, TB, 0));
            dim3 grid((unsigned)(dev_sms * std::max(1, std::min(per_sm, 4)))), block(TB);
            const uint64_t* k_ = keys;
            int leaf_ = c->leaf;
            unsigned long long* st_ = c->lvl_status.as<unsigned long long>();
            int *nf = c->nfirst.as<int>(), *ncnt = c->ncount.as<int>(), *nlv = c->nlevel.as<int>();
            int *npar = c->nparent.as<int>(), *ncf = c->nchildf.as<int>(), *nnc = c->nnchild.as<int>();
            void* args[] = {(void*)&k_, (void*)&leaf_, (void*)&cap, (void*)&ctl, (void*)&st_, (void*)&nf,
                            (void*)&ncnt, (void*)&nlv, (void*)&npar, (void*)&ncf, (void*)&nnc};
            GB_CUDA(cudaLaunchCooperativeKernel((const void*)split_levels_k, grid, block, args, 0, s));
            GB_LAUNCH("split_levels_k");
        }
        int serr = 0;
        {
            HostReads hr(c);
            LevelCtl* hh = hr.read<LevelCtl>(ctl);
            int* hbad = hr.read<int>(c->errflag.p);
            int* hserr = hr.read<int>(sort_err(c));
            hr.wait();
            h = *hh;
            bad = *hbad;
            serr = *hserr;
        }
        if (bad) return FMM_ERR_INVALID;
        sort_err_throw(c, serr);
        if (h.err) throw FmmError{FMM_ERR_TIMEOUT, "octree: a level tile waited too long for the tiles before it"};
        if (!h.overflow) break;
        // the levels that were built report their sizes: grow past the last one and retry
        int64_t known = nsys;
        for (int L = 1; L <= MAX_LEVEL + 1 && h.start[L] >= h.start[L - 1]; L++) known = std::max<int64_t>(known, h.start[L]);
        if (attempt >= 8) throw FmmError{FMM_ERR_CAPACITY, "octree: node arrays still too small after 8 retries"};
        ensure_nodes(c, std::max<int64_t>(2 * c->cap_nodes, known + known / 2));
        roots_k<<<grid_for(nsys, TB), TB, 0, s>>>(off, nsys, c->nfirst.as<int>(), c->ncount.as<int>(),
                                                  c->nlevel.as<int>(), c->nparent.as<int>(), c->nchildf.as<int>(),
                                                  c->nnchild.as<int>());
        GB_LAUNCH("roots_k");
    }
    c->level_start.assign(1, 0);
    c->level_start.push_back(nsys);
    for (int L = 2; L <= MAX_LEVEL + 1 && h.start[L] > h.start[L - 1]; L++) c->level_start.push_back(h.start[L]);
    n_nodes = c->level_start.back();
    leaf_of_k<<<grid_for(n_nodes, TB), TB, 0, s>>>((int)n_nodes, c->nfirst.as<int>(), c->ncount.as<int>(),
                                                   c->nnchild.as<int>(), c->leaf_of.as<int>());
    GB_LAUNCH("leaf_of_k");
    c->n_levels = (int)c->level_start.size() - 1;
    c->n_nodes = n_nodes;
    // centres of mass, bottom-up
    int nn = (int)n_nodes;
    size_t db = sizeof(double) * (size_t)nn;
    for (DevBuf* b : {&c->nM, &c->nSx, &c->nSy, &c->nSz, &c->nZx, &c->nZy, &c->nZz, &c->nrmax}) ensure(*b, db);
    ensure(c->nr2, sizeof(unsigned long long) * (size_t)nn);
    com_leaf_k<<<grid_for(nn, TB), TB, 0, s>>>(nn, c->nfirst.as<int>(), c->ncount.as<int>(), c->nnchild.as<int>(),
                                               c->xs.as<double>(), c->ys.as<double>(), c->zs.as<double>(),
                                               c->ms.as<double>(), c->nM.as<double>(), c->nSx.as<double>(),
                                               c->nSy.as<double>(), c->nSz.as<double>(), c->nZx.as<double>(),
                                               c->nZy.as<double>(), c->nZz.as<double>());
    GB_LAUNCH("com_leaf_k");
    for (int l = c->n_levels - 2; l >= 0; l--) {
        int lo = c->level_start[l], hi = c->level_start[l + 1];
        com_inner_k<<<grid_for(hi - lo, TB), TB, 0, s>>>(lo, hi, c->nfirst.as<int>(), c->nchildf.as<int>(),
                                                         c->nnchild.as<int>(), c->xs.as<double>(),
                                                         c->ys.as<double>(), c->zs.as<double>(), c->nM.as<double>(),
                                                         c->nSx.as<double>(), c->nSy.as<double>(),
                                                         c->nSz.as<double>(), c->nZx.as<double>(),
                                                         c->nZy.as<double>(), c->nZz.as<double>());
        GB_LAUNCH("com_inner_k");
    }
    // r_max: binary32 prefilter, then binary64 for the particles near each node's maximum
    ensure(c->zhl, sizeof(float4) * 2 * (size_t)nn);
    float4* zh = c->zhl.as<float4>();
    float4* zl = zh + nn;
    centre_words_k<<<grid_for(nn, TB), TB, 0, s>>>(nn, c->nZx.as<double>(), c->nZy.as<double>(), c->nZz.as<double>(),
                                                   zh, zl);
    GB_LAUNCH("centre_words_k");
    ensure(c->nr2f, sizeof(unsigned) * (size_t)nn);
    GB_CUDA(cudaMemsetAsync(c->nr2f.p, 0, sizeof(unsigned) * (size_t)nn, s));
    GB_CUDA(cudaMemsetAsync(c->nr2.p, 0, sizeof(unsigned long long) * (size_t)nn, s));
    rmax2f_k<<<grid_for(n, TB), TB, 0, s>>>(n, c->n_levels, c->leaf_of.as<int>(), c->nlevel.as<int>(),
                                            c->nparent.as<int>(), c->xs.as<double>(), c->ys.as<double>(),
                                            c->zs.as<double>(), zh, zl, c->nr2f.as<unsigned>());
    GB_LAUNCH("rmax2f_k");
    rmax2_k<<<grid_for(n, TB), TB, 0, s>>>(n, c->n_levels, c->leaf_of.as<int>(), c->nlevel.as<int>(),
                                           c->nparent.as<int>(), c->xs.as<double>(), c->ys.as<double>(),
                                           c->zs.as<double>(), c->nZx.as<double>(), c->nZy.as<double>(),
                                           c->nZz.as<double>(), zh, zl, c->nr2f.as<unsigned>(),
                                           c->nr2.as<unsigned long long>());
    GB_LAUNCH("rmax2_k");
    rmax_k<<<grid_for(nn, TB), TB, 0, s>>>(nn, c->nr2.as<unsigned long long>(), c->nrmax.as<double>(), zh);
    GB_LAUNCH("rmax_k");
    // nodes by leaf size for the per-leaf kernels (one stable 9-bit radix pass)
    ensure(c->leaf_key, sizeof(uint32_t) * (size_t)nn);
    ensure(c->leaf_order, sizeof(uint32_t) * (size_t)nn);
    leaf_key_k<<<grid_for(nn, TB), TB, 0, s>>>(nn, c->ncount.as<int>(), c->nnchild.as<int>(),
                                               c->leaf_key.as<uint32_t>(), c->leaf_order.as<uint32_t>());
    GB_LAUNCH("leaf_key_k");
    radix_sort32(c, c->leaf_key, c->leaf_key2, &c->leaf_order, &c->leaf_order2, nn, 9);
    return FMM_OK;
}

}  // namespace gbfmm
