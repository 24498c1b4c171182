// Mutual dual-tree walk (Sec. 2: well-separated node pairs by eq. mac_criterion,
// Dehnen-style mutual interactions) as a level-synchronous frontier of cell pairs.
//
//   Self(A): A leaf -> P2P(A, A); else over its children c_i, c_j with i <= j:
//            Self(c_i) if i == j, Pair(c_i, c_j) otherwise.
//   Pair(A, B): R = |Z_A - Z_B| > 0 and r_A + r_B <= theta R  -> M2L(A, B)
//               both leaves                                    -> P2P(A, B)
//               otherwise split A or B into its children: a leaf is never split; between
//               two inner nodes the larger r_max is split, ties -> larger count, then
//               lower id.
// The rule is symmetric in (A, B), so the emitted pair set is unique.  The lists are then
// expanded into directed entries (target, source) and radix-sorted: every cell sees its
// partners in increasing id order, which is also the canonical (min id, max id) order,
// and every later sum runs in that order.  The order in which a frontier step emits its
// outputs therefore cannot change any result, so one kernel per step claims output
// slots with block-aggregated integer atomics, and the host launches a fixed number of
// steps (2 x levels + 2 bounds the recursion depth) without waiting between them.  The
// counters keep counting past the buffers' capacity; one read at the end detects an
// overflow and the walk is run again with buffers of the reported sizes.
#include <algorithm>
#include <vector>

#include "fmm_device.cuh"
#include "fmm_internal.h"

namespace gbfmm {

constexpr int WB = 256;

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

struct WalkCounters {
    int nf[2];       // frontier sizes (read by the step of that parity, appended by the other)
    int n_m2l, n_p2p;
};

// One frontier step.  A block takes WB * WIPT frontier items per round (WIPT per thread),
// decides them, forms every thread's output offsets with one block scan and claims the
// block's output ranges with one atomic per counter, then writes.  Claiming per warp put
// three same-address atomics on every 32 items and made the step contention-bound.
constexpr int WIPT = 4;

__global__ void __launch_bounds__(WB) walk_step_k(const int2* __restrict__ fr_in, int2* __restrict__ fr_out,
                                                  WalkCounters* __restrict__ cnt, int par, NodeView nv, double theta,
                                                  float th2, int2* __restrict__ m2l, int cap_m2l,
                                                  int2* __restrict__ p2p, int cap_p2p, int cap_fr) {
    __shared__ int sbase[3];
    int nf = min(cnt->nf[par], cap_fr);  // a frontier beyond the buffer was not stored (retried)
    for (int64_t base = (int64_t)blockIdx.x * WB * WIPT; base < nf; base += (int64_t)gridDim.x * WB * WIPT) {
        int2 it[WIPT];
        int d[WIPT], nnew[WIPT];
        bool sa[WIPT];
        Cnt3 mine{0, 0, 0};
#pragma unroll
        for (int j = 0; j < WIPT; j++) {
            int64_t i = base + (int64_t)j * WB + threadIdx.x;
            d[j] = -1;
            nnew[j] = 0;
            sa[j] = false;
            it[j] = make_int2(0, 0);
            if (i < nf) {
                it[j] = fr_in[i];
                d[j] = decide(nv, it[j], theta, th2, &nnew[j], &sa[j]);
            }
            mine.a += d[j] == 1;
            mine.b += d[j] == 2;
            mine.c += d[j] == 0 ? nnew[j] : 0;
        }
        Cnt3 tot;
        Cnt3 off = block_exclusive_scan(mine, &tot);
        if (threadIdx.x == 0) {
            sbase[0] = tot.a ? atomicAdd(&cnt->n_m2l, tot.a) : 0;
            sbase[1] = tot.b ? atomicAdd(&cnt->n_p2p, tot.b) : 0;
            sbase[2] = tot.c ? atomicAdd(&cnt->nf[par ^ 1], tot.c) : 0;
        }
        __syncthreads();
        int om = sbase[0] + off.a, op = sbase[1] + off.b, of = sbase[2] + off.c;
#pragma unroll
        for (int j = 0; j < WIPT; j++) {
            if (d[j] == 1) {
                if (om < cap_m2l) m2l[om] = it[j];
                om++;
            } else if (d[j] == 2) {
                if (op < cap_p2p) p2p[op] = it[j];
                op++;
            } else if (d[j] == 0) {
                if (it[j].x == it[j].y) {
                    int c0 = nv.child_first[it[j].x], nc = nv.nchild[it[j].x];
                    int k = of;
                    for (int a = 0; a < nc; a++)
                        for (int b = a; b < nc; b++, k++)
                            if (k < cap_fr) fr_out[k] = make_int2(c0 + a, c0 + b);
                } else {
                    int S = sa[j] ? it[j].x : it[j].y;
                    int c0 = nv.child_first[S], nc = nv.nchild[S];
                    for (int a = 0; a < nc; a++)
                        if (of + a < cap_fr)
                            fr_out[of + a] = sa[j] ? make_int2(c0 + a, it[j].y) : make_int2(it[j].x, c0 + a);
                }
                of += nnew[j];
            }
        }
        __syncthreads();  // sbase is reused by the next round
    }
}

// prepares the next step: its input count is this step's output, its output starts at 0;
// frontier overflow is recorded in *over (the largest frontier seen)
__global__ void walk_advance_k(WalkCounters* cnt, int par, int* max_fr) {
    int nxt = cnt->nf[par ^ 1];
    if (nxt > *max_fr) *max_fr = nxt;
    cnt->nf[par] = 0;
}

// the walk starts with Self(root) of every system of the batch (roots are nodes 0..nsys-1)
__global__ void walk_init_k(WalkCounters* cnt, int2* fr0, int* max_fr, int nsys) {
    int sys = blockIdx.x * WB + threadIdx.x;
    if (sys < nsys) fr0[sys] = make_int2(sys, sys);
    if (sys == 0) {
        cnt->nf[0] = nsys;
        cnt->nf[1] = 0;
        cnt->n_m2l = 0;
        cnt->n_p2p = 0;
        *max_fr = nsys;
    }
}

// ---- per-target segments of the directed lists
// Every mutual pair (A, B) gives a directed entry for target A (partner B) and, unless
// A == B, one for target B (partner A).  Entries are counted per target (integer atomics),
// the counts scanned into segment starts, the entries scattered into their target's
// segment in any order, and every segment then sorted by its key, which starts with the
// partner id: each cell sees its partners in increasing id, the canonical order, whatever
// order the walk and the scatter produced.  The key is the partner (M2L) or
// partner << 32 | (pair << 1 | side) (P2P); the low 32 bits are kept.

__global__ void seg_count_k(const int2* __restrict__ pairs, int64_t n, int* __restrict__ cnt) {
    int64_t k = (int64_t)blockIdx.x * WB + threadIdx.x;
    if (k >= n) return;
    int2 p = pairs[k];
    atomicAdd(&cnt[p.x], 1);
    if (p.x != p.y) atomicAdd(&cnt[p.y], 1);
}

__global__ void seg_scatter_k(const int2* __restrict__ pairs, int64_t n, bool payload,
                              const long long* __restrict__ seg, int* __restrict__ cur,
                              uint64_t* __restrict__ keys) {
    int64_t k = (int64_t)blockIdx.x * WB + threadIdx.x;
    if (k >= n) return;
    int2 p = pairs[k];
    uint64_t ka = payload ? ((uint64_t)(uint32_t)p.y << 32) | (uint64_t)(uint32_t)(2 * k) : (uint64_t)(uint32_t)p.y;
    keys[seg[p.x] + atomicAdd(&cur[p.x], 1)] = ka;
    if (p.x != p.y) {
        uint64_t kb = payload ? ((uint64_t)(uint32_t)p.x << 32) | (uint64_t)(uint32_t)(2 * k + 1)
                              : (uint64_t)(uint32_t)p.x;
        keys[seg[p.y] + atomicAdd(&cur[p.y], 1)] = kb;
    }
}

// partial slots of every P2P pair: nA + nB (a self pair: nA)
__global__ void p2p_psize_k(const int2* __restrict__ pairs, int64_t n, const int* __restrict__ count,
                            long long* __restrict__ psize) {
    int64_t k = (int64_t)blockIdx.x * WB + threadIdx.x;
    if (k >= n) return;
    int2 p = pairs[k];
    psize[k] = p.x != p.y ? (long long)count[p.x] + count[p.y] : (long long)count[p.x];
}

// Segments of at most 256 entries (most): one warp per segment, a bitonic network on
// NR = 1, 2, 4 or 8 registers per lane (wider register networks measured slower than the
// shared-memory sort below).  Element e = r * 32 + lane sits in register r of
// the lane; a compare-exchange at distance j < 32 is a shuffle, at j >= 32 a register swap.
// Padding is the largest key, so it sorts to the end.
template <int NR>
__device__ __forceinline__ void warp_bitonic(uint64_t (&v)[NR], int lane) {
    constexpr int P2 = 32 * NR;
#pragma unroll
    for (int k = 2; k <= P2; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                int jr = j >> 5;
#pragma unroll
                for (int r = 0; r < NR; r++) {
                    int q = r ^ jr;
                    if (q > r) {
                        int e = r * 32 + lane;
                        bool up = (e & k) == 0;
                        uint64_t a = v[r], b = v[q];
                        bool sw = (a > b) == up;
                        v[r] = sw ? b : a;
                        v[q] = sw ? a : b;
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < NR; r++) {
                    int e = r * 32 + lane;
                    uint64_t o = __shfl_xor_sync(FULL, v[r], j);
                    bool lower = (lane & j) == 0;  // this lane holds the lower index of the pair
                    bool up = (e & k) == 0;
                    // the lower index keeps the min when ascending, the max when descending
                    bool keep_min = lower == up;
                    v[r] = keep_min ? (v[r] < o ? v[r] : o) : (v[r] < o ? o : v[r]);
                }
            }
        }
    }
}

template <int NR>
__device__ __forceinline__ void warp_sort_segment(const uint64_t* __restrict__ keys, uint32_t* __restrict__ out,
                                                  long long s0, int L, int lane) {
    uint64_t v[NR];
#pragma unroll
    for (int r = 0; r < NR; r++) {
        int e = r * 32 + lane;
        v[r] = e < L ? keys[s0 + e] : ~0ull;
    }
    warp_bitonic<NR>(v, lane);
#pragma unroll
    for (int r = 0; r < NR; r++) {
        int e = r * 32 + lane;
        if (e < L) out[s0 + e] = (uint32_t)v[r];
    }
}

constexpr int SS_WARP_MAX = 256, SS_MAX = 4096, SSB = 256;

__global__ void __launch_bounds__(SSB) seg_sort_warp_k(const long long* __restrict__ seg, int nn,
                                                       const uint64_t* __restrict__ keys, uint32_t* __restrict__ out,
                                                       int* __restrict__ mid, int* __restrict__ cnt2,
                                                       int* __restrict__ big) {
    int lane = threadIdx.x & 31;
    int64_t w0 = ((int64_t)blockIdx.x * SSB + threadIdx.x) >> 5, nw = ((int64_t)gridDim.x * SSB) >> 5;
    for (int64_t x = w0; x < nn; x += nw) {
        long long s0 = seg[x];
        int L = (int)(seg[x + 1] - s0);  // uniform over the warp
        if (L <= 1) {
            if (L == 1 && lane == 0) out[s0] = (uint32_t)keys[s0];
        } else if (L <= 32) {
            warp_sort_segment<1>(keys, out, s0, L, lane);
        } else if (L <= 64) {
            warp_sort_segment<2>(keys, out, s0, L, lane);
        } else if (L <= 128) {
            warp_sort_segment<4>(keys, out, s0, L, lane);
        } else if (L <= SS_WARP_MAX) {
            warp_sort_segment<8>(keys, out, s0, L, lane);
        } else if (lane == 0) {
            // longer segments are listed for the block sort or the long-segment fallback
            if (L <= SS_MAX)
                mid[atomicAdd(&cnt2[0], 1)] = (int)x;
            else
                big[atomicAdd(&cnt2[1], 1)] = (int)x;
        }
    }
}

// Segments of 257 .. SS_MAX entries, from the list seg_sort_warp_k made: one block per
// segment, bitonic sort in shared memory.
__global__ void __launch_bounds__(SSB) seg_sort_small_k(const long long* __restrict__ seg,
                                                        const uint64_t* __restrict__ keys, uint32_t* __restrict__ out,
                                                        const int* __restrict__ mid, const int* __restrict__ cnt2) {
    __shared__ uint64_t sk[SS_MAX];
    int nmid = cnt2[0];
    for (int i = blockIdx.x; i < nmid; i += gridDim.x) {
        int x = mid[i];
        long long s0 = seg[x];
        int L = (int)(seg[x + 1] - s0);
        int P2 = 2;
        while (P2 < L) P2 <<= 1;
        for (int j = threadIdx.x; j < P2; j += SSB) sk[j] = j < L ? keys[s0 + j] : ~0ull;
        __syncthreads();
        for (int k = 2; k <= P2; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int a = threadIdx.x; a < P2; a += SSB) {
                    int ixj = a ^ j;
                    if (ixj > a) {
                        uint64_t u = sk[a], v = sk[ixj];
                        if ((u > v) == ((a & k) == 0)) {
                            sk[a] = v;
                            sk[ixj] = u;
                        }
                    }
                }
                __syncthreads();
            }
        for (int j = threadIdx.x; j < L; j += SSB) out[s0 + j] = (uint32_t)sk[j];
        __syncthreads();
    }
}

// fallback for the rare long segments (sparse halo cells with thousands of partners):
// their entries are copied with the key (rank of the segment << bits | partner), radix
// sorted together, and the payloads written back
__global__ void big_gather_k(const int* __restrict__ big, const long long* __restrict__ boff,
                             const long long* __restrict__ seg, const uint64_t* __restrict__ keys, int bits,
                             bool payload, uint64_t* __restrict__ bkeys, uint32_t* __restrict__ bvals) {
    int b = blockIdx.x;
    int x = big[b];
    long long s0 = seg[x], L = seg[x + 1] - s0, o = boff[b];
    for (long long i = threadIdx.x; i < L; i += SSB) {
        uint64_t k = keys[s0 + i];
        uint64_t partner = payload ? (k >> 32) : k;
        bkeys[o + i] = ((uint64_t)b << bits) | partner;
        bvals[o + i] = (uint32_t)k;
    }
}

__global__ void big_scatter_k(const int* __restrict__ big, const long long* __restrict__ boff,
                              const long long* __restrict__ seg, const uint32_t* __restrict__ bvals,
                              uint32_t* __restrict__ out) {
    int b = blockIdx.x;
    int x = big[b];
    long long s0 = seg[x], L = seg[x + 1] - s0, o = boff[b];
    for (long long i = threadIdx.x; i < L; i += SSB) out[s0 + i] = bvals[o + i];
}

// builds seg[0..nn] and the sorted per-target lists out[] of the pairs[0..n)
static void build_segments(fmm_ctx* c, const int2* pairs, int64_t n, int nn, bool payload, DevBuf& seg_buf,
                           DevBuf& out_buf) {
    cudaStream_t s = c->stream;
    int bits = c->id_bits;
    ensure(seg_buf, sizeof(long long) * (size_t)(nn + 1));
    ensure(c->seg_cnt, sizeof(int) * (size_t)(2 * nn + 2));
    int* cnt = c->seg_cnt.as<int>();
    int* cur = cnt + nn + 1;
    GB_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)(2 * nn + 2), s));
    if (n > 0) {
        seg_count_k<<<grid_for(n, WB), WB, 0, s>>>(pairs, n, cnt);
        GB_LAUNCH("seg_count_k");
    }
    long long* seg = seg_buf.as<long long>();
    scan_i64(c, cnt, nn, seg);
    int64_t ne = 0;
    GB_CUDA(cudaMemcpyAsync(&ne, seg + nn, sizeof(long long), cudaMemcpyDeviceToHost, s));
    ensure(c->keys1, sizeof(uint64_t) * (size_t)(2 * n > 0 ? 2 * n : 1));
    ensure(out_buf, sizeof(uint32_t) * (size_t)(2 * n > 0 ? 2 * n : 1));
    ensure(c->cnt_off, sizeof(int) * 2);
    int* cnt2 = c->cnt_off.as<int>();  // [segments for the block sort, long segments]
    int* nbig_d = cnt2 + 1;
    GB_CUDA(cudaMemsetAsync(cnt2, 0, sizeof(int) * 2, s));
    uint64_t* keys = c->keys1.as<uint64_t>();
    if (n > 0) {
        seg_scatter_k<<<grid_for(n, WB), WB, 0, s>>>(pairs, n, payload, seg, cur, keys);
        GB_LAUNCH("seg_scatter_k");
    }
    ensure(c->flags, sizeof(int) * (size_t)(nn > 0 ? nn : 1));
    int* big = c->flags.as<int>();
    ensure(c->seg_mid, sizeof(int) * (size_t)(nn > 0 ? nn : 1));
    int* mid = c->seg_mid.as<int>();
    int dev_sms = 0;
    GB_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c->device));
    int g = std::min<int64_t>(nn, (int64_t)dev_sms * 8);
    if (g > 0) {
        seg_sort_warp_k<<<g, SSB, 0, s>>>(seg, nn, keys, out_buf.as<uint32_t>(), mid, cnt2, big);
        GB_LAUNCH("seg_sort_warp_k");
        seg_sort_small_k<<<g, SSB, 0, s>>>(seg, keys, out_buf.as<uint32_t>(), mid, cnt2);
        GB_LAUNCH("seg_sort_small_k");
    }
    int nbig = 0;
    GB_CUDA(cudaMemcpyAsync(&nbig, nbig_d, sizeof(int), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    if (nbig == 0) return;
    // the long segments, in a fixed order (by cell id), sorted together
    std::vector<int> bh(nbig);
    GB_CUDA(cudaMemcpy(bh.data(), big, sizeof(int) * nbig, cudaMemcpyDeviceToHost));
    std::sort(bh.begin(), bh.end());
    std::vector<long long> sh(2 * (size_t)nbig);
    for (int b = 0; b < nbig; b++) {
        GB_CUDA(cudaMemcpy(&sh[2 * b], seg + bh[b], sizeof(long long) * 2, cudaMemcpyDeviceToHost));
    }
    std::vector<long long> boff(nbig + 1, 0);
    for (int b = 0; b < nbig; b++) boff[b + 1] = boff[b] + (sh[2 * b + 1] - sh[2 * b]);
    int64_t tot = boff[nbig];
    GB_CUDA(cudaMemcpyAsync(big, bh.data(), sizeof(int) * nbig, cudaMemcpyHostToDevice, s));
    ensure(c->big_off, sizeof(long long) * (size_t)(nbig + 1));
    GB_CUDA(cudaMemcpyAsync(c->big_off.p, boff.data(), sizeof(long long) * (nbig + 1), cudaMemcpyHostToDevice, s));
    ensure(c->big_k, sizeof(uint64_t) * (size_t)tot);
    ensure(c->big_v, sizeof(uint32_t) * (size_t)tot);
    big_gather_k<<<nbig, SSB, 0, s>>>(big, c->big_off.as<long long>(), seg, keys, bits, payload,
                                      c->big_k.as<uint64_t>(), c->big_v.as<uint32_t>());
    GB_LAUNCH("big_gather_k");
    int bb = 1;
    while (((int64_t)1 << bb) <= nbig) bb++;
    radix_sort(c, c->big_k, c->big_k2, &c->big_v, &c->big_v2, tot, bits + bb);
    big_scatter_k<<<nbig, SSB, 0, s>>>(big, c->big_off.as<long long>(), seg, c->big_v.as<uint32_t>(),
                                       out_buf.as<uint32_t>());
    GB_LAUNCH("big_scatter_k");
    GB_CUDA(cudaStreamSynchronize(s));
}

// Work items over segments seg[0..n]: every segment is cut into chunks of CH entries.
// Full chunks come first (segment-major), then one partial chunk per segment that has a
// remainder, so that warps see chunks of equal length.  fo/po (n + 1 entries) give each
// segment's full-chunk range and partial-chunk rank.
__global__ void items_count_k(const long long* __restrict__ seg, int n, int CH, int* __restrict__ nfull,
                              int* __restrict__ npart) {
    int x = blockIdx.x * WB + threadIdx.x;
    if (x >= n) return;
    long long deg = seg[x + 1] - seg[x];
    nfull[x] = (int)(deg / CH);
    npart[x] = (deg % CH) != 0;
}

__global__ void items_fill_k(const long long* __restrict__ seg, int n, int CH, const long long* __restrict__ fo,
                             const long long* __restrict__ po, long long nfull_total, int4* __restrict__ items) {
    int x = blockIdx.x * WB + threadIdx.x;
    if (x >= n) return;
    long long e0 = seg[x], e1 = seg[x + 1];
    long long k0 = fo[x], nf = fo[x + 1] - k0;
    for (long long k = 0; k < nf; k++)
        items[k0 + k] = make_int4(x, (int)(e0 + k * CH), (int)(e0 + (k + 1) * CH), 0);
    if (po[x + 1] > po[x]) items[nfull_total + po[x]] = make_int4(x, (int)(e0 + nf * CH), (int)e1, 0);
}

void build_items(fmm_ctx* c, const long long* seg, int n, int CH, ItemSet& it) {
    cudaStream_t s = c->stream;
    ensure(c->seg_cnt, sizeof(int) * (size_t)(2 * n + 2));
    int* nfull = c->seg_cnt.as<int>();
    int* npart = nfull + n + 1;
    ensure(it.fo, sizeof(long long) * (size_t)(n + 1));
    ensure(it.po, sizeof(long long) * (size_t)(n + 1));
    items_count_k<<<grid_for(n, WB), WB, 0, s>>>(seg, n, CH, nfull, npart);
    GB_LAUNCH("items_count_k");
    scan_i64(c, nfull, n, it.fo.as<long long>());
    scan_i64(c, npart, n, it.po.as<long long>());
    long long tot[2];
    GB_CUDA(cudaMemcpyAsync(&tot[0], it.fo.as<long long>() + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaMemcpyAsync(&tot[1], it.po.as<long long>() + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    it.n_full = tot[0];
    it.n_items = tot[0] + tot[1];
    it.chunk = CH;
    ensure(it.items, sizeof(int4) * (size_t)(it.n_items > 0 ? it.n_items : 1));
    items_fill_k<<<grid_for(n, WB), WB, 0, s>>>(seg, n, CH, it.fo.as<long long>(), it.po.as<long long>(), it.n_full,
                                                it.items.as<int4>());
    GB_LAUNCH("items_fill_k");
}

static int bits_for(int64_t nn) {
    int b = 1;
    while (((int64_t)1 << b) <= nn) b++;  // ids < 2^b - 1 always
    return b;
}

void run_walk(fmm_ctx* c, double theta) {
    cudaStream_t s = c->stream;
    NodeView nv = node_view(c);
    int64_t nn = c->n_nodes;
    // fixed number of steps, no host round trip between them; one retry if a buffer overflowed
    int steps = 2 * c->n_levels + 2;
    float th2 = (float)theta * (float)theta;  // prefilter only; relative error far inside its margin
    int dev_sms = 0;
    GB_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c->device));
    int grid = dev_sms * 8;
    int64_t n_m2l = 0, n_p2p = 0;
    for (int attempt = 0;; attempt++) {
        int64_t cap_fr = c->cap_fr, cap_m2l = c->cap_m2l, cap_p2p = c->cap_p2p;
        ensure(c->fr0, sizeof(int2) * (size_t)cap_fr);
        ensure(c->fr1, sizeof(int2) * (size_t)cap_fr);
        ensure(c->m2l_pairs, sizeof(int2) * (size_t)cap_m2l);
        ensure(c->p2p_pairs, sizeof(int2) * (size_t)cap_p2p);
        ensure(c->cnt, sizeof(WalkCounters) + 16);
        WalkCounters* cnt = reinterpret_cast<WalkCounters*>(c->cnt.p);
        int* max_fr = reinterpret_cast<int*>(cnt + 1);
        walk_init_k<<<grid_for(c->n_sys, WB), WB, 0, s>>>(cnt, c->fr0.as<int2>(), max_fr, c->n_sys);
        GB_LAUNCH("walk_init_k");
        for (int k = 0; k < steps; k++) {
            int par = k & 1;
            int2* fin = par ? c->fr1.as<int2>() : c->fr0.as<int2>();
            int2* fout = par ? c->fr0.as<int2>() : c->fr1.as<int2>();
            walk_step_k<<<grid, WB, 0, s>>>(fin, fout, cnt, par, nv, theta, th2, c->m2l_pairs.as<int2>(), (int)cap_m2l,
                                            c->p2p_pairs.as<int2>(), (int)cap_p2p, (int)cap_fr);
            GB_LAUNCH("walk_step_k");
            walk_advance_k<<<1, 1, 0, s>>>(cnt, par, max_fr);
            GB_LAUNCH("walk_advance_k");
        }
        WalkCounters h;
        int hmax = 0;
        GB_CUDA(cudaMemcpyAsync(&h, cnt, sizeof(WalkCounters), cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaMemcpyAsync(&hmax, max_fr, sizeof(int), cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaStreamSynchronize(s));
        if (h.nf[0] != 0 || h.nf[1] != 0) throw FmmError{FMM_ERR_CAPACITY, "walk did not finish in 2 x levels + 2 steps"};
        bool over = h.n_m2l > cap_m2l || h.n_p2p > cap_p2p || hmax > cap_fr;
        if (h.n_m2l < 0 || h.n_p2p < 0 || hmax < 0) throw FmmError{FMM_ERR_CAPACITY, "walk counters above 2^31"};
        if (over) {
            // a truncated frontier under-reports what the later steps need: grow each
            // overflowing buffer to at least twice its size and try again
            if (attempt >= 10) throw FmmError{FMM_ERR_CAPACITY, "walk buffers still overflow after 10 retries"};
            if (h.n_m2l > cap_m2l) c->cap_m2l = std::max<int64_t>(2 * cap_m2l, (int64_t)h.n_m2l + h.n_m2l / 8);
            if (h.n_p2p > cap_p2p) c->cap_p2p = std::max<int64_t>(2 * cap_p2p, (int64_t)h.n_p2p + h.n_p2p / 8);
            if (hmax > cap_fr) c->cap_fr = std::max<int64_t>(2 * cap_fr, (int64_t)hmax + hmax / 8);
            c->walk_retries++;
            continue;
        }
        n_m2l = h.n_m2l;
        n_p2p = h.n_p2p;
        break;
    }
    c->n_m2l = n_m2l;
    c->n_p2p = n_p2p;
    int bits = bits_for(nn);
    c->id_bits = bits;
    // M2L: per-target segments of source ids in increasing order
    build_segments(c, c->m2l_pairs.as<int2>(), n_m2l, (int)nn, false, c->m2l_seg, c->m2l_dir);
    // P2P: per-target segments of (pair << 1 | side) in increasing partner order, plus the
    // partial offsets of every pair
    ensure(c->p2p_off, sizeof(long long) * (size_t)(n_p2p + 1));
    ensure(c->p2p_psize, sizeof(long long) * (size_t)(n_p2p + 1));
    if (n_p2p > 0) {
        p2p_psize_k<<<grid_for(n_p2p, WB), WB, 0, s>>>(c->p2p_pairs.as<int2>(), n_p2p, c->ncount.as<int>(),
                                                      c->p2p_psize.as<long long>());
        GB_LAUNCH("p2p_psize_k");
    }
    scan_i64_from_i64(c, c->p2p_psize.as<long long>(), n_p2p, c->p2p_off.as<long long>());
    build_segments(c, c->p2p_pairs.as<int2>(), n_p2p, (int)nn, true, c->p2p_seg, c->p2p_dval);
    // work items: m2l_chunk M2L sources (default 32) and p2p_chunk P2P entries (64) per chunk
    build_items(c, c->m2l_seg.as<long long>(), (int)nn, c->m2l_chunk, c->m2l_items);
    build_items(c, c->p2p_seg.as<long long>(), (int)nn, c->p2p_chunk, c->p2p_items);
    c->list_theta = theta;
    c->walk_gen++;
}

}  // namespace gbfmm
