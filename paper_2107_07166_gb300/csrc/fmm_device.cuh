// Device-side building blocks of the gbfmm CUDA path: launch helpers, a three-phase
// exclusive scan, and a stable LSD radix sort of 64-bit keys (8-bit digits).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gbfmm {

constexpr unsigned FULL = 0xffffffffu;

inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

// ------------------------------------------------------------------ counters

struct Cnt3 {  // per frontier item: new items, M2L pairs, P2P pairs
    int a, b, c;
};
__host__ __device__ inline Cnt3 operator+(Cnt3 x, Cnt3 y) { return Cnt3{x.a + y.a, x.b + y.b, x.c + y.c}; }
__device__ inline Cnt3 shfl_up(Cnt3 v, int d) {
    return Cnt3{__shfl_up_sync(FULL, v.a, d), __shfl_up_sync(FULL, v.b, d), __shfl_up_sync(FULL, v.c, d)};
}
__device__ inline int shfl_up(int v, int d) { return __shfl_up_sync(FULL, v, d); }
__device__ inline long long shfl_up(long long v, int d) { return __shfl_up_sync(FULL, v, d); }
template <class T>
__device__ inline T zero_of() {
    return T{};
}

// ------------------------------------------------------------------ scan
// out[i] = sum_{j<i} in[j]; out[n] = total.  Phase 1 reduces tiles, phase 2 scans the
// tile sums in one block, phase 3 scans inside tiles.  Integer types only, so the
// result does not depend on the grouping.

constexpr int SCAN_BLOCK = 256, SCAN_ITEMS = 8, SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

template <class T>
__device__ T block_exclusive_scan(T v, T* total) {
    __shared__ T warp_tot[SCAN_BLOCK / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = shfl_up(inc, d);
        if (lane >= d) inc = inc + o;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        T t = lane < SCAN_BLOCK / 32 ? warp_tot[lane] : zero_of<T>();
        T ti = t;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T o = shfl_up(ti, d);
            if (lane >= d) ti = ti + o;
        }
        if (lane < SCAN_BLOCK / 32) warp_tot[lane] = ti;  // inclusive over warps
    }
    __syncthreads();
    T before = w > 0 ? warp_tot[w - 1] : zero_of<T>();
    *total = warp_tot[SCAN_BLOCK / 32 - 1];
    __syncthreads();
    // exclusive prefix inside the warp = inclusive prefix of the previous lane
    T ex = shfl_up(inc, 1);
    if (lane == 0) ex = zero_of<T>();
    return before + ex;
}

template <class T, class In>
__global__ void scan_tiles_k(const In* __restrict__ in, int64_t n, T* __restrict__ tile_sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T s = zero_of<T>();
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++)
        if (base + j < n) s = s + T(in[base + j]);
    T tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

template <class T>
__global__ void scan_sums_k(T* __restrict__ tile_sums, int64_t ntiles) {
    T carry = zero_of<T>();
    for (int64_t b = 0; b < ntiles; b += SCAN_BLOCK) {
        int64_t i = b + threadIdx.x;
        T v = i < ntiles ? tile_sums[i] : zero_of<T>();
        T tot;
        T ex = block_exclusive_scan(v, &tot);
        if (i < ntiles) tile_sums[i] = carry + ex;
        carry = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) tile_sums[ntiles] = carry;
}

template <class T, class In>
__global__ void scan_apply_k(const In* __restrict__ in, int64_t n, const T* __restrict__ tile_sums,
                             T* __restrict__ out) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T s = zero_of<T>();
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        v[j] = (base + j < n) ? T(in[base + j]) : zero_of<T>();
        s = s + v[j];
    }
    T tot;
    T ex = block_exclusive_scan(s, &tot);
    T run = tile_sums[blockIdx.x] + ex;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        if (base + j < n) out[base + j] = run;
        run = run + v[j];
    }
    int64_t ntiles = gridDim.x;
    if (blockIdx.x == ntiles - 1 && threadIdx.x == SCAN_BLOCK - 1) out[n] = tile_sums[ntiles];
}

// ------------------------------------------------------------------ ordered tile claims
// Status words of a decoupled look-back: (tag << 32) | value, read and written with relaxed
// gpu-scope accesses (the walk's frontier steps and the octree's levels).
__device__ __forceinline__ unsigned long long ld_status(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_status(unsigned long long* p, unsigned tag, int value) {
    unsigned long long v = ((unsigned long long)tag << 32) | (unsigned)value;
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Exclusive prefix of tile `tile` over the values published before it: tiles t - 1,
// t - 2, ... are read 32 per round by one warp (lane l reads tile t - 1 - l) until one has
// published its inclusive prefix (tag_pre); published counts (tag_agg) are added on the
// way.  Every tile waited on has been claimed by a running block that publishes its count
// without waiting, so the waits end; they are still bounded by spin_limit polls, after
// which *err is set and the partial sum is returned.  Called by one whole warp; the
// result is valid in every lane.
__device__ __forceinline__ int lookback_prefix(const unsigned long long* __restrict__ status, int tile,
                                               unsigned tag_agg, unsigned tag_pre, long long spin_limit,
                                               int* __restrict__ err) {
    int lane = threadIdx.x & 31, ex = 0, t = tile - 1;
    long long spins = 0;
    while (t >= 0) {
        int u = t - lane;
        unsigned long long w = u >= 0 ? ld_status(status + u) : (unsigned long long)tag_pre << 32;
        unsigned tag = (unsigned)(w >> 32);
        unsigned pre = __ballot_sync(FULL, tag == tag_pre);
        unsigned wait = __ballot_sync(FULL, tag != tag_pre && tag != tag_agg);
        int first = pre ? __ffs(pre) - 1 : 32;  // nearest tile with a prefix
        unsigned need = first >= 31 ? FULL : ((2u << first) - 1u);
        if (wait & need) {  // a tile in the window has not published yet
            if (++spins > spin_limit) {
                if (lane == 0) atomicExch(err, 1);
                break;
            }
            __nanosleep(32);
            continue;
        }
        int val = lane <= first ? (int)(unsigned)w : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(FULL, val, o);
        ex += val;
        if (first < 32) break;
        t -= 32;
    }
    return ex;
}

// ------------------------------------------------------------------ radix sort
// Stable least-significant-digit sort of 64-bit keys with optional 32-bit payloads,
// RS_BITS-bit digits (9: seven passes for 63-bit Morton keys, four for 36-bit list keys).
// Each pass: per-tile digit histograms (digit-major so that one exclusive scan gives
// every tile's output offset), then a stable scatter whose in-tile ranks come from
// warp match masks, in the original order (warp-major, then chunk, then lane).

constexpr int RS_BLOCK = 256, RS_ITEMS = 16, RS_TILE = RS_BLOCK * RS_ITEMS, RS_WARPS = RS_BLOCK / 32;
constexpr int RS_BITS = 9, RS_BINS = 1 << RS_BITS;

__global__ void rs_hist_k(const uint64_t* __restrict__ keys, int64_t n, int shift, uint32_t* __restrict__ hist,
                          int ntiles);

template <bool V>
__global__ void rs_scatter_k(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                             uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n, int shift,
                             const uint32_t* __restrict__ offs, int ntiles);

}  // namespace gbfmm
