// Buffers, scans, radix sort and stage timers of the gbfmm CUDA library.
#include <stdio.h>

#include "fmm_device.cuh"
#include "fmm_internal.h"

#include <algorithm>
#include <atomic>
#include <utility>

namespace gbfmm {

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launches() { return g_launches.load(std::memory_order_relaxed); }

// device buffers allocated or freed so far (any context): a recorded CUDA graph holds
// buffer addresses and stays valid only while this count does not change
static std::atomic<long long> g_reallocs{0};
long long realloc_count() { return g_reallocs.load(std::memory_order_relaxed); }

void cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    int code = (e == cudaErrorMemoryAllocation) ? FMM_ERR_OOM : FMM_ERR_CUDA;
    cudaGetLastError();  // clear a sticky launch error so the context stays usable
    throw FmmError{code, std::string(what) + ": " + cudaGetErrorString(e)};
}

void ensure(DevBuf& b, size_t bytes) {
    if (bytes <= b.bytes && b.p) return;
    g_reallocs.fetch_add(1, std::memory_order_relaxed);
    if (b.p) GB_CUDA(cudaFree(b.p));
    b.p = nullptr;
    b.bytes = 0;
    size_t want = bytes + bytes / 4 + 256;  // headroom against repeated growth
    GB_CUDA(cudaMalloc(&b.p, want));
    b.bytes = want;
}

void ensure_keep(DevBuf& b, size_t bytes, cudaStream_t s) {
    if (bytes <= b.bytes && b.p) return;
    size_t want = bytes + bytes / 2 + 256;
    g_reallocs.fetch_add(1, std::memory_order_relaxed);
    void* np = nullptr;
    GB_CUDA(cudaMalloc(&np, want));
    if (b.p) {
        GB_CUDA(cudaMemcpyAsync(np, b.p, b.bytes, cudaMemcpyDeviceToDevice, s));
        GB_CUDA(cudaStreamSynchronize(s));
        GB_CUDA(cudaFree(b.p));
    }
    b.p = np;
    b.bytes = want;
}

void release(DevBuf& b) {
    if (b.p) g_reallocs.fetch_add(1, std::memory_order_relaxed);
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

// ------------------------------------------------------------------ scans

template <class T, class In>
static void scan_impl(fmm_ctx* c, const In* in, int64_t n, T* out) {
    int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (ntiles == 0) ntiles = 1;
    ensure(c->scan_tmp, sizeof(T) * (size_t)(ntiles + 1));
    T* sums = c->scan_tmp.as<T>();
    scan_tiles_k<T, In><<<(unsigned)ntiles, SCAN_BLOCK, 0, c->stream>>>(in, n, sums);
    GB_LAUNCH("scan_tiles_k");
    scan_sums_k<T><<<1, SCAN_BLOCK, 0, c->stream>>>(sums, ntiles);
    GB_LAUNCH("scan_sums_k");
    scan_apply_k<T, In><<<(unsigned)ntiles, SCAN_BLOCK, 0, c->stream>>>(in, n, sums, out);
    GB_LAUNCH("scan_apply_k");
}

void scan_int(fmm_ctx* c, const int* in, int64_t n, int* out) { scan_impl<int, int>(c, in, n, out); }
void scan_i64(fmm_ctx* c, const int* in, int64_t n, long long* out) { scan_impl<long long, int>(c, in, n, out); }
void scan_i64_from_i64(fmm_ctx* c, const long long* in, int64_t n, long long* out) {
    scan_impl<long long, long long>(c, in, n, out);
}

// ------------------------------------------------------------------ radix sort

template <class K>
__global__ void rs_hist_k(const K* __restrict__ keys, int64_t n, int shift, uint32_t* __restrict__ hist,
                          int ntiles) {
    __shared__ uint32_t sh[RS_BINS];
    for (int i = threadIdx.x; i < RS_BINS; i += RS_BLOCK) sh[i] = 0;
    __syncthreads();
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * (32 * RS_ITEMS);
#pragma unroll 4
    for (int j = 0; j < RS_ITEMS; j++) {
        int64_t i = base + j * 32 + lane;
        unsigned d = (i < n) ? (unsigned)((keys[i] >> shift) & (RS_BINS - 1)) : (unsigned)RS_BINS;
        unsigned peers = __match_any_sync(FULL, d);
        if (d < (unsigned)RS_BINS && lane == __ffs(peers) - 1) atomicAdd(&sh[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RS_BINS; d += RS_BLOCK) hist[(int64_t)d * ntiles + blockIdx.x] = sh[d];
}

template <class K, bool V>
__global__ void __launch_bounds__(RS_BLOCK, sizeof(K) == 4 ? 4 : 2) rs_scatter_k(const K* __restrict__ kin,
                                                         const uint32_t* __restrict__ vin,
                                                         K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                         int64_t n, int shift, const uint32_t* __restrict__ offs,
                                                         int ntiles) {
    __shared__ uint32_t wcnt[RS_WARPS][RS_BINS];
    __shared__ uint32_t dbase[RS_BINS];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_BLOCK) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * (32 * RS_ITEMS);
    K k[RS_ITEMS];
    uint32_t v[RS_ITEMS];
    uint32_t rank[RS_ITEMS];
    unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        int64_t i = base + j * 32 + lane;
        bool ok = i < n;
        k[j] = ok ? kin[i] : K(0);
        if (V) v[j] = ok ? vin[i] : 0u;
        unsigned d = ok ? (unsigned)((k[j] >> shift) & (RS_BINS - 1)) : (unsigned)RS_BINS;
        unsigned peers = __match_any_sync(FULL, d);
        uint32_t r = 0;
        if (ok) r = wcnt[warp][d] + (uint32_t)__popc(peers & lt);
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) wcnt[warp][d] += (uint32_t)__popc(peers);
        __syncwarp();
        rank[j] = r;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RS_BINS; d += RS_BLOCK) {
        uint32_t s = 0;
        for (int w = 0; w < RS_WARPS; w++) {
            uint32_t t = wcnt[w][d];
            wcnt[w][d] = s;
            s += t;
        }
        dbase[d] = offs[(int64_t)d * ntiles + blockIdx.x];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        int64_t i = base + j * 32 + lane;
        if (i < n) {
            unsigned d = (unsigned)((k[j] >> shift) & (RS_BINS - 1));
            uint32_t pos = dbase[d] + wcnt[warp][d] + rank[j];
            kout[pos] = k[j];
            if (V) vout[pos] = v[j];
        }
    }
}

// One stable RS_BITS-bit pass of keys + 32-bit payloads on caller-provided buffers: hist
// and offs hold RS_BINS * ntiles + 1 entries, sums (RS_BINS * ntiles) / SCAN_TILE + 2.
// Allocates nothing.
void rs_pass_raw(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout, int64_t n, int shift,
                 uint32_t* hist, int* offs, int* sums, cudaStream_t s) {
    int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
    int64_t nh = (int64_t)RS_BINS * ntiles;
    int nst = (int)((nh + SCAN_TILE - 1) / SCAN_TILE);
    rs_hist_k<uint64_t><<<ntiles, RS_BLOCK, 0, s>>>(kin, n, shift, hist, ntiles);
    scan_tiles_k<int, int><<<nst, SCAN_BLOCK, 0, s>>>(reinterpret_cast<const int*>(hist), nh, sums);
    scan_sums_k<int><<<1, SCAN_BLOCK, 0, s>>>(sums, nst);
    scan_apply_k<int, int><<<nst, SCAN_BLOCK, 0, s>>>(reinterpret_cast<const int*>(hist), nh, sums, offs);
    rs_scatter_k<uint64_t, true><<<ntiles, RS_BLOCK, 0, s>>>(kin, vin, kout, vout, n, shift,
                                                             reinterpret_cast<const uint32_t*>(offs), ntiles);
}


// ------------------------------------------------------------------ one-sweep radix sort
//
// The sort of radix_sort(): every pass is one kernel.  The digit totals of all passes come
// from one read of the keys (rs_ghist_k, integer atomics: order-independent) and one scan
// (rs_gscan_k); inside a pass, tile t learns how many keys of digit d the tiles before it
// hold from their status words (decoupled look-back per digit), so the per-pass tile
// histograms and their scans of the multi-kernel form are gone.  Tiles take their data
// range from an atomic ticket, in launch-independent order, and rank their keys as
// rs_scatter_k does (warp match masks, warp-major order): the sort stays stable and its
// result is the same permutation.

constexpr int RS_MAXP = 8;  // passes per sort (64-bit keys: at most 8 digits of 9 bits)

template <class K>
__global__ void __launch_bounds__(RS_BLOCK) rs_ghist_k(const K* __restrict__ keys, int64_t n, int passes,
                                                       uint32_t* __restrict__ ghist) {
    __shared__ uint32_t sh[RS_MAXP * RS_BINS];
    for (int i = threadIdx.x; i < passes * RS_BINS; i += RS_BLOCK) sh[i] = 0;
    __syncthreads();
    // four keys per thread and round, loaded before their counts are added
    constexpr int U = 4;
    int64_t stride = (int64_t)gridDim.x * RS_BLOCK * U;
    for (int64_t i0 = (int64_t)blockIdx.x * RS_BLOCK * U; i0 < n; i0 += stride) {
        K k[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            int64_t i = i0 + u * RS_BLOCK + threadIdx.x;
            k[u] = i < n ? keys[i] : K(0);
        }
#pragma unroll
        for (int u = 0; u < U; u++)
            if (i0 + u * RS_BLOCK + threadIdx.x < n)
                for (int p = 0; p < passes; p++)
                    atomicAdd(&sh[p * RS_BINS + (unsigned)((k[u] >> (RS_BITS * p)) & (RS_BINS - 1))], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RS_BINS; i += RS_BLOCK)
        if (sh[i]) atomicAdd(&ghist[i], sh[i]);
}

// exclusive scan of each pass's digit totals (one block per pass; RS_BINS = 2 RS_BLOCK)
static_assert(RS_BINS == 2 * RS_BLOCK && RS_BLOCK == SCAN_BLOCK, "rs_gscan_k: two digits per thread");
__global__ void __launch_bounds__(RS_BLOCK) rs_gscan_k(const uint32_t* __restrict__ ghist, uint32_t* __restrict__ gofs) {
    const uint32_t* h = ghist + (int64_t)blockIdx.x * RS_BINS;
    uint32_t* o = gofs + (int64_t)blockIdx.x * RS_BINS;
    int t = threadIdx.x;
    uint32_t a = h[2 * t], b = h[2 * t + 1];
    int tot;
    int ex = block_exclusive_scan<int>((int)(a + b), &tot);
    o[2 * t] = (uint32_t)ex;
    o[2 * t + 1] = (uint32_t)ex + a;
}

// keys of digits d_q = d0 + q RS_BLOCK (q < Q) in the tiles before `tile`: status words of
// tiles tile - 1, tile - 2, ... (R per digit and round, all digits' reads in flight
// together) are summed until one holds its inclusive count (tag_pre); a tile that has not
// published yet is waited for.  Every tile waited on holds an earlier ticket and publishes
// its counts before it waits itself, so the waits end; they are still bounded by
// spin_limit polls, after which *err is set.
template <int Q, int R>
__device__ __forceinline__ void digit_lookback(const unsigned long long* __restrict__ status, int tile, int d0,
                                               unsigned tag_agg, unsigned tag_pre, long long spin_limit,
                                               int* __restrict__ err, int* ex) {
    int t[Q];
    bool done[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) {
        ex[q] = 0;
        t[q] = tile - 1;
        done[q] = t[q] < 0;
    }
    long long spins = 0;
    for (;;) {
        bool all = true;
#pragma unroll
        for (int q = 0; q < Q; q++) all = all && done[q];
        if (all) return;
        unsigned long long w[Q][R];
#pragma unroll
        for (int q = 0; q < Q; q++)
#pragma unroll
            for (int j = 0; j < R; j++)
                w[q][j] = !done[q] && t[q] - j >= 0
                              ? ld_status(status + (int64_t)(t[q] - j) * RS_BINS + d0 + q * RS_BLOCK)
                              : (unsigned long long)tag_pre << 32;
        bool moved = false;
#pragma unroll
        for (int q = 0; q < Q; q++) {
            if (done[q]) continue;
            int j = 0;
            for (; j < R; j++) {
                unsigned tag = (unsigned)(w[q][j] >> 32);
                if (tag == tag_pre) {
                    ex[q] += (int)(unsigned)w[q][j];
                    done[q] = true;
                    break;
                }
                if (tag != tag_agg) break;  // not published yet
                ex[q] += (int)(unsigned)w[q][j];
            }
            if (!done[q]) t[q] -= j;
            moved = moved || done[q] || j > 0;
        }
        if (!moved) {
            if (++spins > spin_limit) {
                atomicExch(err, 1);
                return;
            }
            __nanosleep(32);
        }
    }
}

// Shared memory of rs_sweep_k: the warps' digit counts while the keys are ranked, then the
// tile's keys (and payloads) in digit order.
template <class K, bool V>
constexpr size_t rs_sweep_smem() {
    size_t cnt = sizeof(uint32_t) * RS_WARPS * RS_BINS;
    size_t tile = (sizeof(K) + (V ? sizeof(uint32_t) : 0)) * (size_t)RS_TILE;
    return cnt > tile ? cnt : tile;
}

template <class K, bool V>
__global__ void __launch_bounds__(RS_BLOCK, sizeof(K) == 4 ? 4 : 2) rs_sweep_k(const K* __restrict__ kin,
                                                       const uint32_t* __restrict__ vin, K* __restrict__ kout,
                                                       uint32_t* __restrict__ vout, int64_t n, int shift,
                                                       const uint32_t* __restrict__ gofs,
                                                       unsigned long long* __restrict__ status,
                                                       int* __restrict__ ticket, unsigned tag_agg, unsigned tag_pre,
                                                       long long spin_limit, int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char rs_smem[];
    uint32_t(*wcnt)[RS_BINS] = reinterpret_cast<uint32_t(*)[RS_BINS]>(rs_smem);
    K* ks = reinterpret_cast<K*>(rs_smem);  // after ranking: the tile in digit order
    uint32_t* vs = reinterpret_cast<uint32_t*>(rs_smem + sizeof(K) * RS_TILE);
    __shared__ uint32_t dbase[RS_BINS];
    __shared__ uint32_t lstart[RS_BINS];  // first slot of every digit in the tile's digit order
    __shared__ int tile_s;
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) tile_s = atomicAdd(ticket, 1);
    for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_BLOCK) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    int tile = tile_s;
    int64_t base = (int64_t)tile * RS_TILE + (int64_t)warp * (32 * RS_ITEMS);
    K k[RS_ITEMS];
    uint32_t v[RS_ITEMS];
    uint32_t rank[RS_ITEMS];
    unsigned lt = (1u << lane) - 1u;
    // all of the tile's loads are issued before the ranking: its warp barriers would
    // otherwise keep each load's latency on the critical path
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        int64_t i = base + j * 32 + lane;
        bool ok = i < n;
        k[j] = ok ? kin[i] : K(0);
        if (V) v[j] = ok ? vin[i] : 0u;
    }
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        int64_t i = base + j * 32 + lane;
        bool ok = i < n;
        unsigned d = ok ? (unsigned)((k[j] >> shift) & (RS_BINS - 1)) : (unsigned)RS_BINS;
        unsigned peers = __match_any_sync(FULL, d);
        uint32_t r = 0;
        if (ok) r = wcnt[warp][d] + (uint32_t)__popc(peers & lt);
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) wcnt[warp][d] += (uint32_t)__popc(peers);
        __syncwarp();
        rank[j] = r;
    }
    __syncthreads();
    // the tile's count of every digit (warp offsets left in wcnt), published at once: a
    // later tile may be waiting for it
    constexpr int Q = RS_BINS / RS_BLOCK;
    static_assert(Q == 2, "rs_sweep_k: two digits per thread");
    uint32_t cnt[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) {
        int d = threadIdx.x + q * RS_BLOCK;
        uint32_t s = 0;
        for (int w = 0; w < RS_WARPS; w++) {
            uint32_t t = wcnt[w][d];
            wcnt[w][d] = s;
            s += t;
        }
        cnt[q] = s;
        st_status(status + (int64_t)tile * RS_BINS + d, tile == 0 ? tag_pre : tag_agg, (int)s);
    }
    // digit starts inside the tile (digits 0..255, then 256..511)
    int tot0, tot1;
    int ls0 = block_exclusive_scan<int>((int)cnt[0], &tot0);
    int ls1 = block_exclusive_scan<int>((int)cnt[1], &tot1) + tot0;
    lstart[threadIdx.x] = (uint32_t)ls0;
    lstart[threadIdx.x + RS_BLOCK] = (uint32_t)ls1;
    __syncthreads();
    // every key's slot in the tile's digit order (warp-major, so the order inside a digit
    // is the input order and the sort stays stable)
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        unsigned d = (unsigned)((k[j] >> shift) & (RS_BINS - 1));
        rank[j] += lstart[d] + wcnt[warp][d];
    }
    __syncthreads();  // wcnt is read: its space now takes the staged tile
    int tn = (int)min((int64_t)RS_TILE, n - (int64_t)tile * RS_TILE);
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        int64_t i = base + j * 32 + lane;
        if (i < n) {
            ks[rank[j]] = k[j];
            if (V) vs[rank[j]] = v[j];
        }
    }
    int ex[Q];
    // reads per digit and round: what the registers left by the tile's keys allow
    digit_lookback<Q, sizeof(K) == 8 ? 4 : 2>(status, tile, threadIdx.x, tag_agg, tag_pre, spin_limit, err, ex);
#pragma unroll
    for (int q = 0; q < Q; q++) {
        int d = threadIdx.x + q * RS_BLOCK;
        if (tile > 0) st_status(status + (int64_t)tile * RS_BINS + d, tag_pre, ex[q] + (int)cnt[q]);
        dbase[d] = gofs[d] + (uint32_t)ex[q];
    }
    __syncthreads();
    // the staged tile goes out in digit order: consecutive threads of a digit's run write
    // consecutive outputs
    for (int i = threadIdx.x; i < tn; i += RS_BLOCK) {
        K key = ks[i];
        unsigned d = (unsigned)((key >> shift) & (RS_BINS - 1));
        uint32_t pos = dbase[d] + ((uint32_t)i - lstart[d]);
        if (pos < (uint64_t)n) {  // always, unless a look-back gave up (then the prefix is short)
            kout[pos] = key;
            if (V) vout[pos] = vs[i];
        }
    }
}

// polls of one status word before a sort tile gives up (never reached in a correct run)
constexpr long long RS_SPIN_LIMIT = 1ll << 22;

static unsigned next_tag(fmm_ctx* c) {
    if (++c->rs_epoch == 0u) ++c->rs_epoch;
    return c->rs_epoch;
}

int* sort_err(fmm_ctx* c) {
    if (!c->rs_err.p) {
        ensure(c->rs_err, sizeof(int) * 4);
        GB_CUDA(cudaMemsetAsync(c->rs_err.p, 0, c->rs_err.bytes, c->stream));
    }
    return c->rs_err.as<int>();
}

void sort_err_throw(fmm_ctx* c, int flag) {
    if (!flag) return;
    GB_CUDA(cudaMemsetAsync(c->rs_err.p, 0, sizeof(int), c->stream));
    throw FmmError{FMM_ERR_TIMEOUT, "radix sort: a tile waited too long for the tiles before it"};
}

template <class K>
static void radix_sort_t(fmm_ctx* c, DevBuf& keys, DevBuf& keys_tmp, DevBuf* vals, DevBuf* vals_tmp, int64_t n,
                         int bits) {
    if (n <= 1 || bits <= 0) return;
    if (n >= (int64_t)1 << 31) throw FmmError{FMM_ERR_CAPACITY, "radix sort: more than 2^31 keys"};
    cudaStream_t s = c->stream;
    int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
    int passes = (bits + RS_BITS - 1) / RS_BITS;
    if (passes > RS_MAXP) throw FmmError{FMM_ERR_INVALID, "radix sort: more than 8 digits"};
    ensure(keys_tmp, sizeof(K) * (size_t)n);
    if (vals) ensure(*vals_tmp, sizeof(uint32_t) * (size_t)n);
    // [digit totals | tickets] (cleared per sort), then the digit offsets
    ensure(c->rs_hist, sizeof(uint32_t) * (size_t)(2 * RS_MAXP * RS_BINS + RS_MAXP));
    uint32_t* ghist = c->rs_hist.as<uint32_t>();
    int* tick = reinterpret_cast<int*>(ghist + RS_MAXP * RS_BINS);
    uint32_t* gofs = ghist + RS_MAXP * RS_BINS + RS_MAXP;
    GB_CUDA(cudaMemsetAsync(ghist, 0, sizeof(uint32_t) * (size_t)(RS_MAXP * RS_BINS + RS_MAXP), s));
    // status words (tag << 32 | count) per (tile, digit); tags are new for every pass, so
    // the words of earlier passes read as "not published" and the buffer is cleared only
    // when it is allocated (or the tags wrap)
    void* old = c->rs_status.p;
    ensure(c->rs_status, sizeof(unsigned long long) * (size_t)ntiles * RS_BINS);
    if (c->rs_status.p != old || c->rs_epoch > 0xFFFFFF00u) {
        GB_CUDA(cudaMemsetAsync(c->rs_status.p, 0, c->rs_status.bytes, s));
        c->rs_epoch = 0;
    }
    unsigned long long* status = c->rs_status.as<unsigned long long>();
    int* err = sort_err(c);
    int dev_sms = 0;
    GB_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c->device));
    K* ka = keys.as<K>();
    K* kb = keys_tmp.as<K>();
    uint32_t* va = vals ? vals->as<uint32_t>() : nullptr;
    uint32_t* vb = vals ? vals_tmp->as<uint32_t>() : nullptr;
    int gh = std::min(ntiles, dev_sms * 4);
    rs_ghist_k<K><<<gh, RS_BLOCK, 0, s>>>(ka, n, passes, ghist);
    GB_LAUNCH("rs_ghist_k");
    rs_gscan_k<<<passes, RS_BLOCK, 0, s>>>(ghist, gofs);
    GB_LAUNCH("rs_gscan_k");
    constexpr size_t shm_v = rs_sweep_smem<K, true>(), shm_k = rs_sweep_smem<K, false>();
    GB_CUDA(cudaFuncSetAttribute(rs_sweep_k<K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_v));
    GB_CUDA(cudaFuncSetAttribute(rs_sweep_k<K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_k));
    for (int ps = 0; ps < passes; ps++) {
        int shift = RS_BITS * ps;
        unsigned ta = next_tag(c), tp = next_tag(c);
        if (vals)
            rs_sweep_k<K, true><<<ntiles, RS_BLOCK, shm_v, s>>>(ka, va, kb, vb, n, shift, gofs + ps * RS_BINS, status,
                                                                tick + ps, ta, tp, RS_SPIN_LIMIT, err);
        else
            rs_sweep_k<K, false><<<ntiles, RS_BLOCK, shm_k, s>>>(ka, nullptr, kb, nullptr, n, shift,
                                                                 gofs + ps * RS_BINS, status, tick + ps, ta, tp,
                                                                 RS_SPIN_LIMIT, err);
        GB_LAUNCH("rs_sweep_k");
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (passes & 1) {  // result sits in the temporary: swap buffer ownership
        std::swap(keys, keys_tmp);
        if (vals) std::swap(*vals, *vals_tmp);
    }
}

void radix_sort(fmm_ctx* c, DevBuf& keys, DevBuf& keys_tmp, DevBuf* vals, DevBuf* vals_tmp, int64_t n, int bits) {
    radix_sort_t<uint64_t>(c, keys, keys_tmp, vals, vals_tmp, n, bits);
}

void radix_sort32(fmm_ctx* c, DevBuf& keys, DevBuf& keys_tmp, DevBuf* vals, DevBuf* vals_tmp, int64_t n, int bits) {
    radix_sort_t<uint32_t>(c, keys, keys_tmp, vals, vals_tmp, n, bits);
}

// ------------------------------------------------------------------ side stream

void fork_side(fmm_ctx* c) {
    if (!c->side) {
        GB_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
        GB_CUDA(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
        GB_CUDA(cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming));
    }
    GB_CUDA(cudaEventRecord(c->fork_ev, c->stream));
    GB_CUDA(cudaStreamWaitEvent(c->side, c->fork_ev, 0));
}

void join_side(fmm_ctx* c) {
    GB_CUDA(cudaEventRecord(c->join_ev, c->side));
    GB_CUDA(cudaStreamWaitEvent(c->stream, c->join_ev, 0));
}

SideLaunches::SideLaunches(fmm_ctx* ctx) : c(ctx), main(ctx->stream) { c->stream = c->side; }
SideLaunches::~SideLaunches() { c->stream = main; }

// ------------------------------------------------------------------ stage timers

void stage_begin(fmm_ctx* c, Stage s) {
    if (c->capturing) return;
    if (!c->ev[2 * s]) {
        GB_CUDA(cudaEventCreate(&c->ev[2 * s]));
        GB_CUDA(cudaEventCreate(&c->ev[2 * s + 1]));
    }
    GB_CUDA(cudaEventRecord(c->ev[2 * s], c->stream));
}

void stage_end(fmm_ctx* c, Stage s) {
    if (c->capturing) return;
    GB_CUDA(cudaEventRecord(c->ev[2 * s + 1], c->stream));
    c->stage_valid[s] = true;
}

NodeView node_view(const fmm_ctx* c) {
    return NodeView{c->nfirst.as<int>(), c->ncount.as<int>(),  c->nparent.as<int>(),
                    c->nchildf.as<int>(), c->nnchild.as<int>(), c->nZx.as<double>(),
                    c->nZy.as<double>(),  c->nZz.as<double>(),  c->nrmax.as<double>(),
                    c->zhl.as<float4>(),  c->zhl.as<float4>() + c->n_nodes};
}

}  // namespace gbfmm
