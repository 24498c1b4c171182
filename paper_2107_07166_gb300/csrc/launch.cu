// Buffers, scans, radix sort and stage timers of the gbfmm CUDA library.
#include <stdio.h>

#include "fmm_device.cuh"
#include "fmm_internal.h"

#include <atomic>

namespace gbfmm {

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launches() { return g_launches.load(std::memory_order_relaxed); }

void cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    int code = (e == cudaErrorMemoryAllocation) ? FMM_ERR_OOM : FMM_ERR_CUDA;
    cudaGetLastError();  // clear a sticky launch error so the context stays usable
    throw FmmError{code, std::string(what) + ": " + cudaGetErrorString(e)};
}

void ensure(DevBuf& b, size_t bytes) {
    if (bytes <= b.bytes && b.p) return;
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

template <class K>
static void radix_sort_t(fmm_ctx* c, DevBuf& keys, DevBuf& keys_tmp, DevBuf* vals, DevBuf* vals_tmp, int64_t n,
                         int bits) {
    if (n <= 1 || bits <= 0) return;
    if (n >= (int64_t)1 << 31) throw FmmError{FMM_ERR_CAPACITY, "radix sort: more than 2^31 keys"};
    int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
    ensure(keys_tmp, sizeof(K) * (size_t)n);
    if (vals) ensure(*vals_tmp, sizeof(uint32_t) * (size_t)n);
    ensure(c->rs_hist, sizeof(uint32_t) * (size_t)(RS_BINS * ntiles + 1));
    ensure(c->rs_offs, sizeof(int) * (size_t)(RS_BINS * ntiles + 1));
    K* ka = keys.as<K>();
    K* kb = keys_tmp.as<K>();
    uint32_t* va = vals ? vals->as<uint32_t>() : nullptr;
    uint32_t* vb = vals ? vals_tmp->as<uint32_t>() : nullptr;
    int passes = (bits + RS_BITS - 1) / RS_BITS;
    for (int ps = 0; ps < passes; ps++) {
        int shift = RS_BITS * ps;
        uint32_t* hist = c->rs_hist.as<uint32_t>();
        rs_hist_k<K><<<ntiles, RS_BLOCK, 0, c->stream>>>(ka, n, shift, hist, ntiles);
        GB_LAUNCH("rs_hist_k");
        scan_int(c, reinterpret_cast<const int*>(hist), (int64_t)RS_BINS * ntiles, c->rs_offs.as<int>());
        const uint32_t* offs = reinterpret_cast<const uint32_t*>(c->rs_offs.as<int>());
        if (vals)
            rs_scatter_k<K, true><<<ntiles, RS_BLOCK, 0, c->stream>>>(ka, va, kb, vb, n, shift, offs, ntiles);
        else
            rs_scatter_k<K, false><<<ntiles, RS_BLOCK, 0, c->stream>>>(ka, nullptr, kb, nullptr, n, shift, offs, ntiles);
        GB_LAUNCH("rs_scatter_k");
        K* tk = ka;
        ka = kb;
        kb = tk;
        uint32_t* tv = va;
        va = vb;
        vb = tv;
    }
    if (passes & 1) {  // result sits in the temporary: swap buffer ownership
        DevBuf t = keys;
        keys = keys_tmp;
        keys_tmp = t;
        if (vals) {
            DevBuf u = *vals;
            *vals = *vals_tmp;
            *vals_tmp = u;
        }
    }
}

void radix_sort(fmm_ctx* c, DevBuf& keys, DevBuf& keys_tmp, DevBuf* vals, DevBuf* vals_tmp, int64_t n, int bits) {
    radix_sort_t<uint64_t>(c, keys, keys_tmp, vals, vals_tmp, n, bits);
}

void radix_sort32(fmm_ctx* c, DevBuf& keys, DevBuf& keys_tmp, DevBuf* vals, DevBuf* vals_tmp, int64_t n, int bits) {
    radix_sort_t<uint32_t>(c, keys, keys_tmp, vals, vals_tmp, n, bits);
}

// ------------------------------------------------------------------ stage timers

void stage_begin(fmm_ctx* c, Stage s) {
    if (!c->ev[2 * s]) {
        GB_CUDA(cudaEventCreate(&c->ev[2 * s]));
        GB_CUDA(cudaEventCreate(&c->ev[2 * s + 1]));
    }
    GB_CUDA(cudaEventRecord(c->ev[2 * s], c->stream));
}

void stage_end(fmm_ctx* c, Stage s) {
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
