// fmm_morton_sort_noalloc: the first steps of fmm_build (bounding cube, Morton keys,
// stable radix sort of the keys) for callers that cannot allocate device memory.
//
// All scratch lives in one file-scope device array of fixed size (NOALLOC_SCRATCH_BYTES,
// held by every GPU that loads the library until the process exits).  Host code may
// not use the array's name as a device address, so the address is looked up once per
// device with cudaGetSymbolAddress while that device is current, and the kernels get
// that pointer.  Every call shares the array: calls whose work overlaps on the GPU
// race, and each call clears what must start at zero.
#include <mutex>
#include <string>

#include "fmm_device.cuh"
#include "fmm_internal.h"

namespace gbfmm {

// kernels of the tree build (tree.cu) and of the radix sort (launch.cu)
__global__ void bbox_partial_k(const double* __restrict__ x, const double* __restrict__ m, int64_t n,
                               double* __restrict__ part, int* __restrict__ bad);
__global__ void bbox_final_k(const double* __restrict__ part, int nb, double* __restrict__ geom);
__global__ void keys_k(const double* __restrict__ x, int64_t n, const double* __restrict__ geom,
                       uint64_t* __restrict__ keys, uint32_t* __restrict__ idx);
void rs_pass_raw(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout, int64_t n, int shift,
                 uint32_t* hist, int* offs, int* sums, cudaStream_t s);

namespace {

constexpr int64_t NA_MAX_N = FMM_NOALLOC_MAX_N;                     // particles per call
constexpr int NA_TB = 256;                                          // bbox block size
constexpr int NA_MAX_TILES = (int)(NA_MAX_N / RS_TILE);             // 32 sort tiles
constexpr int NA_HIST = RS_BINS * NA_MAX_TILES + 1;
constexpr int NA_MAX_BB = (int)(NA_MAX_N / NA_TB);                  // 512 bbox blocks

constexpr size_t al256(size_t b) { return (b + 255) / 256 * 256; }
// scratch layout (byte offsets)
constexpr size_t OFF_KEYS_B = 0;
constexpr size_t OFF_VALS_A = OFF_KEYS_B + al256(sizeof(uint64_t) * NA_MAX_N);
constexpr size_t OFF_VALS_B = OFF_VALS_A + al256(sizeof(uint32_t) * NA_MAX_N);
constexpr size_t OFF_HIST = OFF_VALS_B + al256(sizeof(uint32_t) * NA_MAX_N);
constexpr size_t OFF_OFFS = OFF_HIST + al256(sizeof(uint32_t) * NA_HIST);
constexpr size_t OFF_SUMS = OFF_OFFS + al256(sizeof(int) * NA_HIST);
constexpr size_t OFF_PART = OFF_SUMS + al256(sizeof(int) * 64);
constexpr size_t OFF_GEOM = OFF_PART + al256(sizeof(double) * 6 * NA_MAX_BB);
constexpr size_t OFF_FLAG = OFF_GEOM + al256(sizeof(double) * 8);
constexpr size_t NOALLOC_SCRATCH_BYTES = OFF_FLAG + al256(sizeof(int) * 4);   // ~2.2 MiB
// the cube kernel reads N zero masses from vals_a..vals_b (see below): the two payload
// regions must be adjacent, exactly 4 NA_MAX_N bytes apart, and end before the histograms
static_assert(OFF_VALS_B - OFF_VALS_A == sizeof(uint32_t) * NA_MAX_N, "payload regions must be adjacent");
static_assert(OFF_HIST - OFF_VALS_A >= sizeof(double) * NA_MAX_N, "zero masses must fit before the histograms");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NA_MAX_DEV = 64;
std::mutex g_na_mutex;
unsigned char* g_na_addr[NA_MAX_DEV] = {};

__global__ void widen_perm_k(const uint32_t* __restrict__ v, int64_t n, int64_t* __restrict__ perm) {
    int64_t i = (int64_t)blockIdx.x * NA_TB + threadIdx.x;
    if (i < n) perm[i] = v[i];
}

// true when p is memory the kernels on device dev may access directly: device memory of
// dev itself, or managed memory
bool is_device_memory(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace
}  // namespace gbfmm

using namespace gbfmm;

namespace gbfmm {
void set_last_error(const char* msg);
}

// a failed CUDA step: clear the sticky error, record which step failed and why
static int na_cuda_fail(const char* step, cudaError_t e) {
    cudaGetLastError();
    std::string msg = std::string("fmm_morton_sort_noalloc: ") + step + ": " + cudaGetErrorString(e);
    set_last_error(msg.c_str());
    return FMM_ERR_CUDA;
}

extern "C" int fmm_morton_sort_noalloc(const double* x, int64_t N, uint64_t* keys_sorted, int64_t* perm,
                                       double* lo, double* side, void* cuda_stream) {
    if (!x || !keys_sorted || !perm) {
        set_last_error("fmm_morton_sort_noalloc: x, keys_sorted and perm are required");
        return FMM_ERR_INVALID;
    }
    if (N < 1) {
        set_last_error("fmm_morton_sort_noalloc: N must be >= 1");
        return FMM_ERR_INVALID;
    }
    if (N > NA_MAX_N) {
        set_last_error("fmm_morton_sort_noalloc: N exceeds FMM_NOALLOC_MAX_N (131072)");
        return FMM_ERR_CAPACITY;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_cuda_fail("cudaGetDevice", e);
    if (dev < 0 || dev >= NA_MAX_DEV) {
        set_last_error("fmm_morton_sort_noalloc: device ordinal above the supported 64");
        return FMM_ERR_CUDA;
    }
    if (!is_device_memory(x, dev) || !is_device_memory(keys_sorted, dev) || !is_device_memory(perm, dev) ||
        (lo && !is_device_memory(lo, dev)) || (side && !is_device_memory(side, dev))) {
        set_last_error("fmm_morton_sort_noalloc: every array must be device memory of the current device");
        return FMM_ERR_INVALID;
    }
    // one-time set-up on this device: the device address of the scratch array
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> g(g_na_mutex);
        if (!g_na_addr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess) return na_cuda_fail("cudaGetSymbolAddress of the scratch array", e);
            if (!ptr) {
                set_last_error("fmm_morton_sort_noalloc: the scratch array has no device address");
                return FMM_ERR_CUDA;
            }
            g_na_addr[dev] = static_cast<unsigned char*>(ptr);
        }
        base = g_na_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    uint64_t* keys_a = keys_sorted;
    uint64_t* keys_b = reinterpret_cast<uint64_t*>(base + OFF_KEYS_B);
    uint32_t* vals_a = reinterpret_cast<uint32_t*>(base + OFF_VALS_A);
    uint32_t* vals_b = reinterpret_cast<uint32_t*>(base + OFF_VALS_B);
    uint32_t* hist = reinterpret_cast<uint32_t*>(base + OFF_HIST);
    int* offs = reinterpret_cast<int*>(base + OFF_OFFS);
    int* sums = reinterpret_cast<int*>(base + OFF_SUMS);
    double* part = reinterpret_cast<double*>(base + OFF_PART);
    double* geom = reinterpret_cast<double*>(base + OFF_GEOM);
    int* flag = reinterpret_cast<int*>(base + OFF_FLAG);
    int nb = (int)((N + NA_TB - 1) / NA_TB);
    e = cudaMemsetAsync(flag, 0, sizeof(int) * 4, s);
    if (e != cudaSuccess) return na_cuda_fail("clearing the status flag", e);
    // a1: cube, with the finiteness check of the coordinates.  The cube kernel also checks
    // masses; none are given here, so it reads N zero doubles (+0.0, a valid mass) from the
    // payload regions vals_a..vals_b (8 N bytes, cleared here, overwritten by the keys step).
    e = cudaMemsetAsync(vals_a, 0, sizeof(double) * (size_t)N, s);
    if (e != cudaSuccess) return na_cuda_fail("clearing the zero masses", e);
    bbox_partial_k<<<nb, NA_TB, 0, s>>>(x, reinterpret_cast<const double*>(vals_a), N, part, flag);
    bbox_final_k<<<1, 512, 0, s>>>(part, nb, geom);
    // a2: keys and identity payload
    keys_k<<<(unsigned)((N + NA_TB - 1) / NA_TB), NA_TB, 0, s>>>(x, N, geom, keys_a, vals_a);
    // a3: stable RS_BITS-bit passes over the 63-bit keys
    int passes = (63 + RS_BITS - 1) / RS_BITS;
    for (int ps = 0; ps < passes; ps++) {
        rs_pass_raw(keys_a, vals_a, keys_b, vals_b, N, RS_BITS * ps, hist, offs, sums, s);
        uint64_t* tk = keys_a;
        keys_a = keys_b;
        keys_b = tk;
        uint32_t* tv = vals_a;
        vals_a = vals_b;
        vals_b = tv;
    }
    if (keys_a != keys_sorted &&
        (e = cudaMemcpyAsync(keys_sorted, keys_a, sizeof(uint64_t) * (size_t)N, cudaMemcpyDeviceToDevice, s)) !=
            cudaSuccess)
        return na_cuda_fail("copying the sorted keys", e);
    widen_perm_k<<<(unsigned)((N + NA_TB - 1) / NA_TB), NA_TB, 0, s>>>(vals_a, N, perm);
    if (lo && (e = cudaMemcpyAsync(lo, geom, sizeof(double) * 3, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return na_cuda_fail("copying lo", e);
    if (side && (e = cudaMemcpyAsync(side, geom + 3, sizeof(double), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return na_cuda_fail("copying side", e);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_cuda_fail("a kernel launch", e);
    // the finiteness flag is read back on the host: the call waits for its stream here
    int bad = 0;
    if ((e = cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return na_cuda_fail("reading the status flag", e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return na_cuda_fail("synchronising the stream", e);
    if (bad) set_last_error("fmm_morton_sort_noalloc: non-finite coordinate");
    return bad ? FMM_ERR_INVALID : FMM_OK;
}
