// fmm_probe_fma_rate: the fused multiply-add rate of the device's binary64 or binary32
// units, measured with a kernel of independent FMA chains.  It is the denominator of the
// roofline of the ALU-bound pair kernels (M2L and P2P), so that their utilisation is
// stated against a measured rate rather than a unit count.
#include <math.h>

#include "fmm_device.cuh"
#include "fmm_internal.h"

namespace gbfmm {

constexpr int PB = 256;      // threads per block
constexpr int PCHAINS = 8;   // independent chains per thread (covers the FMA latency)

template <class T>
__global__ void __launch_bounds__(PB) fma_rate_k(T a, T b, int iters, T* __restrict__ out) {
    T x[PCHAINS];
#pragma unroll
    for (int j = 0; j < PCHAINS; j++) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < PCHAINS; j++) x[j] = fma(x[j], a, b);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < PCHAINS; j++) s += x[j];
    if (s == (T)-1) out[0] = s;  // never true (the chains stay near b / (1 - a)): keeps the work
}

}  // namespace gbfmm

using namespace gbfmm;

namespace gbfmm {
void set_last_error(const char* msg);
}

extern "C" int fmm_probe_fma_rate(int device, int precision, double* tflops) {
    if (!tflops || (precision != FMM_FP64 && precision != FMM_MIXED)) {
        set_last_error("fmm_probe_fma_rate: precision must be FMM_FP64 or FMM_MIXED and tflops non-NULL");
        return FMM_ERR_INVALID;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    void* out = nullptr;
    int rc = FMM_OK;
    auto bad = [&](cudaError_t e, const char* what) {
        if (e == cudaSuccess) return false;
        cudaGetLastError();
        set_last_error((std::string("fmm_probe_fma_rate: ") + what + ": " + cudaGetErrorString(e)).c_str());
        rc = FMM_ERR_CUDA;
        return true;
    };
    int sms = 0;
    if (bad(cudaSetDevice(device), "cudaSetDevice") ||
        bad(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device), "SM count") ||
        bad(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream") || bad(cudaEventCreate(&e0), "event") ||
        bad(cudaEventCreate(&e1), "event") || bad(cudaMalloc(&out, 16), "cudaMalloc")) {
    } else {
        // binary32: ~20 ms at 80 TFLOP/s; binary64: ~20 ms at 1.25 TFLOP/s
        int iters = precision == FMM_MIXED ? (1 << 19) : (1 << 13);
        unsigned grid = (unsigned)sms * 4;
        double flops = 2.0 * PCHAINS * (double)iters * grid * PB;
        double best = 0.0;
        for (int rep = 0; rep < 4 && rc == FMM_OK; rep++) {
            cudaEventRecord(e0, s);
            if (precision == FMM_MIXED)
                fma_rate_k<float><<<grid, PB, 0, s>>>(0.999999f, 1e-7f, iters, static_cast<float*>(out));
            else
                fma_rate_k<double><<<grid, PB, 0, s>>>(0.999999, 1e-7, iters, static_cast<double*>(out));
            count_launch();
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (bad(cudaGetLastError(), "launch") || bad(cudaEventSynchronize(e1), "synchronise") ||
                bad(cudaEventElapsedTime(&ms, e0, e1), "elapsed time"))
                break;
            if (rep > 0 && ms > 0.f) best = fmax(best, flops / (ms * 1e-3) / 1e12);  // first run warms up
        }
        if (rc == FMM_OK) *tflops = best;
    }
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}
