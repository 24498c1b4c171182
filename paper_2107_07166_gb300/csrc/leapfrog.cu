// Kick-drift-kick leapfrog driven by this library's FMM forces, for momentum-drift runs:
// each step kicks v by a dt/2, drifts x by v dt, rebuilds the tree, evaluates forces and
// kicks again.  With central, antisymmetric pair forces (the conserving variant) both
// substeps conserve total linear and angular momentum exactly in exact arithmetic, so
// their drift measures roundoff only; the standard variant shows the spurious torque of
// the truncated expansion (Sec. 2, eq. total_torque).  Everything stays on the device;
// the momenta are summed in a fixed order after every step.
#include <algorithm>
#include <string>

#include "fmm_device.cuh"
#include "fmm_internal.h"

namespace gbfmm {

void set_last_error(const char* msg);
constexpr int LB = 256;

__global__ void kick_k(int64_t n, double* __restrict__ v, const double* __restrict__ a, double h) {
    int64_t i = (int64_t)blockIdx.x * LB + threadIdx.x;
    if (i < 3 * n) v[i] = fma(h, a[i], v[i]);
}

__global__ void drift_k(int64_t n, double* __restrict__ x, const double* __restrict__ v, double dt) {
    int64_t i = (int64_t)blockIdx.x * LB + threadIdx.x;
    if (i < 3 * n) x[i] = fma(dt, v[i], x[i]);
}

__device__ double lf_block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = LB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// per-block sums of m v and m x x v (fixed grid, fixed order)
__global__ void momenta_partial_k(int64_t n, const double* __restrict__ x, const double* __restrict__ v,
                                  const double* __restrict__ m, double* __restrict__ part) {
    __shared__ double sh[LB];
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * LB + threadIdx.x; i < n; i += (int64_t)gridDim.x * LB) {
        double mi = m[i], px = mi * v[3 * i], py = mi * v[3 * i + 1], pz = mi * v[3 * i + 2];
        double X = x[3 * i], Y = x[3 * i + 1], Z = x[3 * i + 2];
        s[0] += px;
        s[1] += py;
        s[2] += pz;
        s[3] += Y * pz - Z * py;
        s[4] += Z * px - X * pz;
        s[5] += X * py - Y * px;
    }
    for (int d = 0; d < 6; d++) {
        double r = lf_block_sum(s[d], sh);
        if (threadIdx.x == 0) part[6 * blockIdx.x + d] = r;
    }
}

__global__ void momenta_final_k(int nb, const double* __restrict__ part, double* __restrict__ out) {
    __shared__ double sh[LB];
    for (int d = 0; d < 6; d++) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nb; b += LB) v += part[6 * b + d];
        double r = lf_block_sum(v, sh);
        if (threadIdx.x == 0) out[d] = r;
    }
}

}  // namespace gbfmm

using namespace gbfmm;

static bool lf_is_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

extern "C" int fmm_leapfrog(fmm_ctx* c, double* x, double* v, const double* m, int64_t N, int leaf_size, int p,
                            double theta, int variant, double dt, int nsteps, double* diag) {
    if (!c || !x || !v || !m) {
        set_last_error("fmm_leapfrog: NULL argument");
        return FMM_ERR_INVALID;
    }
    if (nsteps < 0 || !(dt == dt) || N < 1) {
        set_last_error("fmm_leapfrog: bad N, dt or nsteps");
        return FMM_ERR_INVALID;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->device) cudaSetDevice(c->device);
    int rc = FMM_OK;
    try {
        cudaStream_t s = c->stream;
        size_t b3 = sizeof(double) * 3 * (size_t)N, b1 = sizeof(double) * (size_t)N;
        bool xd = lf_is_device(x), vd = lf_is_device(v), md = lf_is_device(m);
        ensure(c->lf_x, b3);
        ensure(c->lf_v, b3);
        ensure(c->lf_m, b1);
        ensure(c->lf_a, b3);
        int nb = (int)std::min<int64_t>((N + LB - 1) / LB, 592);
        ensure(c->lf_diag, sizeof(double) * (size_t)(6 * nb + 6 * (nsteps + 1)));
        double* X = c->lf_x.as<double>();
        double* V = c->lf_v.as<double>();
        double* M = c->lf_m.as<double>();
        double* A = c->lf_a.as<double>();
        double* part = c->lf_diag.as<double>();
        double* mom = part + 6 * nb;
        GB_CUDA(cudaMemcpyAsync(X, x, b3, xd ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        GB_CUDA(cudaMemcpyAsync(V, v, b3, vd ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        GB_CUDA(cudaMemcpyAsync(M, m, b1, md ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        auto record = [&](int k) {
            momenta_partial_k<<<nb, LB, 0, s>>>(N, X, V, M, part);
            GB_LAUNCH("momenta_partial_k");
            momenta_final_k<<<1, LB, 0, s>>>(nb, part, mom + 6 * k);
            GB_LAUNCH("momenta_final_k");
        };
        auto forces = [&]() {
            int r = fmm_build(c, X, M, N, leaf_size);
            if (r == FMM_OK) r = fmm_forces(c, p, theta, variant, A, nullptr);
            if (r != FMM_OK) throw FmmError{r, std::string("fmm_leapfrog: ") + fmm_last_error()};
        };
        unsigned g3 = grid_for(3 * N, LB);
        forces();
        record(0);
        for (int k = 0; k < nsteps; k++) {
            kick_k<<<g3, LB, 0, s>>>(N, V, A, 0.5 * dt);
            GB_LAUNCH("kick_k");
            drift_k<<<g3, LB, 0, s>>>(N, X, V, dt);
            GB_LAUNCH("drift_k");
            forces();
            kick_k<<<g3, LB, 0, s>>>(N, V, A, 0.5 * dt);
            GB_LAUNCH("kick_k");
            record(k + 1);
        }
        GB_CUDA(cudaMemcpyAsync(x, X, b3, xd ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaMemcpyAsync(v, V, b3, vd ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        if (diag)
            GB_CUDA(cudaMemcpyAsync(diag, mom, sizeof(double) * 6 * (size_t)(nsteps + 1), cudaMemcpyDefault, s));
        GB_CUDA(cudaStreamSynchronize(s));
    } catch (const FmmError& e) {
        set_last_error(e.msg.c_str());
        rc = e.code;
    }
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    return rc;
}
