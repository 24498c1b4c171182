// a12 mutual particle-particle interactions (eq. jia and its gradient) and a14 diagnostics.
//
// One warp per leaf pair of the P2P list.  For distinct leaves the smaller one is held
// in lanes ("fixed", accumulators in registers) and the larger one is staged in shared
// memory ("rotating"); in step s lane l meets rotating particle (l + s) mod n_rot, so
// every particle pair is met exactly once and, within a step, no two lanes touch the
// same rotating accumulator.  A self pair uses cyclic distances 1 .. n/2.  Each pair
// force is applied to both partners (action = reaction).  The per-pair results go to a
// partial buffer and are summed per particle, in increasing partner id, by the final
// per-particle kernel: no floating-point atomics, run-to-run identical.
#include "fmm_device.cuh"
#include "fmm_internal.h"

namespace gbfmm {

constexpr int PB = 128;                // 4 warps
constexpr int PW = PB / 32;

struct PState {
    double x, y, z, m;
};

// pair force pieces: d = Xa - Xb, returns m-free factors
__device__ __forceinline__ bool pair_kernel(double dx, double dy, double dz, double& ir, double& ir3) {
    double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0) return false;  // coincident particles do not interact
    ir = rsqrt(r2);
    ir3 = ir * ir * ir;
    return true;
}

__global__ void __launch_bounds__(PB) p2p_k(int64_t npairs, const int2* __restrict__ pairs,
                                            const long long* __restrict__ off, const int* __restrict__ nfirst,
                                            const int* __restrict__ ncount, const double* __restrict__ xs,
                                            const double* __restrict__ ys, const double* __restrict__ zs,
                                            const double* __restrict__ ms, double4* __restrict__ part) {
    __shared__ PState sp[PW][32];
    __shared__ double4 sa[PW][32];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t gw = (int64_t)blockIdx.x * PW + w, nw = (int64_t)gridDim.x * PW;
    for (int64_t k = gw; k < npairs; k += nw) {
        int2 pr = pairs[k];
        int A = pr.x, B = pr.y;
        int nA = ncount[A], nB = ncount[B], fA = nfirst[A], fB = nfirst[B];
        long long o = off[k];
        if (A == B && nA <= 32) {
            // ---- self pair
            int n = nA;
            double xi = 0, yi = 0, zi = 0, mi = 0;
            if (lane < n) {
                xi = xs[fA + lane];
                yi = ys[fA + lane];
                zi = zs[fA + lane];
                mi = ms[fA + lane];
                sp[w][lane] = PState{xi, yi, zi, mi};
                sa[w][lane] = make_double4(0, 0, 0, 0);
            }
            __syncwarp();
            double ax = 0, ay = 0, az = 0, ph = 0;
            int half = n / 2;
            for (int s = 1; s <= half; s++) {
                bool act = lane < n && (2 * s < n || lane < half);
                if (act) {
                    int j = lane + s;
                    if (j >= n) j -= n;
                    PState q = sp[w][j];
                    double dx = xi - q.x, dy = yi - q.y, dz = zi - q.z, ir, ir3;
                    if (pair_kernel(dx, dy, dz, ir, ir3)) {
                        double fb = q.m * ir3, fa = mi * ir3;
                        ax -= fb * dx;
                        ay -= fb * dy;
                        az -= fb * dz;
                        ph -= q.m * ir;
                        double4 t = sa[w][j];
                        t.x += fa * dx;
                        t.y += fa * dy;
                        t.z += fa * dz;
                        t.w -= mi * ir;
                        sa[w][j] = t;
                    }
                }
                __syncwarp();
            }
            if (lane < n) {
                double4 t = sa[w][lane];
                part[o + lane] = make_double4(ax + t.x, ay + t.y, az + t.z, ph + t.w);
            }
            __syncwarp();
        } else if (A != B && nA <= 32 && nB <= 32) {
            // ---- distinct leaves: smaller side fixed in lanes, larger side rotating
            bool a_fixed = nA <= nB;
            int nF = a_fixed ? nA : nB, nR = a_fixed ? nB : nA;
            int fF = a_fixed ? fA : fB, fR = a_fixed ? fB : fA;
            long long oF = a_fixed ? o : o + nA, oR = a_fixed ? o + nA : o;
            if (lane < nR) {
                sp[w][lane] = PState{xs[fR + lane], ys[fR + lane], zs[fR + lane], ms[fR + lane]};
                sa[w][lane] = make_double4(0, 0, 0, 0);
            }
            double xi = 0, yi = 0, zi = 0, mi = 0;
            if (lane < nF) {
                xi = xs[fF + lane];
                yi = ys[fF + lane];
                zi = zs[fF + lane];
                mi = ms[fF + lane];
            }
            __syncwarp();
            double ax = 0, ay = 0, az = 0, ph = 0;
            int j = lane;
            for (int s = 0; s < nR; s++) {
                if (lane < nF) {
                    PState q = sp[w][j];
                    double dx = xi - q.x, dy = yi - q.y, dz = zi - q.z, ir, ir3;
                    if (pair_kernel(dx, dy, dz, ir, ir3)) {
                        double fb = q.m * ir3, fa = mi * ir3;
                        ax -= fb * dx;
                        ay -= fb * dy;
                        az -= fb * dz;
                        ph -= q.m * ir;
                        double4 t = sa[w][j];
                        t.x += fa * dx;
                        t.y += fa * dy;
                        t.z += fa * dz;
                        t.w -= mi * ir;
                        sa[w][j] = t;
                    }
                }
                j = (j + 1 == nR) ? 0 : j + 1;
                __syncwarp();
            }
            if (lane < nF) part[oF + lane] = make_double4(ax, ay, az, ph);
            if (lane < nR) part[oR + lane] = sa[w][lane];
            __syncwarp();
        } else {
            // ---- leaves above 32 particles (only at the deepest level): one side at a time
            for (int side = 0; side < (A == B ? 1 : 2); side++) {
                int fT = side ? fB : fA, nT = side ? nB : nA, fS = side ? fA : fB, nS = side ? nA : nB;
                long long oT = side ? o + nA : o;
                for (int t = lane; t < nT; t += 32) {
                    double xi = xs[fT + t], yi = ys[fT + t], zi = zs[fT + t];
                    double ax = 0, ay = 0, az = 0, ph = 0;
                    for (int u = 0; u < nS; u++) {
                        if (A == B && u == t) continue;
                        double dx = xi - xs[fS + u], dy = yi - ys[fS + u], dz = zi - zs[fS + u], ir, ir3;
                        if (pair_kernel(dx, dy, dz, ir, ir3)) {
                            double fb = ms[fS + u] * ir3;
                            ax -= fb * dx;
                            ay -= fb * dy;
                            az -= fb * dz;
                            ph -= ms[fS + u] * ir;
                        }
                    }
                    part[oT + t] = make_double4(ax, ay, az, ph);
                }
            }
        }
    }
}

void run_p2p(fmm_ctx* c, bool want_pot) {
    (void)want_pot;
    cudaStream_t s = c->stream;
    long long total = 0;
    GB_CUDA(cudaMemcpyAsync(&total, c->p2p_off.as<long long>() + c->n_p2p, sizeof(long long),
                            cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    ensure(c->p2p_part, sizeof(double4) * (size_t)(total > 0 ? total : 1));
    int dev_sms = 0;
    GB_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c->device));
    int64_t blocks = (c->n_p2p + PW - 1) / PW;
    int64_t cap = (int64_t)dev_sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    stage_begin(c, ST_P2P);
    p2p_k<<<(unsigned)blocks, PB, 0, s>>>(c->n_p2p, c->p2p_pairs.as<int2>(), c->p2p_off.as<long long>(),
                                          c->nfirst.as<int>(), c->ncount.as<int>(), c->xs.as<double>(),
                                          c->ys.as<double>(), c->zs.as<double>(), c->ms.as<double>(),
                                          c->p2p_part.as<double4>());
    GB_LAUNCH("p2p_k");
    stage_end(c, ST_P2P);
}

// ------------------------------------------------------------------ diagnostics

constexpr int DB = 256;

__device__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = DB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// fixed-order sums of m a and m X x a over sorted particles: per-block tree, then one block
__global__ void diag_partial_k(int n, const double* __restrict__ xs, const double* __restrict__ ys,
                               const double* __restrict__ zs, const double* __restrict__ ms,
                               const double* __restrict__ acc, double* __restrict__ part) {
    __shared__ double sh[DB];
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int i = blockIdx.x * DB + threadIdx.x; i < n; i += gridDim.x * DB) {
        double m = ms[i], ax = acc[i], ay = acc[n + i], az = acc[2 * (int64_t)n + i];
        double x = xs[i], y = ys[i], z = zs[i];
        v[0] += m * ax;
        v[1] += m * ay;
        v[2] += m * az;
        v[3] += m * (y * az - z * ay);
        v[4] += m * (z * ax - x * az);
        v[5] += m * (x * ay - y * ax);
    }
    for (int d = 0; d < 6; d++) {
        double r = block_sum(v[d], sh);
        if (threadIdx.x == 0) part[6 * blockIdx.x + d] = r;
    }
}

__global__ void diag_final_k(int nb, const double* __restrict__ part, double* __restrict__ out) {
    __shared__ double sh[DB];
    for (int d = 0; d < 6; d++) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nb; b += DB) v += part[6 * b + d];
        double r = block_sum(v, sh);
        if (threadIdx.x == 0) out[d] = r;
    }
}

void run_diagnostics(fmm_ctx* c, double* out6) {
    cudaStream_t s = c->stream;
    int n = (int)c->N;
    int nb = (n + DB - 1) / DB;
    if (nb > 592) nb = 592;
    ensure(c->diag_tmp, sizeof(double) * (size_t)(6 * nb + 6));
    double* part = c->diag_tmp.as<double>();
    diag_partial_k<<<nb, DB, 0, s>>>(n, c->xs.as<double>(), c->ys.as<double>(), c->zs.as<double>(),
                                     c->ms.as<double>(), c->acc_s.as<double>(), part);
    GB_LAUNCH("diag_partial_k");
    diag_final_k<<<1, DB, 0, s>>>(nb, part, part + 6 * nb);
    GB_LAUNCH("diag_final_k");
    GB_CUDA(cudaMemcpyAsync(out6, part + 6 * nb, sizeof(double) * 6, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
}

}  // namespace gbfmm
