// a12 mutual particle-particle interactions (eq. jia and its gradient) and a14 diagnostics.
//
// One warp per leaf pair (A, B) of the P2P list (A == B: a leaf with itself).  The
// nA x nB particle pairs are spread flat over the 32 lanes, so lanes stay busy whatever
// the leaf sizes (leaves hold ~10 particles on average): lane t of a round takes pair
// (a, b) = (t / ncol, t % ncol) of a column panel, forms d = X_a - X_b, r^-1 and d r^-3
// and stores them in a shared-memory panel.  Two passes then sum the panel with one lane
// per (particle, component): rows give a_a = -sum_b m_b d r^-3 (phi_a = -sum_b m_b r^-1),
// columns give a_b = +sum_a m_a d r^-3 (phi_b = -sum_a m_a r^-1).  Each pair force is
// formed once and applied to both partners (action = reaction).  A self pair keeps a < b.
// Results go to a per-(pair, side, slot) partial buffer that the final per-particle
// kernels sum in increasing partner id: no floating-point atomics, run-to-run identical.
#include "fmm_device.cuh"
#include "fmm_internal.h"

namespace gbfmm {

constexpr int PB = 128;                 // 4 warps
constexpr int PW = PB / 32;
constexpr int PCOL = 16;                // panel columns
constexpr int PROW = PCOL * 4 + 4;      // doubles per panel row: [col][comp], padded (row stride = 4 mod 16)
constexpr int PANEL = 32 * PROW;        // doubles per warp panel

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

template <bool POT>
__global__ void __launch_bounds__(PB) p2p_k(int64_t npairs, const int2* __restrict__ pairs,
                                            const long long* __restrict__ off, const int* __restrict__ nfirst,
                                            const int* __restrict__ ncount, const double* __restrict__ xs,
                                            const double* __restrict__ ys, const double* __restrict__ zs,
                                            const double* __restrict__ ms, double4* __restrict__ part) {
    extern __shared__ double smem[];
    __shared__ PState sA[PW][32], sB[PW][32];
    __shared__ double4 cacc[PW][32];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* F = smem + (size_t)w * PANEL;
    double* cac = reinterpret_cast<double*>(&cacc[w][0]);
    int64_t gw = (int64_t)blockIdx.x * PW + w, nw = (int64_t)gridDim.x * PW;
    for (int64_t k = gw; k < npairs; k += nw) {
        int2 pr = pairs[k];
        int A = pr.x, B = pr.y;
        int nA = ncount[A], nB = ncount[B], fA = nfirst[A], fB = nfirst[B];
        long long o = off[k];
        bool self = A == B;
        if (nA <= 32 && nB <= 32) {
            if (lane < nA) sA[w][lane] = PState{xs[fA + lane], ys[fA + lane], zs[fA + lane], ms[fA + lane]};
            if (lane < nB) sB[w][lane] = PState{xs[fB + lane], ys[fB + lane], zs[fB + lane], ms[fB + lane]};
            cacc[w][lane] = make_double4(0.0, 0.0, 0.0, 0.0);
            double racc[4] = {0.0, 0.0, 0.0, 0.0};  // row task tau = lane + 32 q: (a, comp) = (tau >> 2, tau & 3)
            __syncwarp();
            for (int cb = 0; cb < nB; cb += PCOL) {
                int ncol = min(PCOL, nB - cb);
                int nint = nA * ncol;
                // pair terms of the panel
                for (int t = lane; t < nint; t += 32) {
                    int a = t / ncol, bl = t - a * ncol, b = cb + bl;
                    double fx = 0.0, fy = 0.0, fz = 0.0, fr = 0.0;
                    if (!self || a < b) {
                        PState pa = sA[w][a], pb = sB[w][b];
                        double dx = pa.x - pb.x, dy = pa.y - pb.y, dz = pa.z - pb.z, ir, ir3;
                        if (pair_kernel(dx, dy, dz, ir, ir3)) {
                            fx = dx * ir3;
                            fy = dy * ir3;
                            fz = dz * ir3;
                            fr = ir;
                        }
                    }
                    double* e = F + a * PROW + bl * 4;
                    reinterpret_cast<double2*>(e)[0] = make_double2(fx, fy);
                    reinterpret_cast<double2*>(e)[1] = make_double2(fz, fr);
                }
                __syncwarp();
                // rows: sum_b m_b F[a][b]
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    int tau = lane + 32 * q, a = tau >> 2, c = tau & 3;
                    if (a < nA && (POT || c < 3)) {
                        const double* row = F + a * PROW + c;
                        double s = racc[q];
                        for (int bl = 0; bl < ncol; bl++) s = fma(sB[w][cb + bl].m, row[bl * 4], s);
                        racc[q] = s;
                    }
                }
                // columns: sum_a m_a F[a][b]
#pragma unroll
                for (int q = 0; q < 2; q++) {
                    int tau = lane + 32 * q, bl = tau >> 2, c = tau & 3;
                    if (bl < ncol && (POT || c < 3)) {
                        const double* col = F + bl * 4 + c;
                        double s = 0.0;
                        for (int a = 0; a < nA; a++) s = fma(sA[w][a].m, col[a * PROW], s);
                        cac[(cb + bl) * 4 + c] += s;
                    }
                }
                __syncwarp();
            }
            // write: rows are a_a = -sum (and phi_a = -sum); columns a_b = +sum, phi_b = -sum
            double* pd = reinterpret_cast<double*>(part);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                int tau = lane + 32 * q, a = tau >> 2, c = tau & 3;
                if (a < nA) {
                    double v = -racc[q];
                    if (self) v += (c < 3) ? cac[a * 4 + c] : -cac[a * 4 + c];
                    pd[(o + a) * 4 + c] = (POT || c < 3) ? v : 0.0;
                }
            }
            if (!self) {
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    int tau = lane + 32 * q, b = tau >> 2, c = tau & 3;
                    if (b < nB) {
                        double v = cac[b * 4 + c];
                        pd[(o + nA + b) * 4 + c] = (c < 3) ? v : (POT ? -v : 0.0);
                    }
                }
            }
            __syncwarp();
        } else {
            // ---- leaves above 32 particles (only at the deepest level): one side at a time
            for (int side = 0; side < (self ? 1 : 2); side++) {
                int fT = side ? fB : fA, nT = side ? nB : nA, fS = side ? fA : fB, nS = side ? nA : nB;
                long long oT = side ? o + nA : o;
                for (int t = lane; t < nT; t += 32) {
                    double xi = xs[fT + t], yi = ys[fT + t], zi = zs[fT + t];
                    double ax = 0, ay = 0, az = 0, ph = 0;
                    for (int u = 0; u < nS; u++) {
                        if (self && u == t) continue;
                        double dx = xi - xs[fS + u], dy = yi - ys[fS + u], dz = zi - zs[fS + u], ir, ir3;
                        if (pair_kernel(dx, dy, dz, ir, ir3)) {
                            double fb = ms[fS + u] * ir3;
                            ax -= fb * dx;
                            ay -= fb * dy;
                            az -= fb * dz;
                            ph -= ms[fS + u] * ir;
                        }
                    }
                    part[oT + t] = make_double4(ax, ay, az, POT ? ph : 0.0);
                }
            }
        }
    }
}

void run_p2p(fmm_ctx* c, bool want_pot) {
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
    size_t shm = sizeof(double) * (size_t)PANEL * PW;
    auto kern = want_pot ? p2p_k<true> : p2p_k<false>;
    GB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    kern<<<(unsigned)blocks, PB, shm, s>>>(c->n_p2p, c->p2p_pairs.as<int2>(), c->p2p_off.as<long long>(),
                                           c->nfirst.as<int>(), c->ncount.as<int>(), c->xs.as<double>(),
                                           c->ys.as<double>(), c->zs.as<double>(), c->ms.as<double>(),
                                           c->p2p_part.as<double4>());
    GB_LAUNCH("p2p_k");
    stage_end(c, ST_P2P);
}

// a12/a13 first level: one warp per P2P work item (up to P2P_CHUNK directed entries of
// one leaf); lane = particle slot of the leaf.  Sums the per-pair partials of the
// item's entries (increasing partner id) into ipart[islot[item] + slot].
//   part[] holds double4 (ax, ay, az, phi) per (pair, side, slot); pair k's block starts
//   at off[k]: first the slots of pairs[k].x, then (if distinct) those of pairs[k].y.
__global__ void __launch_bounds__(PB) p2p_gather_k(int64_t nitems, const int4* __restrict__ items,
                                                   const int* __restrict__ ncount, const uint32_t* __restrict__ pdval,
                                                   const int2* __restrict__ pairs, const long long* __restrict__ poff,
                                                   const double4* __restrict__ part,
                                                   const long long* __restrict__ islot, double4* __restrict__ ipart) {
    int64_t it = ((int64_t)blockIdx.x * PB + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (it >= nitems) return;
    int4 w = items[it];
    int cnt = ncount[w.x];
    for (int slot = lane; slot < cnt; slot += 32) {
        double px = 0.0, py = 0.0, pz = 0.0, pp = 0.0;
        for (int e = w.y; e < w.z; e++) {
            uint32_t v = pdval[e];
            uint32_t k = v >> 1;
            long long o = poff[k] + ((v & 1u) ? (long long)ncount[pairs[k].x] : 0ll) + slot;
            double4 q = part[o];
            px += q.x;
            py += q.y;
            pz += q.z;
            pp += q.w;
        }
        ipart[islot[it] + slot] = make_double4(px, py, pz, pp);
    }
}

// slot offsets of the P2P items: islot[i] = sum of the leaf sizes of items before i
__global__ void item_slots_k(int64_t nitems, const int4* __restrict__ items, const int* __restrict__ ncount,
                             long long* __restrict__ sizes) {
    int64_t i = (int64_t)blockIdx.x * PB + threadIdx.x;
    if (i < nitems) sizes[i] = ncount[items[i].x];
}

void run_p2p_gather(fmm_ctx* c) {
    cudaStream_t s = c->stream;
    const ItemSet& it = c->p2p_items;
    int64_t ni = it.n_items;
    ensure(c->p2p_islot, sizeof(long long) * (size_t)(ni + 1));
    ensure(c->flags, sizeof(long long) * (size_t)(ni + 1));
    item_slots_k<<<grid_for(ni, PB), PB, 0, s>>>(ni, it.items.as<int4>(), c->ncount.as<int>(), c->flags.as<long long>());
    GB_LAUNCH("item_slots_k");
    scan_i64_from_i64(c, c->flags.as<long long>(), ni, c->p2p_islot.as<long long>());
    long long nslots = 0;
    GB_CUDA(cudaMemcpyAsync(&nslots, c->p2p_islot.as<long long>() + ni, sizeof(long long), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    ensure(c->p2p_ipart, sizeof(double4) * (size_t)(nslots > 0 ? nslots : 1));
    p2p_gather_k<<<grid_for(ni * 32, PB), PB, 0, s>>>(ni, it.items.as<int4>(), c->ncount.as<int>(),
                                                       c->p2p_dval.as<uint32_t>(), c->p2p_pairs.as<int2>(),
                                                       c->p2p_off.as<long long>(), c->p2p_part.as<double4>(),
                                                       c->p2p_islot.as<long long>(), c->p2p_ipart.as<double4>());
    GB_LAUNCH("p2p_gather_k");
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
