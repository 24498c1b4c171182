// Expansion kernels of order P (included once per P by the generated expansion_p*.cu):
// P2M, M2M (upward pass), target-major M2L, L2L (downward pass) and the final
// per-particle kernel (L2P + P2P partial reduction + return to input order).
//
// Layouts (device, node ids breadth-first):
//   mom[n * NM + k]     raw moments M_alpha about Z_n, alpha in generated order
//   loc[n * NM + k]     standard locals L_gamma                       (variant 0)
//   loc[n * NSU + k]    conserving locals [S | Ux | Uy | Uz]          (variant 1)
//   m2l_dir[e]          directed entry tgt << bits | src, sorted; m2l_seg[n] = first entry of n
#pragma once
#include "fmm_device.cuh"
#include "fmm_internal.h"
#include "fmm_math.cuh"
#include "prec.cuh"

namespace gbfmm {

constexpr int EB = 128;

// a5 P2M: moments of every leaf from its particles (y = X - Z)
template <int P>
__global__ void __launch_bounds__(EB) p2m_k(int nn, const int* __restrict__ nfirst, const int* __restrict__ ncount,
                                            const int* __restrict__ nnchild, const double* __restrict__ xs,
                                            const double* __restrict__ ys, const double* __restrict__ zs,
                                            const double* __restrict__ ms, const double* __restrict__ Zx,
                                            const double* __restrict__ Zy, const double* __restrict__ Zz,
                                            double* __restrict__ mom) {
    using E = Exp<P>;
    int nd = blockIdx.x * EB + threadIdx.x;
    if (nd >= nn || nnchild[nd] != 0) return;
    double M[E::NM];
#pragma unroll
    for (int k = 0; k < E::NM; k++) M[k] = 0.0;
    double zx = Zx[nd], zy = Zy[nd], zz = Zz[nd];
    int f = nfirst[nd], e = f + ncount[nd];
    for (int i = f; i < e; i++) E::p2m(ms[i], xs[i] - zx, ys[i] - zy, zs[i] - zz, M);
#pragma unroll
    for (int k = 0; k < E::NM; k++) mom[(int64_t)nd * E::NM + k] = M[k];
}


// a8 M2L, standard, one work item = up to M2L_CHUNK directed entries of one target cell
// (sources in increasing id): L_gamma += sum_beta M_beta D_{beta+gamma}(Z_tgt - Z_src),
// in the pair-kernel type T; centres are stored as S = Prec<T>::S and R is formed in S.
// The item's partial local goes to part[item]; m2l_reduce_k sums a cell's items in order.
template <int P, class T>
__global__ void __launch_bounds__(EB) m2l_std_k(int64_t nitems, const int4* __restrict__ items,
                                                const uint64_t* __restrict__ dir, int bits,
                                                const double* __restrict__ Zx, const double* __restrict__ Zy,
                                                const double* __restrict__ Zz,
                                                const T* __restrict__ mom, T* __restrict__ part) {
    using E = Exp<P>;
    int64_t it = (int64_t)blockIdx.x * EB + threadIdx.x;
    if (it >= nitems) return;
    int4 w = items[it];
    T L[E::NM];
#pragma unroll
    for (int k = 0; k < E::NM; k++) L[k] = T(0);
    double zx = Zx[w.x], zy = Zy[w.x], zz = Zz[w.x];
    uint64_t mask = (1ull << bits) - 1ull;
    for (int e = w.y; e < w.z; e++) {
        int src = (int)(dir[e] & mask);
        // R = Z_tgt - Z_src in binary64, then narrowed to the kernel type
        T rx = to_kernel(zx - Zx[src], T()), ry = to_kernel(zy - Zy[src], T()), rz = to_kernel(zz - Zz[src], T());
        T D[E::NM];
        E::dtensor(rx, ry, rz, D);
        E::m2l_std(mom + (int64_t)src * E::NM, D, L);
    }
#pragma unroll
    for (int k = 0; k < E::NM; k++) part[it * E::NM + k] = Prec<T>::fin(L[k]);
}

// a8' M2L, conserving: S and U of the realigned pair forces, from conserving moments
template <int P, class T>
__global__ void __launch_bounds__(EB) m2l_con_k(int64_t nitems, const int4* __restrict__ items,
                                                const uint64_t* __restrict__ dir, int bits,
                                                const double* __restrict__ Zx, const double* __restrict__ Zy,
                                                const double* __restrict__ Zz,
                                                const T* __restrict__ cmom, T* __restrict__ part) {
    using E = Exp<P>;
    int64_t it = (int64_t)blockIdx.x * EB + threadIdx.x;
    if (it >= nitems) return;
    int4 w = items[it];
    T SU[E::NSU];
#pragma unroll
    for (int k = 0; k < E::NSU; k++) SU[k] = T(0);
    double zx = Zx[w.x], zy = Zy[w.x], zz = Zz[w.x];
    uint64_t mask = (1ull << bits) - 1ull;
    for (int e = w.y; e < w.z; e++) {
        int src = (int)(dir[e] & mask);
        // R = Z_tgt - Z_src in binary64, then narrowed to the kernel type
        T rx = to_kernel(zx - Zx[src], T()), ry = to_kernel(zy - Zy[src], T()), rz = to_kernel(zz - Zz[src], T());
        T H[E::NQ];
        E::htensor(rx, ry, rz, H);
        if constexpr (sizeof(T) == 4) {
            // binary32: the source block (4 nmi(p-1) floats, a multiple of 4) in 16-byte loads
            T Cs[E::NSU];
            const float4* src4 = reinterpret_cast<const float4*>(cmom + (int64_t)src * E::NSU);
#pragma unroll
            for (int k = 0; k < E::NSU / 4; k++) {
                float4 v = src4[k];
                Cs[4 * k] = v.x;
                Cs[4 * k + 1] = v.y;
                Cs[4 * k + 2] = v.z;
                Cs[4 * k + 3] = v.w;
            }
            E::m2l_con(Cs, H, rx, ry, rz, SU);
        } else {
            E::m2l_con(cmom + (int64_t)src * E::NSU, H, rx, ry, rz, SU);
        }
    }
#pragma unroll
    for (int k = 0; k < E::NSU; k++) part[it * E::NSU + k] = Prec<T>::fin(SU[k]);
}

// a9: loc[x][k] = sum over the cell's items (full chunks in order, then the partial one),
// accumulated in binary64
__device__ __forceinline__ double as_double(double v) { return v; }
__device__ __forceinline__ double as_double(float v) { return (double)v; }
__device__ __forceinline__ double as_double(df64 v) { return to_double(v); }

template <int NL, class T>
__global__ void m2l_reduce_k(int nn, const long long* __restrict__ fo, const long long* __restrict__ po,
                             long long nfull, const T* __restrict__ part, double* __restrict__ loc) {
    int64_t t = (int64_t)blockIdx.x * EB + threadIdx.x;
    if (t >= (int64_t)nn * NL) return;
    int x = (int)(t / NL), k = (int)(t - (int64_t)x * NL);
    double acc = 0.0;
    for (long long i = fo[x]; i < fo[x + 1]; i++) acc += as_double(part[i * NL + k]);
    if (po[x + 1] > po[x]) acc += as_double(part[(nfull + po[x]) * NL + k]);
    loc[t] = acc;
}

// binary64 arrays converted to the pair-kernel / storage types
template <class T>
__global__ void convert_k(int64_t n, const double* __restrict__ in, T* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * EB + threadIdx.x;
    if (i < n) out[i] = to_kernel(in[i], T());
}

// conserving source moments of every cell (formed once per moment build)
template <int P>
__global__ void __launch_bounds__(EB) con_moments_k(int nn, const double* __restrict__ mom, double* __restrict__ cmom) {
    using E = Exp<P>;
    int nd = blockIdx.x * EB + threadIdx.x;
    if (nd >= nn) return;
    double C[E::NSU];
    E::con_moments(mom + (int64_t)nd * E::NM, C);
#pragma unroll
    for (int k = 0; k < E::NSU; k++) cmom[(int64_t)nd * E::NSU + k] = C[k];
}

// ---- coefficient-parallel translations: one warp per node, lanes over output coefficients.
// On GB300 a warp's binary64 instructions issue at one per 16 SM cycles, so a level whose
// threads each run a long serial chain takes the chain's length in time; spreading the
// coefficients over lanes shortens every chain ~NM-fold.

// position of multi-index (ax, ay, az) in the degree-major order (ax, then ay descending)
__device__ __forceinline__ int mi_index(int ax, int ay, int az) {
    int n = ax + ay + az, j = n - ax;
    return n * (n + 1) * (n + 2) / 6 + j * (j + 1) / 2 + (j - ay);
}

__device__ __forceinline__ void mi_decode(int k, int& ax, int& ay, int& az) {
    int n = 0;
    while ((n + 1) * (n + 2) * (n + 3) / 6 <= k) n++;
    int rem = k - n * (n + 1) * (n + 2) / 6, j = 0;
    while ((j + 1) * (j + 2) / 2 <= rem) j++;
    ay = j - (rem - j * (j + 1) / 2);
    ax = n - j;
    az = n - ax - ay;
}

// 1/e for the small integers of factorials (constants, no binary64 division)
__device__ __forceinline__ double recip_small(int e) {
    return e == 1 ? 1.0 : e == 2 ? 0.5 : e == 3 ? 1.0 / 3.0 : e == 4 ? 0.25 : e == 5 ? 0.2 : e == 6 ? 1.0 / 6.0
         : e == 7 ? 1.0 / 7.0 : 0.125;
}

// w[b] = v^b / b! for |b| <= p, written by the warp's lanes into shared memory
template <int NMP>
__device__ __forceinline__ void fill_mono(double vx, double vy, double vz, double* w, int lane) {
    for (int k = lane; k < NMP; k += 32) {
        int bx, by, bz;
        mi_decode(k, bx, by, bz);
        double t = 1.0;
        for (int e = 1; e <= bx; e++) t *= vx * recip_small(e);
        for (int e = 1; e <= by; e++) t *= vy * recip_small(e);
        for (int e = 1; e <= bz; e++) t *= vz * recip_small(e);
        w[k] = t;
    }
}

constexpr int TWB = 128;  // translation blocks: 4 warps
constexpr int TWW = TWB / 32;

// Dependent binary64 instructions are slow to retire on GB300, so every lane keeps
// several independent accumulators (one per child for M2M, four interleaved partial
// sums for L2L) and adds them in a fixed order at the end.

// a6 M2M: M^P_alpha = sum_children sum_{beta<=alpha} M^c_{alpha-beta} (-c)^beta/beta!
template <int P>
__global__ void __launch_bounds__(TWB) m2m_warp_k(int lo, int hi, const int* __restrict__ nchildf,
                                                  const int* __restrict__ nnchild, const double* __restrict__ Zx,
                                                  const double* __restrict__ Zy, const double* __restrict__ Zz,
                                                  double* __restrict__ mom) {
    using E = Exp<P>;
    constexpr int NM = E::NM, PER = (NM + 31) / 32;
    __shared__ double ws[TWW][8][NM];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int nd = lo + (int)(((int64_t)blockIdx.x * TWB + threadIdx.x) >> 5);
    if (nd >= hi || nnchild[nd] == 0) return;  // warp-uniform
    int c0 = nchildf[nd], nc = nnchild[nd];
    double zx = Zx[nd], zy = Zy[nd], zz = Zz[nd];
    // monomials (-c)^b / b! of every child
    for (int t = lane; t < nc * NM; t += 32) {
        int ch = t / NM, k = t - ch * NM;
        int bx, by, bz;
        mi_decode(k, bx, by, bz);
        double vx = -(Zx[c0 + ch] - zx), vy = -(Zy[c0 + ch] - zy), vz = -(Zz[c0 + ch] - zz);
        double tx = 1.0, ty = 1.0, tz = 1.0;
        for (int e = 1; e <= bx; e++) tx *= vx * recip_small(e);
        for (int e = 1; e <= by; e++) ty *= vy * recip_small(e);
        for (int e = 1; e <= bz; e++) tz *= vz * recip_small(e);
        ws[w][ch][k] = tx * ty * tz;
    }
    __syncwarp();
    const double* Mc = mom + (int64_t)c0 * NM;
#pragma unroll
    for (int q = 0; q < PER; q++) {
        int k = lane + 32 * q;
        if (k < NM) {
            int ax, ay, az;
            mi_decode(k, ax, ay, az);
            double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            for (int bx = 0; bx <= ax; bx++)
                for (int by = 0; by <= ay; by++)
                    for (int bz = 0; bz <= az; bz++) {
                        int r = mi_index(ax - bx, ay - by, az - bz), b = mi_index(bx, by, bz);
#pragma unroll
                        for (int ch = 0; ch < 8; ch++)
                            if (ch < nc) acc[ch] = fma(Mc[(int64_t)ch * NM + r], ws[w][ch][b], acc[ch]);
                    }
            mom[(int64_t)nd * NM + k] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
        }
    }
}

// a10 L2L standard: L_child[g] += sum_{|g+b|<=p} L_parent[g+b] s^b/b!, s = Z_child - Z_parent
template <int P>
__global__ void __launch_bounds__(TWB) l2l_std_warp_k(int lo, int hi, const int* __restrict__ nparent,
                                                      const double* __restrict__ Zx, const double* __restrict__ Zy,
                                                      const double* __restrict__ Zz, double* __restrict__ loc) {
    using E = Exp<P>;
    constexpr int NM = E::NM, PER = (NM + 31) / 32;
    __shared__ double ws[TWW][NM];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int nd = lo + (int)(((int64_t)blockIdx.x * TWB + threadIdx.x) >> 5);
    if (nd >= hi) return;
    int par = nparent[nd];
    fill_mono<NM>(Zx[nd] - Zx[par], Zy[nd] - Zy[par], Zz[nd] - Zz[par], ws[w], lane);
    __syncwarp();
    const double* Lp = loc + (int64_t)par * NM;
#pragma unroll
    for (int q = 0; q < PER; q++) {
        int k = lane + 32 * q;
        if (k < NM) {
            int gx, gy, gz;
            mi_decode(k, gx, gy, gz);
            int rem = P - (gx + gy + gz);
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            int j = 0;
            for (int bx = 0; bx <= rem; bx++)
                for (int by = 0; by <= rem - bx; by++)
                    for (int bz = 0; bz <= rem - bx - by; bz++, j++)
                        acc[j & 3] = fma(Lp[mi_index(gx + bx, gy + by, gz + bz)], ws[w][mi_index(bx, by, bz)], acc[j & 3]);
            loc[(int64_t)nd * NM + k] += (acc[0] + acc[1]) + (acc[2] + acc[3]);
        }
    }
}

// a10 L2L conserving: S' = shift(S), U'_i = shift(U_i) + s_i shift(S) (degree p-1)
template <int P>
__global__ void __launch_bounds__(TWB) l2l_con_warp_k(int lo, int hi, const int* __restrict__ nparent,
                                                      const double* __restrict__ Zx, const double* __restrict__ Zy,
                                                      const double* __restrict__ Zz, double* __restrict__ loc) {
    using E = Exp<P>;
    constexpr int NQ = E::NQ, NSU = E::NSU, PER = (NSU + 31) / 32, Q = P - 1;
    __shared__ double ws[TWW][NQ];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int nd = lo + (int)(((int64_t)blockIdx.x * TWB + threadIdx.x) >> 5);
    if (nd >= hi) return;
    int par = nparent[nd];
    double sv[3] = {Zx[nd] - Zx[par], Zy[nd] - Zy[par], Zz[nd] - Zz[par]};
    fill_mono<NQ>(sv[0], sv[1], sv[2], ws[w], lane);
    __syncwarp();
    const double* Lp = loc + (int64_t)par * NSU;
#pragma unroll
    for (int q = 0; q < PER; q++) {
        int t = lane + 32 * q;
        if (t < NSU) {
            int comp = t / NQ, k = t - comp * NQ;
            int gx, gy, gz;
            mi_decode(k, gx, gy, gz);
            int rem = Q - (gx + gy + gz);
            double sh[2] = {0.0, 0.0}, su[2] = {0.0, 0.0};
            int j = 0;
            for (int bx = 0; bx <= rem; bx++)
                for (int by = 0; by <= rem - bx; by++)
                    for (int bz = 0; bz <= rem - bx - by; bz++, j++) {
                        int src = mi_index(gx + bx, gy + by, gz + bz);
                        double wb = ws[w][mi_index(bx, by, bz)];
                        sh[j & 1] = fma(Lp[src], wb, sh[j & 1]);
                        if (comp > 0) su[j & 1] = fma(Lp[comp * NQ + src], wb, su[j & 1]);
                    }
            double shv = sh[0] + sh[1], suv = su[0] + su[1];
            loc[(int64_t)nd * NSU + t] += (comp == 0 ? shv : fma(sv[comp - 1], shv, suv));
        }
    }
}

// a11 + a13: far field at every particle from its leaf's locals, plus the leaf's P2P item
// sums (full chunks in order, then the partial one), written in input order.
template <int P, int V, class G>
__global__ void __launch_bounds__(EB) finish_k(int n, const int* __restrict__ leaf_of, const int* __restrict__ nfirst,
                                               const double* __restrict__ xs, const double* __restrict__ ys,
                                               const double* __restrict__ zs, const double* __restrict__ Zx,
                                               const double* __restrict__ Zy, const double* __restrict__ Zz,
                                               const double* __restrict__ loc, const double* __restrict__ locp,
                                               const long long* __restrict__ fo, const long long* __restrict__ po,
                                               long long nfull, const long long* __restrict__ islot,
                                               const Quad<G>* __restrict__ ipart, const uint32_t* __restrict__ perm,
                                               double* __restrict__ acc_s, double* __restrict__ pot_s,
                                               double* __restrict__ acc_out, double* __restrict__ pot_out) {
    using E = Exp<P>;
    int i = blockIdx.x * EB + threadIdx.x;
    if (i >= n) return;
    int lf = leaf_of[i];
    int slot = i - nfirst[lf];
    double x = xs[i] - Zx[lf], y = ys[i] - Zy[lf], z = zs[i] - Zz[lf];
    double ax, ay, az, ph = 0.0;
    if (V == 0) {
        E::l2p_std(loc + (int64_t)lf * E::NM, x, y, z, ax, ay, az, ph);
    } else {
        E::l2p_con(loc + (int64_t)lf * E::NSU, x, y, z, ax, ay, az);
        if (locp) {
            double bx, by, bz;
            E::l2p_std(locp + (int64_t)lf * E::NM, x, y, z, bx, by, bz, ph);
        }
    }
    double px = 0.0, py = 0.0, pz = 0.0, pp = 0.0;
    for (long long k = fo[lf]; k < fo[lf + 1]; k++) {
        Quad<G> q = ipart[islot[k] + slot];
        px += as_double(q.x);
        py += as_double(q.y);
        pz += as_double(q.z);
        pp += as_double(q.w);
    }
    if (po[lf + 1] > po[lf]) {
        Quad<G> q = ipart[islot[nfull + po[lf]] + slot];
        px += as_double(q.x);
        py += as_double(q.y);
        pz += as_double(q.z);
        pp += as_double(q.w);
    }
    ax += px;
    ay += py;
    az += pz;
    ph += pp;
    acc_s[i] = ax;
    acc_s[n + i] = ay;
    acc_s[2 * (int64_t)n + i] = az;
    int64_t j = perm[i];
    acc_out[3 * j] = ax;
    acc_out[3 * j + 1] = ay;
    acc_out[3 * j + 2] = az;
    if (pot_out) {
        pot_s[i] = ph;
        pot_out[j] = ph;
    }
}

// host side, one order P
template <int P>
void run_moments_p(fmm_ctx* c) {
    using E = Exp<P>;
    cudaStream_t s = c->stream;
    int nn = (int)c->n_nodes;
    ensure(c->mom, sizeof(double) * (size_t)nn * E::NM);
    p2m_k<P><<<grid_for(nn, EB), EB, 0, s>>>(nn, c->nfirst.as<int>(), c->ncount.as<int>(), c->nnchild.as<int>(),
                                             c->xs.as<double>(), c->ys.as<double>(), c->zs.as<double>(),
                                             c->ms.as<double>(), c->nZx.as<double>(), c->nZy.as<double>(),
                                             c->nZz.as<double>(), c->mom.as<double>());
    GB_LAUNCH("p2m_k");
    for (int l = c->n_levels - 2; l >= 0; l--) {
        int lo = c->level_start[l], hi = c->level_start[l + 1];
        m2m_warp_k<P><<<grid_for((int64_t)(hi - lo) * 32, TWB), TWB, 0, s>>>(
            lo, hi, c->nchildf.as<int>(), c->nnchild.as<int>(), c->nZx.as<double>(), c->nZy.as<double>(),
            c->nZz.as<double>(), c->mom.as<double>());
        GB_LAUNCH("m2m_warp_k");
    }
    ensure(c->cmom, sizeof(double) * (size_t)nn * E::NSU);
    con_moments_k<P><<<grid_for(nn, EB), EB, 0, s>>>(nn, c->mom.as<double>(), c->cmom.as<double>());
    GB_LAUNCH("con_moments_k");
    // moments in the pair-kernel type
    if (c->precision != FMM_FP64) {
        int64_t nm = (int64_t)nn * E::NM, nc = (int64_t)nn * E::NSU;
        if (c->precision == FMM_DF64) {
            ensure(c->momT, sizeof(df64) * (size_t)nm);
            ensure(c->cmomT, sizeof(df64) * (size_t)nc);
            convert_k<df64><<<grid_for(nm, EB), EB, 0, s>>>(nm, c->mom.as<double>(), c->momT.as<df64>());
            convert_k<df64><<<grid_for(nc, EB), EB, 0, s>>>(nc, c->cmom.as<double>(), c->cmomT.as<df64>());
        } else {
            ensure(c->momT, sizeof(float) * (size_t)nm);
            ensure(c->cmomT, sizeof(float) * (size_t)nc);
            convert_k<float><<<grid_for(nm, EB), EB, 0, s>>>(nm, c->mom.as<double>(), c->momT.as<float>());
            convert_k<float><<<grid_for(nc, EB), EB, 0, s>>>(nc, c->cmom.as<double>(), c->cmomT.as<float>());
        }
        GB_LAUNCH("convert_k");
    }
}

template <int P, class T>
void m2l_launch(fmm_ctx* c, int variant, bool std_locals) {
    using E = Exp<P>;
    cudaStream_t s = c->stream;
    int nn = (int)c->n_nodes;
    const uint64_t* dir = c->m2l_dir.as<uint64_t>();
    const ItemSet& it = c->m2l_items;
    int64_t ni = it.n_items;
    bool native = c->precision == FMM_FP64;
    const T* mom = native ? c->mom.as<T>() : c->momT.as<T>();
    const T* cmom = native ? c->cmom.as<T>() : c->cmomT.as<T>();
    const double *zx = c->nZx.as<double>(), *zy = c->nZy.as<double>(), *zz = c->nZz.as<double>();
    int nl_max = E::NSU > E::NM ? E::NSU : E::NM;
    ensure(c->m2l_part, sizeof(T) * (size_t)(ni > 0 ? ni : 1) * nl_max);
    T* part = c->m2l_part.as<T>();
    if (variant == 1) {
        ensure(c->loc, sizeof(double) * (size_t)nn * E::NSU);
        if (ni > 0) {
            m2l_con_k<P, T><<<grid_for(ni, EB), EB, 0, s>>>(ni, it.items.as<int4>(), dir, c->id_bits, zx, zy, zz, cmom,
                                                            part);
            GB_LAUNCH("m2l_con_k");
        }
        m2l_reduce_k<E::NSU, T><<<grid_for((int64_t)nn * E::NSU, EB), EB, 0, s>>>(
            nn, it.fo.as<long long>(), it.po.as<long long>(), it.n_full, part, c->loc.as<double>());
        GB_LAUNCH("m2l_reduce_k");
    }
    if (std_locals) {
        DevBuf& L = variant == 0 ? c->loc : c->locp;
        ensure(L, sizeof(double) * (size_t)nn * E::NM);
        if (ni > 0) {
            m2l_std_k<P, T><<<grid_for(ni, EB), EB, 0, s>>>(ni, it.items.as<int4>(), dir, c->id_bits, zx, zy, zz, mom,
                                                            part);
            GB_LAUNCH("m2l_std_k");
        }
        m2l_reduce_k<E::NM, T><<<grid_for((int64_t)nn * E::NM, EB), EB, 0, s>>>(
            nn, it.fo.as<long long>(), it.po.as<long long>(), it.n_full, part, L.as<double>());
        GB_LAUNCH("m2l_reduce_k");
    }
}

template <int P>
void run_far_field_p(fmm_ctx* c, int variant, bool want_pot) {
    cudaStream_t s = c->stream;
    bool std_locals = (variant == 0) || want_pot;
    stage_begin(c, ST_M2L);
    if (c->precision == FMM_FP64)
        m2l_launch<P, double>(c, variant, std_locals);
    else if (c->precision == FMM_DF64) {
        if constexpr (P <= FMM_DF64_P_MAX) m2l_launch<P, df64>(c, variant, std_locals);
    } else
        m2l_launch<P, float>(c, variant, std_locals);
    stage_end(c, ST_M2L);
    stage_begin(c, ST_L2L);
    for (int l = 1; l < c->n_levels; l++) {
        int lo = c->level_start[l], hi = c->level_start[l + 1];
        if (variant == 1) {
            l2l_con_warp_k<P><<<grid_for((int64_t)(hi - lo) * 32, TWB), TWB, 0, s>>>(
                lo, hi, c->nparent.as<int>(), c->nZx.as<double>(), c->nZy.as<double>(), c->nZz.as<double>(),
                c->loc.as<double>());
            GB_LAUNCH("l2l_con_warp_k");
        }
        if (std_locals) {
            DevBuf& L = variant == 0 ? c->loc : c->locp;
            l2l_std_warp_k<P><<<grid_for((int64_t)(hi - lo) * 32, TWB), TWB, 0, s>>>(
                lo, hi, c->nparent.as<int>(), c->nZx.as<double>(), c->nZy.as<double>(), c->nZz.as<double>(),
                L.as<double>());
            GB_LAUNCH("l2l_std_warp_k");
        }
    }
    stage_end(c, ST_L2L);
}

template <int P, class G>
static void finish_launch(fmm_ctx* c, int variant, bool want_pot, double* acc_out, double* pot_out) {
    cudaStream_t s = c->stream;
    int n = (int)c->N;
    const ItemSet& it = c->p2p_items;
    const double* locp = (variant == 1 && want_pot) ? c->locp.as<double>() : nullptr;
    auto args = [&](auto kern) {
        kern<<<grid_for(n, EB), EB, 0, s>>>(
            n, c->leaf_of.as<int>(), c->nfirst.as<int>(), c->xs.as<double>(), c->ys.as<double>(), c->zs.as<double>(),
            c->nZx.as<double>(), c->nZy.as<double>(), c->nZz.as<double>(), c->loc.as<double>(), locp,
            it.fo.as<long long>(), it.po.as<long long>(), it.n_full, c->p2p_islot.as<long long>(),
            c->p2p_ipart.as<Quad<G>>(), c->perm.as<uint32_t>(), c->acc_s.as<double>(), c->pot_s.as<double>(), acc_out,
            want_pot ? pot_out : nullptr);
    };
    if (variant == 0)
        args(finish_k<P, 0, G>);
    else
        args(finish_k<P, 1, G>);
    GB_LAUNCH("finish_k");
}

template <int P>
void run_finish_p(fmm_ctx* c, int variant, bool want_pot, double* acc_out, double* pot_out) {
    if (c->precision == FMM_FP64)
        finish_launch<P, double>(c, variant, want_pot, acc_out, pot_out);
    else
        finish_launch<P, df64>(c, variant, want_pot, acc_out, pot_out);
}

// One translation unit per order instantiates the order's stages; the M2L launches of
// each arithmetic type get translation units of their own (compiled in parallel).
#define GBFMM_INSTANTIATE(P)                                                                             \
    extern template void m2l_launch<P, double>(fmm_ctx*, int, bool);                                    \
    extern template void m2l_launch<P, float>(fmm_ctx*, int, bool);                                     \
    extern template void m2l_launch<P, df64>(fmm_ctx*, int, bool);                                      \
    template void run_moments_p<P>(fmm_ctx*);                                                           \
    template void run_far_field_p<P>(fmm_ctx*, int, bool);                                              \
    template void run_finish_p<P>(fmm_ctx*, int, bool, double*, double*);

#define GBFMM_INSTANTIATE_M2L(P, T) template void m2l_launch<P, T>(fmm_ctx*, int, bool);

}  // namespace gbfmm
