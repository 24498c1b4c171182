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

// a6 M2M in two steps per level: one thread per (parent, child) shifts the child's
// moments to the parent centre (straight-line, independent accumulators), then one thread
// per (parent, coefficient) adds the children's shifted moments in child order.  A single
// thread per parent would run one long binary64 chain per level, which on GB300 sets the
// level's time.
template <int P>
__global__ void __launch_bounds__(EB) m2m_child_k(int lo, int hi, int cfirst, const int* __restrict__ nparent,
                                                  const double* __restrict__ Zx, const double* __restrict__ Zy,
                                                  const double* __restrict__ Zz, const double* __restrict__ mom,
                                                  double* __restrict__ shifted) {
    using E = Exp<P>;
    // children of the parents in [lo, hi) are the nodes [cfirst, cfirst + gridDim-covered)
    int ch = cfirst + blockIdx.x * EB + threadIdx.x;
    if (ch >= hi) return;
    int par = nparent[ch];
    double M[E::NM];
#pragma unroll
    for (int k = 0; k < E::NM; k++) M[k] = 0.0;
    E::m2m(mom + (int64_t)ch * E::NM, Zx[ch] - Zx[par], Zy[ch] - Zy[par], Zz[ch] - Zz[par], M);
#pragma unroll
    for (int k = 0; k < E::NM; k++) shifted[(int64_t)(ch - cfirst) * E::NM + k] = M[k];
    (void)lo;
}

template <int P>
__global__ void m2m_sum_k(int lo, int hi, int cfirst, const int* __restrict__ nchildf, const int* __restrict__ nnchild,
                          const double* __restrict__ shifted, double* __restrict__ mom) {
    using E = Exp<P>;
    int64_t t = (int64_t)blockIdx.x * EB + threadIdx.x;
    if (t >= (int64_t)(hi - lo) * E::NM) return;
    int nd = lo + (int)(t / E::NM), k = (int)(t - (int64_t)(nd - lo) * E::NM);
    int nc = nnchild[nd];
    if (nc == 0) return;
    int c0 = nchildf[nd] - cfirst;
    double s = 0.0;
    for (int c = 0; c < nc; c++) s += shifted[(int64_t)(c0 + c) * E::NM + k];
    mom[(int64_t)nd * E::NM + k] = s;
}

// a10 L2L, one level: child += shift(parent) by s = Z_child - Z_parent
template <int P>
__global__ void __launch_bounds__(EB) l2l_std_k(int lo, int hi, const int* __restrict__ nparent,
                                                const double* __restrict__ Zx, const double* __restrict__ Zy,
                                                const double* __restrict__ Zz, double* __restrict__ loc) {
    using E = Exp<P>;
    int nd = lo + blockIdx.x * EB + threadIdx.x;
    if (nd >= hi) return;
    int par = nparent[nd];
    double L[E::NM];
#pragma unroll
    for (int k = 0; k < E::NM; k++) L[k] = loc[(int64_t)nd * E::NM + k];
    E::l2l(loc + (int64_t)par * E::NM, Zx[nd] - Zx[par], Zy[nd] - Zy[par], Zz[nd] - Zz[par], L);
#pragma unroll
    for (int k = 0; k < E::NM; k++) loc[(int64_t)nd * E::NM + k] = L[k];
}

template <int P>
__global__ void __launch_bounds__(EB) l2l_con_k(int lo, int hi, const int* __restrict__ nparent,
                                                const double* __restrict__ Zx, const double* __restrict__ Zy,
                                                const double* __restrict__ Zz, double* __restrict__ loc) {
    using E = Exp<P>;
    constexpr int NQ = E::NQ;
    int nd = lo + blockIdx.x * EB + threadIdx.x;
    if (nd >= hi) return;
    int par = nparent[nd];
    double sx = Zx[nd] - Zx[par], sy = Zy[nd] - Zy[par], sz = Zz[nd] - Zz[par];
    const double* Lp = loc + (int64_t)par * E::NSU;
    double* Lc = loc + (int64_t)nd * E::NSU;
    double sh[NQ];
#pragma unroll
    for (int k = 0; k < NQ; k++) sh[k] = 0.0;
    E::l2l_q(Lp, sx, sy, sz, sh);  // shifted parent S
    double t[NQ];
#pragma unroll
    for (int k = 0; k < NQ; k++) t[k] = Lc[k] + sh[k];
#pragma unroll
    for (int k = 0; k < NQ; k++) Lc[k] = t[k];
    const double s3[3] = {sx, sy, sz};
#pragma unroll
    for (int d = 0; d < 3; d++) {
#pragma unroll
        for (int k = 0; k < NQ; k++) t[k] = Lc[(d + 1) * NQ + k];
        E::l2l_q(Lp + (d + 1) * NQ, sx, sy, sz, t);
#pragma unroll
        for (int k = 0; k < NQ; k++) Lc[(d + 1) * NQ + k] = fma(s3[d], sh[k], t[k]);
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
        // the children of level l are exactly level l + 1
        int c_lo = c->level_start[l + 1], c_hi = c->level_start[l + 2];
        ensure(c->m2m_tmp, sizeof(double) * (size_t)(c_hi - c_lo) * E::NM);
        m2m_child_k<P><<<grid_for(c_hi - c_lo, EB), EB, 0, s>>>(lo, c_hi, c_lo, c->nparent.as<int>(),
                                                                c->nZx.as<double>(), c->nZy.as<double>(),
                                                                c->nZz.as<double>(), c->mom.as<double>(),
                                                                c->m2m_tmp.as<double>());
        GB_LAUNCH("m2m_child_k");
        m2m_sum_k<P><<<grid_for((int64_t)(hi - lo) * E::NM, EB), EB, 0, s>>>(
            lo, hi, c_lo, c->nchildf.as<int>(), c->nnchild.as<int>(), c->m2m_tmp.as<double>(), c->mom.as<double>());
        GB_LAUNCH("m2m_sum_k");
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
            l2l_con_k<P><<<grid_for(hi - lo, EB), EB, 0, s>>>(lo, hi, c->nparent.as<int>(), c->nZx.as<double>(),
                                                              c->nZy.as<double>(), c->nZz.as<double>(),
                                                              c->loc.as<double>());
            GB_LAUNCH("l2l_con_k");
        }
        if (std_locals) {
            DevBuf& L = variant == 0 ? c->loc : c->locp;
            l2l_std_k<P><<<grid_for(hi - lo, EB), EB, 0, s>>>(lo, hi, c->nparent.as<int>(), c->nZx.as<double>(),
                                                              c->nZy.as<double>(), c->nZz.as<double>(),
                                                              L.as<double>());
            GB_LAUNCH("l2l_std_k");
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
