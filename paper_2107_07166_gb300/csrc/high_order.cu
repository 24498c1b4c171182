// a8 / a8' M2L and a10 L2L for the high orders p = 7, 8 in binary64, table-driven.
//
// At these orders the straight-line operators of the lower orders need 165 moments, 165
// tensor entries and up to 480 locals per thread: fully unrolled they spill tens of
// kilobytes per thread.  Here one warp takes one work item (a target and up to a chunk
// of sources) and every lane owns a slice of the output coefficients, so each lane keeps
// a few accumulators in registers; per source the warp stages the source's moments and
// the derivative tensor in shared memory.
//
//   standard   : L_g += sum_{|b| + |g| <= p} M_b D_{b+g}(R),  D = d^a (-1/r)
//   conserving : S_g += sum_{|b| + |g| <= p-1} M_b h_{b+g}(R),
//                U_{i,g} += sum_b (R_i M_b + (b_i + 1) M_{b+e_i}) h_{b+g}(R),  h = d^a (-r^-3)
//
// The tensor is the closed form d^a f = sum_k prod_d [a_d! / (2^k_d k_d! (a_d - 2k_d)!)]
// R^(a - 2k) f_(|a| - |k|), with the radial derivatives f_m = (r^-1 d/dr)^m f, one tensor
// entry per lane at a time.  Outputs and partial layouts are those of m2l_std_k /
// m2l_con_k, so m2l_reduce_k sums them unchanged.
#include "fmm_device.cuh"
#include "fmm_internal.h"

namespace gbfmm {

namespace {

constexpr int GB = 128;  // 4 warps per block
constexpr int GW = GB / 32;
constexpr int PG = 8;    // largest order of this kernel

constexpr int nmi_c(int p) { return p < 0 ? 0 : (p + 1) * (p + 2) * (p + 3) / 6; }

// multi-index tables in the generated order (by degree, then a_x descending, then a_y
// descending), built per block in shared memory
struct MiTables {
    unsigned char a[nmi_c(PG)][3];
    short idx[PG + 1][PG + 1][PG + 1];
};

__device__ void build_tables(MiTables& t, int p) {
    if (threadIdx.x == 0) {
        int k = 0;
        for (int n = 0; n <= p; n++)
            for (int ax = n; ax >= 0; ax--)
                for (int ay = n - ax; ay >= 0; ay--) {
                    int az = n - ax - ay;
                    t.a[k][0] = (unsigned char)ax;
                    t.a[k][1] = (unsigned char)ay;
                    t.a[k][2] = (unsigned char)az;
                    t.idx[ax][ay][az] = (short)k;
                    k++;
                }
    }
    __syncthreads();
}

__device__ const double k_fact[PG + 1] = {1.0, 1.0, 2.0, 6.0, 24.0, 120.0, 720.0, 5040.0, 40320.0};

// d^a f at R for all |a| <= q, one entry per lane at a time, into T[]; kind 0: f = -1/r,
// kind 1: f = -r^-3
__device__ void tensor_warp(const MiTables& t, int q, int kind, double rx, double ry, double rz,
                            double* __restrict__ T, int lane) {
    double r2 = rx * rx + ry * ry + rz * rz;
    double ri = rsqrt(r2);
    double ri2 = ri * ri;
    double g[PG + 1];
    g[0] = kind == 0 ? -ri : -ri * ri2;
    for (int m = 1; m <= q; m++) g[m] = g[m - 1] * ri2 * (double)(kind == 0 ? -(2 * m - 1) : -(2 * m + 1));
    double px[PG + 1], py[PG + 1], pz[PG + 1];
    px[0] = py[0] = pz[0] = 1.0;
    for (int n = 1; n <= q; n++) {
        px[n] = px[n - 1] * rx;
        py[n] = py[n - 1] * ry;
        pz[n] = pz[n - 1] * rz;
    }
    int nq = nmi_c(q);
    for (int j = lane; j < nq; j += 32) {
        int ax = t.a[j][0], ay = t.a[j][1], az = t.a[j][2];
        double sum = 0.0;
        for (int kx = 0; 2 * kx <= ax; kx++)
            for (int ky = 0; 2 * ky <= ay; ky++)
                for (int kz = 0; 2 * kz <= az; kz++) {
                    double c = k_fact[ax] / (k_fact[kx] * k_fact[ax - 2 * kx] * (double)(1 << kx)) * k_fact[ay] /
                               (k_fact[ky] * k_fact[ay - 2 * ky] * (double)(1 << ky)) * k_fact[az] /
                               (k_fact[kz] * k_fact[az - 2 * kz] * (double)(1 << kz));
                    sum += c * px[ax - 2 * kx] * py[ay - 2 * ky] * pz[az - 2 * kz] * g[ax + ay + az - kx - ky - kz];
                }
        T[j] = sum;
    }
}

}  // namespace

// standard form; NM = nmi(P) locals, lane owns outputs g = lane, lane + 32, ...
template <int P>
__global__ void __launch_bounds__(GB) m2l_std_gen_k(int64_t nitems, const int4* __restrict__ items,
                                                    const uint32_t* __restrict__ dir, const double* __restrict__ Zx,
                                                    const double* __restrict__ Zy, const double* __restrict__ Zz,
                                                    const double* __restrict__ mom, double* __restrict__ part) {
    constexpr int NM = nmi_c(P), OW = (NM + 31) / 32;
    __shared__ MiTables t;
    __shared__ double sM[GW][NM], sT[GW][NM];
    build_tables(t, P);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t it = (int64_t)blockIdx.x * GW + w;
    if (it >= nitems) return;  // after the block barrier of build_tables
    int4 wi = items[it];
    double acc[OW];
#pragma unroll
    for (int o = 0; o < OW; o++) acc[o] = 0.0;
    double zx = Zx[wi.x], zy = Zy[wi.x], zz = Zz[wi.x];
    for (int e = wi.y; e < wi.z; e++) {
        int src = (int)dir[e];
        for (int j = lane; j < NM; j += 32) sM[w][j] = mom[(int64_t)src * NM + j];
        tensor_warp(t, P, 0, zx - Zx[src], zy - Zy[src], zz - Zz[src], sT[w], lane);
        __syncwarp();
#pragma unroll
        for (int o = 0; o < OW; o++) {
            int g = lane + 32 * o;
            if (g < NM) {
                int gx = t.a[g][0], gy = t.a[g][1], gz = t.a[g][2];
                int nb = nmi_c(P - (gx + gy + gz));
                double s = acc[o];
                for (int b = 0; b < nb; b++)
                    s = fma(sM[w][b], sT[w][t.idx[t.a[b][0] + gx][t.a[b][1] + gy][t.a[b][2] + gz]], s);
                acc[o] = s;
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int o = 0; o < OW; o++) {
        int g = lane + 32 * o;
        if (g < NM) part[it * NM + g] = acc[o];
    }
}

// conserving form; locals [S (NQ) | Ux | Uy | Uz], lane owns g = lane, lane + 32, ... of
// every block
template <int P>
__global__ void __launch_bounds__(GB) m2l_con_gen_k(int64_t nitems, const int4* __restrict__ items,
                                                    const uint32_t* __restrict__ dir, const double* __restrict__ Zx,
                                                    const double* __restrict__ Zy, const double* __restrict__ Zz,
                                                    const double* __restrict__ mom, double* __restrict__ part) {
    constexpr int NM = nmi_c(P), NQ = nmi_c(P - 1), OW = (NQ + 31) / 32;
    __shared__ MiTables t;
    __shared__ double sM[GW][NM], sT[GW][NQ], sC[GW][4][NQ];
    build_tables(t, P);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t it = (int64_t)blockIdx.x * GW + w;
    if (it >= nitems) return;
    int4 wi = items[it];
    double acc[OW][4];
#pragma unroll
    for (int o = 0; o < OW; o++)
#pragma unroll
        for (int i = 0; i < 4; i++) acc[o][i] = 0.0;
    double zx = Zx[wi.x], zy = Zy[wi.x], zz = Zz[wi.x];
    for (int e = wi.y; e < wi.z; e++) {
        int src = (int)dir[e];
        double rx = zx - Zx[src], ry = zy - Zy[src], rz = zz - Zz[src];
        for (int j = lane; j < NM; j += 32) sM[w][j] = mom[(int64_t)src * NM + j];
        tensor_warp(t, P - 1, 1, rx, ry, rz, sT[w], lane);
        __syncwarp();
        // per source: C_0b = M_b and C_ib = R_i M_b + (b_i + 1) M_{b+e_i}
        for (int b = lane; b < NQ; b += 32) {
            int bx = t.a[b][0], by = t.a[b][1], bz = t.a[b][2];
            double m = sM[w][b];
            sC[w][0][b] = m;
            sC[w][1][b] = fma(rx, m, (double)(bx + 1) * sM[w][t.idx[bx + 1][by][bz]]);
            sC[w][2][b] = fma(ry, m, (double)(by + 1) * sM[w][t.idx[bx][by + 1][bz]]);
            sC[w][3][b] = fma(rz, m, (double)(bz + 1) * sM[w][t.idx[bx][by][bz + 1]]);
        }
        __syncwarp();
#pragma unroll
        for (int o = 0; o < OW; o++) {
            int g = lane + 32 * o;
            if (g < NQ) {
                int gx = t.a[g][0], gy = t.a[g][1], gz = t.a[g][2];
                int nb = nmi_c(P - 1 - (gx + gy + gz));
                double s0 = acc[o][0], s1 = acc[o][1], s2 = acc[o][2], s3 = acc[o][3];
                for (int b = 0; b < nb; b++) {
                    double hv = sT[w][t.idx[t.a[b][0] + gx][t.a[b][1] + gy][t.a[b][2] + gz]];
                    s0 = fma(sC[w][0][b], hv, s0);
                    s1 = fma(sC[w][1][b], hv, s1);
                    s2 = fma(sC[w][2][b], hv, s2);
                    s3 = fma(sC[w][3][b], hv, s3);
                }
                acc[o][0] = s0;
                acc[o][1] = s1;
                acc[o][2] = s2;
                acc[o][3] = s3;
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int o = 0; o < OW; o++) {
        int g = lane + 32 * o;
        if (g < NQ)
#pragma unroll
            for (int i = 0; i < 4; i++) part[it * 4 * NQ + i * NQ + g] = acc[o][i];
    }
}

// ---- L2L: child locals += parent locals shifted by s = Z_child - Z_parent, one thread per
// node.  Every thread walks the same index sequence, so the multi-index tables sit in
// constant memory (broadcast reads) and the monomials s^b/b! in registers/local memory.

__constant__ unsigned char c_mi[nmi_c(PG)][3];
__constant__ short c_idx[PG + 1][PG + 1][PG + 1];

static void upload_tables() {
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && done[dev]) return;
    unsigned char a[nmi_c(PG)][3];
    short idx[PG + 1][PG + 1][PG + 1] = {};
    int k = 0;
    for (int n = 0; n <= PG; n++)
        for (int ax = n; ax >= 0; ax--)
            for (int ay = n - ax; ay >= 0; ay--) {
                int az = n - ax - ay;
                a[k][0] = (unsigned char)ax;
                a[k][1] = (unsigned char)ay;
                a[k][2] = (unsigned char)az;
                idx[ax][ay][az] = (short)k;
                k++;
            }
    GB_CUDA(cudaMemcpyToSymbol(c_mi, a, sizeof(a)));
    GB_CUDA(cudaMemcpyToSymbol(c_idx, idx, sizeof(idx)));
    if (dev >= 0 && dev < 64) done[dev] = true;
}

// out[g] += sum_{|g| + |b| <= q} in[g + b] w[b]  (g over nmi(q) entries)
template <int Q>
__device__ __forceinline__ void shift_poly(const double* __restrict__ in, const double* w, double* __restrict__ out) {
    constexpr int NQ = nmi_c(Q);
    for (int g = 0; g < NQ; g++) {
        int gx = c_mi[g][0], gy = c_mi[g][1], gz = c_mi[g][2];
        int nb = nmi_c(Q - (gx + gy + gz));
        double acc = out[g];
        for (int b = 0; b < nb; b++) acc = fma(in[c_idx[gx + c_mi[b][0]][gy + c_mi[b][1]][gz + c_mi[b][2]]], w[b], acc);
        out[g] = acc;
    }
}

// monomials s^b / b!, |b| <= q
template <int Q>
__device__ __forceinline__ void monomials(double sx, double sy, double sz, double* w) {
    double px[PG + 1], py[PG + 1], pz[PG + 1];
    px[0] = py[0] = pz[0] = 1.0;
    for (int n = 1; n <= Q; n++) {
        px[n] = px[n - 1] * sx / (double)n;
        py[n] = py[n - 1] * sy / (double)n;
        pz[n] = pz[n - 1] * sz / (double)n;
    }
    for (int k = 0; k < nmi_c(Q); k++) w[k] = px[c_mi[k][0]] * py[c_mi[k][1]] * pz[c_mi[k][2]];
}

template <int P>
__global__ void __launch_bounds__(128) l2l_std_gen_k(int lo, int hi, const int* __restrict__ nparent,
                                                     const double* __restrict__ Zx, const double* __restrict__ Zy,
                                                     const double* __restrict__ Zz, double* __restrict__ loc) {
    constexpr int NM = nmi_c(P);
    int nd = lo + blockIdx.x * 128 + threadIdx.x;
    if (nd >= hi) return;
    int par = nparent[nd];
    double w[NM];
    monomials<P>(Zx[nd] - Zx[par], Zy[nd] - Zy[par], Zz[nd] - Zz[par], w);
    shift_poly<P>(loc + (int64_t)par * NM, w, loc + (int64_t)nd * NM);
}

// conserving locals [S | Ux | Uy | Uz] of degree q = P - 1: S' = S(x + s) and
// U_i' = U_i(x + s) + s_i S(x + s)
template <int P>
__global__ void __launch_bounds__(128) l2l_con_gen_k(int lo, int hi, const int* __restrict__ nparent,
                                                     const double* __restrict__ Zx, const double* __restrict__ Zy,
                                                     const double* __restrict__ Zz, double* __restrict__ loc) {
    constexpr int Q = P - 1, NQ = nmi_c(Q);
    int nd = lo + blockIdx.x * 128 + threadIdx.x;
    if (nd >= hi) return;
    int par = nparent[nd];
    double s3[3] = {Zx[nd] - Zx[par], Zy[nd] - Zy[par], Zz[nd] - Zz[par]};
    double w[NQ], sh[NQ];
    monomials<Q>(s3[0], s3[1], s3[2], w);
    const double* Lp = loc + (int64_t)par * 4 * NQ;
    double* Lc = loc + (int64_t)nd * 4 * NQ;
    for (int g = 0; g < NQ; g++) sh[g] = 0.0;
    shift_poly<Q>(Lp, w, sh);
    for (int g = 0; g < NQ; g++) Lc[g] += sh[g];
    for (int d = 0; d < 3; d++) {
        shift_poly<Q>(Lp + (d + 1) * NQ, w, Lc + (d + 1) * NQ);
        for (int g = 0; g < NQ; g++) Lc[(d + 1) * NQ + g] = fma(s3[d], sh[g], Lc[(d + 1) * NQ + g]);
    }
}

// one level of the high-order L2L (variant 0 standard, else conserving)
void l2l_generic_launch(fmm_ctx* c, int p, int variant, int lo, int hi, double* loc) {
    if (hi <= lo) return;
    upload_tables();
    unsigned blocks = (unsigned)((hi - lo + 127) / 128);
    cudaStream_t s = c->stream;
    const int* par = c->nparent.as<int>();
    const double *zx = c->nZx.as<double>(), *zy = c->nZy.as<double>(), *zz = c->nZz.as<double>();
    if (p == 7) {
        if (variant == 0)
            l2l_std_gen_k<7><<<blocks, 128, 0, s>>>(lo, hi, par, zx, zy, zz, loc);
        else
            l2l_con_gen_k<7><<<blocks, 128, 0, s>>>(lo, hi, par, zx, zy, zz, loc);
    } else {
        if (variant == 0)
            l2l_std_gen_k<8><<<blocks, 128, 0, s>>>(lo, hi, par, zx, zy, zz, loc);
        else
            l2l_con_gen_k<8><<<blocks, 128, 0, s>>>(lo, hi, par, zx, zy, zz, loc);
    }
    GB_LAUNCH("l2l_gen_k");
}

// launches the high-order binary64 M2L of one variant (0 standard, 1 conserving) into the
// item partials
void m2l_generic_launch(fmm_ctx* c, int p, int variant, double* part) {
    const ItemSet& it = c->m2l_items;
    int64_t ni = it.n_items;
    if (ni <= 0) return;
    unsigned blocks = (unsigned)((ni + GW - 1) / GW);
    const uint32_t* dir = c->m2l_dir.as<uint32_t>();
    const double *zx = c->nZx.as<double>(), *zy = c->nZy.as<double>(), *zz = c->nZz.as<double>();
    const double* mom = c->mom.as<double>();
    cudaStream_t s = c->stream;
    if (p == 7) {
        if (variant == 0)
            m2l_std_gen_k<7><<<blocks, GB, 0, s>>>(ni, it.items.as<int4>(), dir, zx, zy, zz, mom, part);
        else
            m2l_con_gen_k<7><<<blocks, GB, 0, s>>>(ni, it.items.as<int4>(), dir, zx, zy, zz, mom, part);
    } else {
        if (variant == 0)
            m2l_std_gen_k<8><<<blocks, GB, 0, s>>>(ni, it.items.as<int4>(), dir, zx, zy, zz, mom, part);
        else
            m2l_con_gen_k<8><<<blocks, GB, 0, s>>>(ni, it.items.as<int4>(), dir, zx, zy, zz, mom, part);
    }
    GB_LAUNCH("m2l_gen_k");
}

}  // namespace gbfmm
