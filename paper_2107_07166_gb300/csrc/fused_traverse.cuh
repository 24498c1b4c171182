// The fused schedule: the mutual walk's interactions evaluated as a per-target traversal,
// with no interaction list, list sort, P2P partial buffer or gather (binary64).
//
// The list schedule runs the mutual walk once (walk.cu), stores its M2L and P2P pairs,
// sorts the directed entries by target and evaluates them.  Here every target node T
// walks the same recursion (Sec. 2, eq. mac_criterion, the mutual walk's split rule)
// restricted to the pairs that contain one of T's ancestors:
//   Self(X), X on T's root path: a leaf gives P2P(T, T) when X = T; otherwise, unless
//     X = T, its child on the path, cp, meets every other child c in Pair(cp, c) and
//     recurses into Self(cp);
//   Pair(X, Y), X on the path: the walk's decision (walk_rule.cuh) on (X, Y); M2L and P2P
//     are T's interactions when X = T; a split of X continues with X's child on the path
//     (unless X = T, whose children receive the pair), a split of Y with every child of Y.
// The rule is symmetric in the two cells, so T receives exactly the pairs (T, Y) the
// mutual walk emits, each once; the traversal is a depth-first search with an explicit
// stack, in a fixed order.  One warp runs one target's traversal with every lane taking
// the same steps (the decisions depend on the nodes only).
//   Far field: the M2L sources of T are buffered 32 at a time and evaluated one per lane
//     (binary64, the list schedule's operators with a tensor per entry), and the lanes'
//     sums are added in a fixed butterfly order at the end: one write per target.
//   Near field (target leaves): T's particles against each P2P partner's particles, each
//     pair force formed from T's side (so every pair is formed twice over the two
//     partners, where the list schedule forms it once); lanes are (particle, group) with
//     the partner's particles dealt round-robin to the groups, and the groups' sums are
//     added in a fixed order at the end: one write per particle.
// Every sum runs in a fixed order, so results are run-to-run identical.  The traversal
// stack is bounded (FSTACK entries per warp); a traversal that would overflow it sets an
// error flag and stops (FMM_ERR_CAPACITY), which no octree of depth <= 21 can reach.
#pragma once
#include "fmm_device.cuh"
#include "fmm_internal.h"
#include "prec.cuh"
#include "walk_rule.cuh"

namespace gbfmm {

constexpr int FB = 128;        // 4 warps per block
constexpr int FW = FB / 32;
constexpr int FSTACK = 256;    // traversal stack entries per warp (at most 7 + 8 per level are live)
constexpr int FMAXDEPTH = 22;  // levels 0 .. 21

// T's root path: path[0] = its system's root, path[kT] = T
__device__ __forceinline__ int root_path(const NodeView& nv, int T, int* path) {
    int tmp[FMAXDEPTH];
    int d = 0;
    for (int x = T; x >= 0 && d < FMAXDEPTH; x = nv.parent[x]) tmp[d++] = x;
    for (int i = 0; i < d; i++) path[i] = tmp[d - 1 - i];
    return d - 1;
}

// One target's traversal (see the file comment); vis.m2l(Y) and vis.p2p(Y) receive T's
// interactions in depth-first order.  Stack entries (k, Y): Y < 0 is Self(path[k]),
// otherwise Pair(path[k], Y).  Every lane of the warp runs it identically.
template <class V>
__device__ __forceinline__ void traverse(const NodeView& nv, int T, double theta, float th2, int2* __restrict__ stk,
                                         int* __restrict__ err, V& vis) {
    int path[FMAXDEPTH];
    int kT = root_path(nv, T, path);
    int top = 0;
    stk[top++] = make_int2(0, -1);
    bool over = false;
    while (top > 0) {
        int2 e = stk[--top];
        int k = e.x, X = path[k];
        if (e.y < 0) {  // Self(X)
            int nc = nv.nchild[X];
            if (nc == 0) {
                if (k == kT) vis.p2p(X);
                continue;
            }
            if (k == kT) continue;
            int cp = path[k + 1], c0 = nv.child_first[X];
            if (top + nc > FSTACK) {
                over = true;
                break;
            }
            for (int c = c0 + nc - 1; c >= c0; c--) stk[top++] = c == cp ? make_int2(k + 1, -1) : make_int2(k + 1, c);
            continue;
        }
        int Y = e.y, nnew = 0;
        bool sa = false;
        int d = decide(nv, make_int2(X, Y), theta, th2, &nnew, &sa);
        if (d == 1) {
            if (k == kT) vis.m2l(Y);
        } else if (d == 2) {
            if (k == kT) vis.p2p(Y);
        } else if (sa) {
            if (k == kT) continue;
            if (top + 1 > FSTACK) {
                over = true;
                break;
            }
            stk[top++] = make_int2(k + 1, Y);
        } else {
            int c0 = nv.child_first[Y], nc = nv.nchild[Y];
            if (top + nc > FSTACK) {
                over = true;
                break;
            }
            for (int c = c0 + nc - 1; c >= c0; c--) stk[top++] = make_int2(k, c);
        }
    }
    if (over && (threadIdx.x & 31) == 0) atomicExch(err, 1);
}

// ---------------------------------------------------------------- far field

template <int P, int KIND>
struct FarVisitor {
    using E = Exp<P>;
    static constexpr int NO = KIND == 0 ? E::NM : E::NSU;
    const NodeView* nv;
    const double* src;  // KIND 0: raw moments (NM per node); 1: root-relative conserving moments (NSU)
    int* buf;           // the warp's 32 buffered sources
    int T, cnt, lane;
    double O[NO];

    __device__ void flush() {
        __syncwarp();
        if (lane < cnt) {
            int Y = buf[lane];
            double rx = nv->Zx[T] - nv->Zx[Y], ry = nv->Zy[T] - nv->Zy[Y], rz = nv->Zz[T] - nv->Zz[Y];
            if constexpr (KIND == 0) {
                double D[E::NM];
                E::dtensor(rx, ry, rz, D);
                E::m2l_std(src + (int64_t)Y * E::NM, D, O);
            } else {
                double H[E::NQ];
                E::htensor(rx, ry, rz, H);
                E::m2l_con_o(src + (int64_t)Y * E::NSU, H, O);
            }
        }
        cnt = 0;
        __syncwarp();
    }
    __device__ void m2l(int Y) {
        if (lane == 0) buf[cnt] = Y;
        if (++cnt == 32) flush();
    }
    __device__ void p2p(int) {}
};

// a8/a8' without lists: one warp per target node, loc[T] = the target's M2L sums
// (KIND 0: standard locals L; 1: S and the root-relative part of U, completed by
// con_origin_k as in the list schedule)
template <int P, int KIND>
__global__ void __launch_bounds__(FB) fused_m2l_k(int nn, NodeView nv, double theta, float th2,
                                                  const double* __restrict__ src, double* __restrict__ loc,
                                                  int* __restrict__ err) {
    __shared__ int2 stk[FW][FSTACK];
    __shared__ int sbuf[FW][32];
    using Vis = FarVisitor<P, KIND>;
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int T = blockIdx.x * FW + w; T < nn; T += gridDim.x * FW) {
        Vis vis;
        vis.nv = &nv;
        vis.src = src;
        vis.buf = sbuf[w];
        vis.T = T;
        vis.cnt = 0;
        vis.lane = lane;
#pragma unroll
        for (int k = 0; k < Vis::NO; k++) vis.O[k] = 0.0;
        traverse(nv, T, theta, th2, stk[w], err, vis);
        if (vis.cnt > 0) vis.flush();
        // the lanes' sums in a fixed butterfly order; lane l writes coefficients l, l + 32, ...
#pragma unroll
        for (int k = 0; k < Vis::NO; k++) {
            double v = vis.O[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
            if ((k & 31) == lane) loc[(int64_t)T * Vis::NO + k] = v;
        }
        __syncwarp();
    }
}


template <int P>
void fused_m2l_launch(fmm_ctx* c, int kind, double theta, double* loc) {
    NodeView nv = node_view(c);
    float th2 = (float)theta * (float)theta;
    int nn = (int)c->n_nodes;
    int* err = c->errflag.as<int>() + 2;
    int sms = 0;
    GB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    if (kind == 0)
        fused_m2l_k<P, 0><<<sms * 8, FB, 0, c->stream>>>(nn, nv, theta, th2, c->mom.as<double>(), loc, err);
    else
        fused_m2l_k<P, 1><<<sms * 8, FB, 0, c->stream>>>(nn, nv, theta, th2, c->cmom.as<double>(), loc, err);
    GB_LAUNCH("fused_m2l_k");
}

}  // namespace gbfmm
