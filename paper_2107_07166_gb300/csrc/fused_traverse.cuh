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
// mutual walk emits, each once.  One warp runs one target's traversal, deciding up to
// 32 pending pairs at a time (one per lane) and keeping the order of everything fixed by
// the tree.
//   Far field: the M2L sources of T are buffered 32 at a time and evaluated one per lane
//     (binary64, the list schedule's operators with a tensor per entry), and the lanes'
//     sums are added in a fixed butterfly order at the end: one write per target.
//   Near field (target leaves): T's particles against each P2P partner's particles, each
//     pair force formed from T's side (so every pair is formed twice over the two
//     partners, where the list schedule forms it once); lanes are (particle, group) with
//     the partner's particles dealt round-robin to the groups, and the groups' sums are
//     added in a fixed order at the end: one write per particle.
// Every sum runs in a fixed order, so results are run-to-run identical.  The pending pairs
// of one traversal stay below FQCAP per warp (see traverse); a traversal that would
// exceed them would set an error flag and stop (FMM_ERR_CAPACITY).
#pragma once
#include "fmm_device.cuh"
#include "fmm_internal.h"
#include "prec.cuh"
#include "walk_rule.cuh"

namespace gbfmm {

constexpr int FB = 64;         // 2 warps per block
constexpr int FW = FB / 32;
constexpr int FQCAP = 2048;    // stack of pending pairs per warp
constexpr int FMAXDEPTH = 22;  // levels 0 .. 21

// T's root path: path[0] = its system's root, path[kT] = T
__device__ __forceinline__ int root_path(const NodeView& nv, int T, int* path) {
    int tmp[FMAXDEPTH];
    int d = 0;
    for (int x = T; x >= 0 && d < FMAXDEPTH; x = nv.parent[x]) tmp[d++] = x;
    for (int i = 0; i < d; i++) path[i] = tmp[d - 1 - i];
    return d - 1;
}

// One target's traversal (see the file comment), warp-parallel: the warp pops up to 32
// pending pairs at a time from the top of a stack in shared memory, one per lane, decides
// them, hands T's interactions to the visitor in lane order (vis.m2l(Y), vis.p2p(Y), called
// by the whole warp with the same Y) and pushes the pairs they split into, in lane order
// and child order.  The order of everything is a fixed function of the tree.  Pending
// entries (k, Y): Y < 0 is Self(path[k]), otherwise Pair(path[k], Y).
// Bound: a popped pair pushes at most 8, so popping n of them at stack size s leaves at
// most s + 7n.  The batch is cut to n <= (FQCAP - FHEAD - s) / 7 when that is below 32, down
// to n = 1: one-at-a-time depth-first order, which grows by at most 7 per step of the pair
// recursion, and a step goes one level deeper on one side of the pair, so at most 42
// steps (21 levels a side: 7 x 42 = 294 < FHEAD).  The stack therefore never exceeds
// FQCAP; the check below only guards the argument.
constexpr int FHEAD = 320;

template <class V>
__device__ __forceinline__ void traverse(const NodeView& nv, int T, double theta, float th2, int2* __restrict__ q,
                                         int* __restrict__ err, V& vis) {
    int lane = threadIdx.x & 31;
    int path[FMAXDEPTH];
    int kT = root_path(nv, T, path);
    int top = 1;
    if (lane == 0) q[0] = make_int2(0, -1);
    __syncwarp();
    while (top > 0) {
        int n = min(32, top);
        int room = (FQCAP - FHEAD - top) / 7;
        if (room < n) n = max(1, room);
        bool act = lane < n;
        int2 e = act ? q[top - n + lane] : make_int2(0, 0);
        top -= n;
        __syncwarp();  // the slots just read may be refilled below
        int k = e.x, Y = e.y, X = act ? path[k] : 0;
        int emit = 0, ey = 0;  // 1: M2L(T, ey), 2: P2P(T, ey)
        int mode = 0, nk = 0, cf = 0;  // children: 1 Self(X)'s, 2 path child of X, 3 Y's
        if (act) {
            if (Y < 0) {
                int nc = nv.nchild[X];
                if (nc == 0) {
                    if (k == kT) {
                        emit = 2;
                        ey = X;
                    }
                } else if (k != kT) {
                    mode = 1;
                    nk = nc;
                    cf = nv.child_first[X];
                }
            } else {
                int nnew = 0;
                bool sa = false;
                int d = decide(nv, make_int2(X, Y), theta, th2, &nnew, &sa);
                if (d == 1 || d == 2) {
                    if (k == kT) {
                        emit = d;
                        ey = Y;
                    }
                } else if (sa) {
                    if (k != kT) {
                        mode = 2;
                        nk = 1;
                    }
                } else {
                    mode = 3;
                    nk = nv.nchild[Y];
                    cf = nv.child_first[Y];
                }
            }
        }
        // T's interactions, in lane order
        unsigned em = __ballot_sync(FULL, emit != 0);
        while (em) {
            int j = __ffs(em) - 1;
            em &= em - 1;
            int t = __shfl_sync(FULL, emit, j), y = __shfl_sync(FULL, ey, j);
            if (t == 1)
                vis.m2l(y);
            else
                vis.p2p(y);
        }
        // the new pending pairs, in lane order
        int inc = nk;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += u;
        }
        int tot = __shfl_sync(FULL, inc, 31), pos = inc - nk;
        if (top + tot > FQCAP) {
            if (lane == 0) atomicExch(err, 1);
            break;
        }
        int at = top + pos;
        if (mode == 1) {
            int cp = path[k + 1];
            for (int i = 0; i < nk; i++) q[at + i] = cf + i == cp ? make_int2(k + 1, -1) : make_int2(k + 1, cf + i);
        } else if (mode == 2) {
            q[at] = make_int2(k + 1, Y);
        } else if (mode == 3) {
            for (int i = 0; i < nk; i++) q[at + i] = make_int2(k, cf + i);
        }
        top += tot;
        __syncwarp();
    }
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
    __shared__ int2 stk[FW][FQCAP];
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
        fused_m2l_k<P, 0><<<sms * 16, FB, 0, c->stream>>>(nn, nv, theta, th2, c->mom.as<double>(), loc, err);
    else
        fused_m2l_k<P, 1><<<sms * 16, FB, 0, c->stream>>>(nn, nv, theta, th2, c->cmom.as<double>(), loc, err);
    GB_LAUNCH("fused_m2l_k");
}

}  // namespace gbfmm
