// Mutual dual-tree walk (Sec. 2: well-separated node pairs by eq. mac_criterion,
// Dehnen-style mutual interactions) as a level-synchronous frontier of cell pairs.
//
//   Self(A): A leaf -> P2P(A, A); else over its children c_i, c_j with i <= j:
//            Self(c_i) if i == j, Pair(c_i, c_j) otherwise.
//   Pair(A, B): R = |Z_A - Z_B| > 0 and r_A + r_B <= theta R  -> M2L(A, B)
//               both leaves                                    -> P2P(A, B)
//               otherwise split A or B into its children: a leaf is never split; between
//               two inner nodes the larger r_max is split, ties -> larger count, then
//               lower id.
// The rule is symmetric in (A, B), so the emitted pair set is unique.  Each frontier
// step counts every item's outputs, scans the counts and writes the outputs at their
// offsets, so the emission order is deterministic too.  The lists are then expanded
// into directed entries (target, source) and radix-sorted: every cell sees its partners
// in increasing id order, which is also the canonical (min id, max id) order.
#include "fmm_device.cuh"
#include "fmm_internal.h"

namespace gbfmm {

constexpr int WB = 256;

__device__ __forceinline__ bool mac_accept(const NodeView& nv, int A, int B, double theta) {
    double dx = __dsub_rn(nv.Zx[A], nv.Zx[B]);
    double dy = __dsub_rn(nv.Zy[A], nv.Zy[B]);
    double dz = __dsub_rn(nv.Zz[A], nv.Zz[B]);
    double R = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
    return R > 0.0 && __dadd_rn(nv.rmax[A], nv.rmax[B]) <= __dmul_rn(theta, R);
}

// true: split A; false: split B (neither is a leaf here)
__device__ __forceinline__ bool split_a(const NodeView& nv, int A, int B) {
    double ra = nv.rmax[A], rb = nv.rmax[B];
    if (ra != rb) return ra > rb;
    int ca = nv.count[A], cb = nv.count[B];
    if (ca != cb) return ca > cb;
    return A < B;
}

// decision: 0 = split, 1 = M2L, 2 = P2P; *split_node / *nnew for splits
__device__ __forceinline__ int decide(const NodeView& nv, int2 it, double theta, int* nnew, bool* sa) {
    int A = it.x, B = it.y;
    if (A == B) {
        int nc = nv.nchild[A];
        if (nc == 0) return 2;
        *nnew = nc * (nc + 1) / 2;
        return 0;
    }
    if (mac_accept(nv, A, B, theta)) return 1;
    bool la = nv.nchild[A] == 0, lb = nv.nchild[B] == 0;
    if (la && lb) return 2;
    bool s = lb ? true : (la ? false : split_a(nv, A, B));
    *sa = s;
    *nnew = nv.nchild[s ? A : B];
    return 0;
}

__global__ void walk_count_k(const int2* __restrict__ fr, int nf, NodeView nv, double theta, Cnt3* __restrict__ cnt) {
    int i = blockIdx.x * WB + threadIdx.x;
    if (i >= nf) return;
    int nnew = 0;
    bool sa = false;
    int d = decide(nv, fr[i], theta, &nnew, &sa);
    cnt[i] = Cnt3{d == 0 ? nnew : 0, d == 1 ? 1 : 0, d == 2 ? 1 : 0};
}

__global__ void walk_emit_k(const int2* __restrict__ fr, int nf, NodeView nv, double theta,
                            const Cnt3* __restrict__ off, int2* __restrict__ fr_out, int2* __restrict__ m2l,
                            int2* __restrict__ p2p) {
    int i = blockIdx.x * WB + threadIdx.x;
    if (i >= nf) return;
    int2 it = fr[i];
    int nnew = 0;
    bool sa = false;
    int d = decide(nv, it, theta, &nnew, &sa);
    Cnt3 o = off[i];
    if (d == 1) {
        m2l[o.b] = it;
    } else if (d == 2) {
        p2p[o.c] = it;
    } else if (it.x == it.y) {
        int c0 = nv.child_first[it.x], nc = nv.nchild[it.x];
        int k = o.a;
        for (int a = 0; a < nc; a++)
            for (int b = a; b < nc; b++) fr_out[k++] = make_int2(c0 + a, c0 + b);
    } else {
        int S = sa ? it.x : it.y;
        int c0 = nv.child_first[S], nc = nv.nchild[S];
        for (int a = 0; a < nc; a++) fr_out[o.a + a] = sa ? make_int2(c0 + a, it.y) : make_int2(it.x, c0 + a);
    }
}

// directed M2L entries: (A -> B) and (B -> A) for every mutual pair
__global__ void m2l_dir_k(const int2* __restrict__ pairs, int64_t n, int bits, uint64_t* __restrict__ keys) {
    int64_t k = (int64_t)blockIdx.x * WB + threadIdx.x;
    if (k >= n) return;
    int2 p = pairs[k];
    keys[2 * k] = ((uint64_t)p.x << bits) | (uint64_t)p.y;
    keys[2 * k + 1] = ((uint64_t)p.y << bits) | (uint64_t)p.x;
}

// directed P2P entries carry (pair << 1 | side); a self pair has one entry, its second
// slot holds the all-ones key, which sorts after every real entry
__global__ void p2p_dir_k(const int2* __restrict__ pairs, int64_t n, int bits, uint64_t* __restrict__ keys,
                          uint32_t* __restrict__ vals, const int* __restrict__ count, long long* __restrict__ psize) {
    int64_t k = (int64_t)blockIdx.x * WB + threadIdx.x;
    if (k >= n) return;
    int2 p = pairs[k];
    keys[2 * k] = ((uint64_t)p.x << bits) | (uint64_t)p.y;
    vals[2 * k] = (uint32_t)(2 * k);
    if (p.x != p.y) {
        keys[2 * k + 1] = ((uint64_t)p.y << bits) | (uint64_t)p.x;
        vals[2 * k + 1] = (uint32_t)(2 * k + 1);
        psize[k] = (long long)count[p.x] + count[p.y];
    } else {
        keys[2 * k + 1] = (1ull << (2 * bits)) - 1ull;
        vals[2 * k + 1] = 0xffffffffu;
        psize[k] = count[p.x];
    }
}

__global__ void seg_count_k(const uint64_t* __restrict__ keys, int64_t n, int bits, int* __restrict__ cnt) {
    int64_t i = (int64_t)blockIdx.x * WB + threadIdx.x;
    if (i >= n) return;
    uint64_t k = keys[i];
    if (k == (1ull << (2 * bits)) - 1ull) return;
    atomicAdd(&cnt[k >> bits], 1);  // integer counts: order independent
}

// Work items over segments seg[0..n]: every segment is cut into chunks of CH entries.
// Full chunks come first (segment-major), then one partial chunk per segment that has a
// remainder, so that warps see chunks of equal length.  fo/po (n + 1 entries) give each
// segment's full-chunk range and partial-chunk rank.
__global__ void items_count_k(const long long* __restrict__ seg, int n, int CH, int* __restrict__ nfull,
                              int* __restrict__ npart) {
    int x = blockIdx.x * WB + threadIdx.x;
    if (x >= n) return;
    long long deg = seg[x + 1] - seg[x];
    nfull[x] = (int)(deg / CH);
    npart[x] = (deg % CH) != 0;
}

__global__ void items_fill_k(const long long* __restrict__ seg, int n, int CH, const long long* __restrict__ fo,
                             const long long* __restrict__ po, long long nfull_total, int4* __restrict__ items) {
    int x = blockIdx.x * WB + threadIdx.x;
    if (x >= n) return;
    long long e0 = seg[x], e1 = seg[x + 1];
    long long k0 = fo[x], nf = fo[x + 1] - k0;
    for (long long k = 0; k < nf; k++)
        items[k0 + k] = make_int4(x, (int)(e0 + k * CH), (int)(e0 + (k + 1) * CH), 0);
    if (po[x + 1] > po[x]) items[nfull_total + po[x]] = make_int4(x, (int)(e0 + nf * CH), (int)e1, 0);
}

void build_items(fmm_ctx* c, const long long* seg, int n, int CH, ItemSet& it) {
    cudaStream_t s = c->stream;
    ensure(c->seg_cnt, sizeof(int) * (size_t)(2 * n + 2));
    int* nfull = c->seg_cnt.as<int>();
    int* npart = nfull + n + 1;
    ensure(it.fo, sizeof(long long) * (size_t)(n + 1));
    ensure(it.po, sizeof(long long) * (size_t)(n + 1));
    items_count_k<<<grid_for(n, WB), WB, 0, s>>>(seg, n, CH, nfull, npart);
    GB_LAUNCH("items_count_k");
    scan_i64(c, nfull, n, it.fo.as<long long>());
    scan_i64(c, npart, n, it.po.as<long long>());
    long long tot[2];
    GB_CUDA(cudaMemcpyAsync(&tot[0], it.fo.as<long long>() + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaMemcpyAsync(&tot[1], it.po.as<long long>() + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    it.n_full = tot[0];
    it.n_items = tot[0] + tot[1];
    it.chunk = CH;
    ensure(it.items, sizeof(int4) * (size_t)(it.n_items > 0 ? it.n_items : 1));
    items_fill_k<<<grid_for(n, WB), WB, 0, s>>>(seg, n, CH, it.fo.as<long long>(), it.po.as<long long>(), it.n_full,
                                                it.items.as<int4>());
    GB_LAUNCH("items_fill_k");
}

static int bits_for(int64_t nn) {
    int b = 1;
    while (((int64_t)1 << b) <= nn) b++;  // ids < 2^b - 1 always
    return b;
}

void run_walk(fmm_ctx* c, double theta) {
    cudaStream_t s = c->stream;
    NodeView nv = node_view(c);
    int64_t nn = c->n_nodes;
    // frontier starts with Self(root)
    int64_t cap_fr = 4096;
    ensure(c->fr0, sizeof(int2) * (size_t)cap_fr);
    int2 root = make_int2(0, 0);
    GB_CUDA(cudaMemcpyAsync(c->fr0.p, &root, sizeof(int2), cudaMemcpyHostToDevice, s));
    int64_t nf = 1, n_m2l = 0, n_p2p = 0;
    while (nf > 0) {
        if (nf >= ((int64_t)1 << 31)) throw FmmError{FMM_ERR_CAPACITY, "walk frontier above 2^31"};
        ensure(c->cnt, sizeof(Cnt3) * (size_t)nf);
        ensure(c->cnt_off, sizeof(Cnt3) * (size_t)(nf + 1));
        walk_count_k<<<grid_for(nf, WB), WB, 0, s>>>(c->fr0.as<int2>(), (int)nf, nv, theta, c->cnt.as<Cnt3>());
        GB_LAUNCH("walk_count_k");
        scan_cnt3(c, c->cnt.as<Cnt3>(), nf, c->cnt_off.as<Cnt3>());
        Cnt3 tot;
        GB_CUDA(cudaMemcpyAsync(&tot, c->cnt_off.as<Cnt3>() + nf, sizeof(Cnt3), cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaStreamSynchronize(s));
        if ((int64_t)n_m2l + tot.b >= ((int64_t)1 << 31) || (int64_t)n_p2p + tot.c >= ((int64_t)1 << 30))
            throw FmmError{FMM_ERR_CAPACITY, "interaction lists above 2^31 entries"};
        ensure(c->fr1, sizeof(int2) * (size_t)(tot.a > 0 ? tot.a : 1));
        ensure_keep(c->m2l_pairs, sizeof(int2) * (size_t)(n_m2l + tot.b + 1), s);
        ensure_keep(c->p2p_pairs, sizeof(int2) * (size_t)(n_p2p + tot.c + 1), s);
        walk_emit_k<<<grid_for(nf, WB), WB, 0, s>>>(c->fr0.as<int2>(), (int)nf, nv, theta, c->cnt_off.as<Cnt3>(),
                                                    c->fr1.as<int2>(), c->m2l_pairs.as<int2>() + n_m2l,
                                                    c->p2p_pairs.as<int2>() + n_p2p);
        GB_LAUNCH("walk_emit_k");
        n_m2l += tot.b;
        n_p2p += tot.c;
        nf = tot.a;
        DevBuf t = c->fr0;
        c->fr0 = c->fr1;
        c->fr1 = t;
    }
    c->n_m2l = n_m2l;
    c->n_p2p = n_p2p;
    int bits = bits_for(nn);
    c->id_bits = bits;
    // M2L: directed entries sorted by (target, source)
    int64_t nd = 2 * n_m2l;
    ensure(c->m2l_dir, sizeof(uint64_t) * (size_t)(nd > 0 ? nd : 1));
    ensure(c->seg_cnt, sizeof(int) * (size_t)(nn + 1));
    ensure(c->m2l_seg, sizeof(long long) * (size_t)(nn + 1));
    if (n_m2l > 0) {
        m2l_dir_k<<<grid_for(n_m2l, WB), WB, 0, s>>>(c->m2l_pairs.as<int2>(), n_m2l, bits, c->m2l_dir.as<uint64_t>());
        GB_LAUNCH("m2l_dir_k");
        radix_sort(c, c->m2l_dir, c->keys1, nullptr, nullptr, nd, 2 * bits);
    }
    GB_CUDA(cudaMemsetAsync(c->seg_cnt.p, 0, sizeof(int) * (size_t)nn, s));
    if (nd > 0) {
        seg_count_k<<<grid_for(nd, WB), WB, 0, s>>>(c->m2l_dir.as<uint64_t>(), nd, bits, c->seg_cnt.as<int>());
        GB_LAUNCH("seg_count_k");
    }
    scan_i64(c, c->seg_cnt.as<int>(), nn, c->m2l_seg.as<long long>());
    // P2P: directed entries with payload (pair << 1 | side), plus partial offsets
    int64_t np = 2 * n_p2p;
    ensure(c->p2p_dir, sizeof(uint64_t) * (size_t)np);
    ensure(c->p2p_dval, sizeof(uint32_t) * (size_t)np);
    ensure(c->p2p_off, sizeof(long long) * (size_t)(n_p2p + 1));
    ensure(c->p2p_seg, sizeof(long long) * (size_t)(nn + 1));
    ensure(c->flags, sizeof(long long) * (size_t)(n_p2p + 1));  // per-pair partial sizes
    p2p_dir_k<<<grid_for(n_p2p, WB), WB, 0, s>>>(c->p2p_pairs.as<int2>(), n_p2p, bits, c->p2p_dir.as<uint64_t>(),
                                                 c->p2p_dval.as<uint32_t>(), c->ncount.as<int>(),
                                                 c->flags.as<long long>());
    GB_LAUNCH("p2p_dir_k");
    scan_i64_from_i64(c, c->flags.as<long long>(), n_p2p, c->p2p_off.as<long long>());
    radix_sort(c, c->p2p_dir, c->keys1, &c->p2p_dval, &c->vals1, np, 2 * bits);
    GB_CUDA(cudaMemsetAsync(c->seg_cnt.p, 0, sizeof(int) * (size_t)nn, s));
    seg_count_k<<<grid_for(np, WB), WB, 0, s>>>(c->p2p_dir.as<uint64_t>(), np, bits, c->seg_cnt.as<int>());
    GB_LAUNCH("seg_count_k");
    scan_i64(c, c->seg_cnt.as<int>(), nn, c->p2p_seg.as<long long>());
    // work items: 32 M2L sources per chunk, 64 P2P entries per chunk
    build_items(c, c->m2l_seg.as<long long>(), (int)nn, M2L_CHUNK, c->m2l_items);
    build_items(c, c->p2p_seg.as<long long>(), (int)nn, P2P_CHUNK, c->p2p_items);
    c->list_theta = theta;
}

}  // namespace gbfmm
