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
// The rule is symmetric in (A, B), so the emitted pair set is unique.  One kernel per
// frontier step decides its items and places the outputs in frontier order (ordered
// claims by look-back over tiles), so the pair lists come out in a fixed order; they are
// then expanded into directed entries (target, partner) and stably radix-sorted by
// target, and every later sum runs in that order.  The host launches a fixed number of
// steps (2 x levels + 2 bounds the recursion depth) without waiting between them.  The
// counters keep counting past the buffers' capacity; one read at the end detects an
// overflow and the walk is run again with buffers of the reported sizes.
#include <algorithm>
#include <vector>

#include "fmm_device.cuh"
#include "fmm_internal.h"
#include "walk_rule.cuh"

namespace gbfmm {

constexpr int WB = 256;

struct WalkCounters {
    int nf[2];                  // frontier sizes (read by the step of that parity)
    int n_m2l, n_p2p;           // pairs emitted by the finished steps
    int ticket;                 // next tile of the running step
    int step_tot[3];            // M2L pairs, P2P pairs and new items of the running step
    int err;                    // a wait for a preceding tile ran out (never expected)
};

// One frontier step.  Blocks take tiles of WTILE consecutive frontier items in the order of
// a ticket counter, decide them (WIPT consecutive items per thread) and form the output
// offsets inside the tile with one block scan.  The tile's place in the outputs comes
// from a decoupled look-back over the tiles before it: each tile publishes its counts,
// then its inclusive prefix, as one 64-bit word (tag << 32 | value) per counter; a
// waiting tile adds published counts backwards, 32 tiles per warp read, until it meets a
// prefix.  Tickets are
// handed out in tile order to running blocks, so every tile waited on has started and
// publishes its counts without waiting itself.  The outputs therefore keep the frontier
// order: every list the walk emits is a fixed function of the tree.  The tags carry the
// step index, so the status words are cleared once per walk.
constexpr int WIPT = 4, WTILE = WB * WIPT;


__global__ void __launch_bounds__(WB, 6) walk_step_k(const int2* __restrict__ fr_in, int2* __restrict__ fr_out,
                                                  WalkCounters* __restrict__ cnt, int par, int step,
                                                  unsigned long long* __restrict__ status, NodeView nv,
                                                  double theta, float th2, int2* __restrict__ m2l, int cap_m2l,
                                                  int2* __restrict__ p2p, int cap_p2p, int cap_fr,
                                                  long long spin_limit, unsigned tag_bias) {
    __shared__ int s_tile;
    __shared__ int sbase[3];
    // after a wait ran out in an earlier step the frontier may hold slots that no tile
    // wrote: the remaining steps read nothing (the host reports FMM_ERR_TIMEOUT)
    if (cnt->err) return;
    int nf = min(cnt->nf[par], cap_fr);  // a frontier beyond the buffer was not stored (retried)
    int bm = cnt->n_m2l, bp = cnt->n_p2p;
    int ntiles = (nf + WTILE - 1) / WTILE;
    const unsigned tag_agg = 2u * (unsigned)step + 1u, tag_pre = 2u * (unsigned)step + 2u;
    // the tags a waiting tile looks for: the published ones, unless a test of the timeout
    // path sets tag_bias != 0, which no tile publishes (every wait then runs out)
    const unsigned want_agg = tag_agg + tag_bias, want_pre = tag_pre + tag_bias;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&cnt->ticket, 1);
        __syncthreads();
        int tile = s_tile;
        if (tile >= ntiles) break;
        int64_t i0 = (int64_t)tile * WTILE + (int64_t)threadIdx.x * WIPT;
        int2 it[WIPT];
        int d[WIPT], nnew[WIPT];
        bool sa[WIPT];
        if (i0 + WIPT <= nf) {
            const int4* f4 = reinterpret_cast<const int4*>(fr_in + i0);
            int4 u = f4[0], v = f4[1];
            it[0] = make_int2(u.x, u.y);
            it[1] = make_int2(u.z, u.w);
            it[2] = make_int2(v.x, v.y);
            it[3] = make_int2(v.z, v.w);
        } else {
#pragma unroll
            for (int j = 0; j < WIPT; j++) it[j] = i0 + j < nf ? fr_in[i0 + j] : make_int2(0, 0);
        }
        Cnt3 mine{0, 0, 0};
#pragma unroll
        for (int j = 0; j < WIPT; j++) {
            d[j] = -1;
            nnew[j] = 0;
            sa[j] = false;
            if (i0 + j < nf) d[j] = decide(nv, it[j], theta, th2, &nnew[j], &sa[j]);
            mine.a += d[j] == 1;
            mine.b += d[j] == 2;
            mine.c += d[j] == 0 ? nnew[j] : 0;
        }
        Cnt3 tot;
        Cnt3 off = block_exclusive_scan(mine, &tot);
        if (threadIdx.x < 96) {
            // warp q claims counter q: publish the tile's count, look back over the tiles
            // before it 32 at a time (lane l reads tile t - l) until one has published its
            // prefix, then publish this tile's prefix
            int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
            int v = q == 0 ? tot.a : (q == 1 ? tot.b : tot.c);
            unsigned long long* word = status + q;  // counter q of tile t: word[3 t]
            int ex = 0;
            if (tile > 0) {
                if (lane == 0) st_status(word + 3 * (int64_t)tile, tag_agg, v);
                int t = tile - 1;
                long long spins = 0;
                for (;;) {
                    int u = t - lane;
                    // before tile 0 every counter starts at 0: a published prefix of 0
                    unsigned long long w = u >= 0 ? ld_status(word + 3 * (int64_t)u) : (unsigned long long)want_pre << 32;
                    unsigned tag = (unsigned)(w >> 32);
                    unsigned pre = __ballot_sync(FULL, tag == want_pre);
                    unsigned wait = __ballot_sync(FULL, tag != want_pre && tag != want_agg);
                    int first = pre ? __ffs(pre) - 1 : 32;  // nearest tile with a prefix
                    unsigned need = first >= 31 ? FULL : ((2u << first) - 1u);
                    if (wait & need) {  // a tile in the window has not published yet
                        if (++spins > spin_limit) {
                            if (lane == 0) atomicExch(&cnt->err, 1);
                            break;
                        }
                        __nanosleep(32);
                        continue;
                    }
                    int val = lane <= first ? (int)(unsigned)w : 0;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(FULL, val, o);
                    ex += val;
                    if (first < 32) break;
                    t -= 32;
                }
            }
            if (lane == 0) {
                st_status(word + 3 * (int64_t)tile, tag_pre, ex + v);
                if (tile == ntiles - 1) cnt->step_tot[q] = ex + v;
                sbase[q] = ex + (q == 0 ? bm : (q == 1 ? bp : 0));
            }
        }
        __syncthreads();
        int om = sbase[0] + off.a, op = sbase[1] + off.b, of = sbase[2] + off.c;
#pragma unroll
        for (int j = 0; j < WIPT; j++) {
            if (d[j] == 1) {
                if (om < cap_m2l) m2l[om] = it[j];
                om++;
            } else if (d[j] == 2) {
                if (op < cap_p2p) p2p[op] = it[j];
                op++;
            } else if (d[j] == 0) {
                if (it[j].x == it[j].y) {
                    int c0 = nv.child_first[it[j].x], nc = nv.nchild[it[j].x];
                    int k = of;
                    for (int a = 0; a < nc; a++)
                        for (int b = a; b < nc; b++, k++)
                            if (k < cap_fr) fr_out[k] = make_int2(c0 + a, c0 + b);
                } else {
                    int S = sa[j] ? it[j].x : it[j].y;
                    int c0 = nv.child_first[S], nc = nv.nchild[S];
                    for (int a = 0; a < nc; a++)
                        if (of + a < cap_fr)
                            fr_out[of + a] = sa[j] ? make_int2(c0 + a, it[j].y) : make_int2(it[j].x, c0 + a);
                }
                of += nnew[j];
            }
        }
        __syncthreads();  // s_tile and sbase are reused by the next tile
    }
}

// closes a step: its totals move into the running counts, its output becomes the next
// step's input, and the tickets start again; frontier overflow is recorded in *max_fr (the
// largest frontier seen)
__global__ void walk_advance_k(WalkCounters* cnt, int par, int* max_fr) {
    int nxt = cnt->step_tot[2];
    if (nxt > *max_fr) *max_fr = nxt;
    cnt->n_m2l += cnt->step_tot[0];
    cnt->n_p2p += cnt->step_tot[1];
    cnt->nf[par ^ 1] = nxt;
    cnt->nf[par] = 0;
    cnt->step_tot[0] = cnt->step_tot[1] = cnt->step_tot[2] = 0;
    cnt->ticket = 0;
}

// the walk starts with Self(root) of every system of the batch (roots are nodes 0..nsys-1)
__global__ void walk_init_k(WalkCounters* cnt, int2* fr0, int* max_fr, int nsys) {
    int sys = blockIdx.x * WB + threadIdx.x;
    if (sys < nsys) fr0[sys] = make_int2(sys, sys);
    if (sys == 0) {
        cnt->nf[0] = nsys;
        cnt->nf[1] = 0;
        cnt->n_m2l = 0;
        cnt->n_p2p = 0;
        cnt->ticket = 0;
        cnt->step_tot[0] = cnt->step_tot[1] = cnt->step_tot[2] = 0;
        cnt->err = 0;
        *max_fr = nsys;
    }
}

// ---- per-target segments of the directed lists
// Every mutual pair k = (A, B) gives a directed entry for target A (partner B) and, unless
// A == B, one for target B (partner A).  The entries are laid out in pair order (2k for A,
// 2k + 1 for B) and stably radix-sorted by target, so every target's segment lists its
// partners in the order the walk emitted the pairs, which is fixed by the tree.  The value
// kept is the partner (M2L) or pair << 1 | side (P2P).  A self pair's second entry takes
// the key 2^bits - 1, above every node id, and sorts past the last segment.

__global__ void seg_expand_k(const int2* __restrict__ pairs, int64_t n, bool payload, uint32_t none,
                             uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    int64_t k = (int64_t)blockIdx.x * WB + threadIdx.x;
    if (k >= n) return;
    int2 p = pairs[k];
    keys[2 * k] = (uint32_t)p.x;
    keys[2 * k + 1] = p.x != p.y ? (uint32_t)p.y : none;
    vals[2 * k] = payload ? (uint32_t)(2 * k) : (uint32_t)p.y;
    vals[2 * k + 1] = payload ? (uint32_t)(2 * k + 1) : (uint32_t)p.x;
}

// seg[t] = the first sorted entry whose target is >= t, t = 0..nn
__global__ void seg_bounds_k(const uint32_t* __restrict__ keys, int64_t ne, int nn, long long* __restrict__ seg) {
    int t = blockIdx.x * WB + threadIdx.x;
    if (t > nn) return;
    int64_t lo = 0, hi = ne;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < (uint32_t)t)
            lo = mid + 1;
        else
            hi = mid;
    }
    seg[t] = lo;
}

// source id of every directed M2L entry (pair << 1 | side): side 0 is the entry of the
// pair's first cell, whose partner is the second (M2L pairs are never self pairs, so all
// 2n entries lie inside the segments)
__global__ void m2l_src_k(int64_t ne, const uint32_t* __restrict__ dirp, const int2* __restrict__ pairs,
                          uint32_t* __restrict__ dir) {
    int64_t e = (int64_t)blockIdx.x * WB + threadIdx.x;
    if (e >= ne) return;
    uint32_t v = dirp[e];
    int2 pr = pairs[v >> 1];
    dir[e] = (uint32_t)((v & 1u) ? pr.x : pr.y);
}

// Partial slots of the P2P pairs, laid out in target order: every sorted directed entry e
// (target t = keys[e]) owns count[t] consecutive slots, so a target's partials form one
// contiguous run in its segment order and the per-particle gather reads them as a stream.
// Target t's run starts at tbase[t], the exclusive scan of tsz[t] = (seg[t+1] - seg[t]) count[t]
// over the targets; entry e of t starts at tbase[t] + (e - seg[t]) count[t].
__global__ void p2p_tslots_k(const long long* __restrict__ seg, int nn, const int* __restrict__ count,
                             long long* __restrict__ tsz) {
    int t = blockIdx.x * WB + threadIdx.x;
    if (t >= nn) return;
    tsz[t] = (seg[t + 1] - seg[t]) * (long long)count[t];
}

// pslot[pair << 1 | side] = first slot of that directed entry (the unused second entry of a
// self pair sorts past the last target and gets none)
__global__ void p2p_slot_of_k(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ dval, int64_t ne,
                              int nn, const long long* __restrict__ seg, const long long* __restrict__ tbase,
                              const int* __restrict__ count, long long* __restrict__ pslot) {
    int64_t e = (int64_t)blockIdx.x * WB + threadIdx.x;
    if (e >= ne) return;
    uint32_t t = keys[e];
    if (t < (uint32_t)nn) pslot[dval[e]] = tbase[t] + (e - seg[t]) * (long long)count[t];
}

// builds seg[0..nn] and the per-target lists out[] of the pairs[0..n)
static void build_segments(fmm_ctx* c, const int2* pairs, int64_t n, int nn, bool payload, DevBuf& seg_buf,
                           DevBuf& out_buf) {
    cudaStream_t s = c->stream;
    int bits = c->id_bits;
    int64_t ne = 2 * n;
    ensure(seg_buf, sizeof(long long) * (size_t)(nn + 1));
    ensure(c->seg_k, sizeof(uint32_t) * (size_t)(ne > 0 ? ne : 1));
    ensure(out_buf, sizeof(uint32_t) * (size_t)(ne > 0 ? ne : 1));
    if (n > 0) {
        seg_expand_k<<<grid_for(n, WB), WB, 0, s>>>(pairs, n, payload, (uint32_t)((1ll << bits) - 1),
                                                  c->seg_k.as<uint32_t>(), out_buf.as<uint32_t>());
        GB_LAUNCH("seg_expand_k");
        radix_sort32(c, c->seg_k, c->seg_k2, &out_buf, &c->seg_v2, ne, bits);
    }
    seg_bounds_k<<<grid_for(nn + 1, WB), WB, 0, s>>>(c->seg_k.as<uint32_t>(), ne, nn, seg_buf.as<long long>());
    GB_LAUNCH("seg_bounds_k");
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

// Work items of two item sets in one host round trip: both sets' chunk counts and scans,
// one read of their totals (with the segment sorts' status and the P2P partial total),
// then both fills.
static void build_item_sets(fmm_ctx* c, int n, const long long* seg_a, int ch_a, ItemSet& a,
                            const long long* seg_b, int ch_b, ItemSet& b) {
    cudaStream_t s = c->stream;
    ensure(c->seg_cnt, sizeof(int) * (size_t)(4 * n + 4));
    int* cnt_a = c->seg_cnt.as<int>();
    int* cnt_b = cnt_a + 2 * n + 2;
    ItemSet* sets[2] = {&a, &b};
    const long long* segs[2] = {seg_a, seg_b};
    int chs[2] = {ch_a, ch_b};
    int* cnts[2] = {cnt_a, cnt_b};
    for (int k = 0; k < 2; k++) {
        ItemSet& it = *sets[k];
        int* nfull = cnts[k];
        int* npart = nfull + n + 1;
        ensure(it.fo, sizeof(long long) * (size_t)(n + 1));
        ensure(it.po, sizeof(long long) * (size_t)(n + 1));
        items_count_k<<<grid_for(n, WB), WB, 0, s>>>(segs[k], n, chs[k], nfull, npart);
        GB_LAUNCH("items_count_k");
        scan_i64(c, nfull, n, it.fo.as<long long>());
        scan_i64(c, npart, n, it.po.as<long long>());
    }
    HostReads hr(c);
    const long long* tot[2][2];
    for (int k = 0; k < 2; k++) {
        tot[k][0] = hr.read<long long>(sets[k]->fo.as<long long>() + n);
        tot[k][1] = hr.read<long long>(sets[k]->po.as<long long>() + n);
    }
    const long long* p2p_total = hr.read<long long>(c->p2p_pbase.as<long long>() + n);
    const int* hserr = hr.read<int>(sort_err(c));  // the segment sorts before this read
    hr.wait();
    sort_err_throw(c, *hserr);
    c->p2p_total = *p2p_total;
    for (int k = 0; k < 2; k++) {
        ItemSet& it = *sets[k];
        it.n_full = *tot[k][0];
        it.n_items = *tot[k][0] + *tot[k][1];
        it.chunk = chs[k];
        ensure(it.items, sizeof(int4) * (size_t)(it.n_items > 0 ? it.n_items : 1));
        items_fill_k<<<grid_for(n, WB), WB, 0, s>>>(segs[k], n, chs[k], it.fo.as<long long>(), it.po.as<long long>(),
                                                    it.n_full, it.items.as<int4>());
        GB_LAUNCH("items_fill_k");
    }
}

static int bits_for(int64_t nn) {
    int b = 1;
    while (((int64_t)1 << b) <= nn) b++;  // ids < 2^b - 1 always
    return b;
}

void run_walk(fmm_ctx* c, double theta) {
    cudaStream_t s = c->stream;
    // the pair buffers are rewritten below: until this walk has finished, no list is valid
    c->list_theta = -1.0;
    NodeView nv = node_view(c);
    int64_t nn = c->n_nodes;
    // fixed number of steps, no host round trip between them; one retry if a buffer overflowed
    int steps = 2 * c->n_levels + 2;
    float th2 = (float)theta * (float)theta;  // prefilter only; relative error far inside its margin
    int dev_sms = 0;
    GB_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c->device));
    int grid = dev_sms * 8;
    int64_t n_m2l = 0, n_p2p = 0;
    for (int attempt = 0;; attempt++) {
        int64_t cap_fr = c->cap_fr, cap_m2l = c->cap_m2l, cap_p2p = c->cap_p2p;
        ensure(c->fr0, sizeof(int2) * (size_t)cap_fr);
        ensure(c->fr1, sizeof(int2) * (size_t)cap_fr);
        ensure(c->m2l_pairs, sizeof(int2) * (size_t)cap_m2l);
        ensure(c->p2p_pairs, sizeof(int2) * (size_t)cap_p2p);
        ensure(c->cnt, sizeof(WalkCounters) + 16);
        WalkCounters* cnt = reinterpret_cast<WalkCounters*>(c->cnt.p);
        int* max_fr = reinterpret_cast<int*>(cnt + 1);
        size_t nstat = 3 * (size_t)(cap_fr / WTILE + 1);
        ensure(c->walk_status, sizeof(unsigned long long) * nstat);
        unsigned long long* status = c->walk_status.as<unsigned long long>();
        GB_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned long long) * nstat, s));
        walk_init_k<<<grid_for(c->n_sys, WB), WB, 0, s>>>(cnt, c->fr0.as<int2>(), max_fr, c->n_sys);
        GB_LAUNCH("walk_init_k");
        for (int k = 0; k < steps; k++) {
            int par = k & 1;
            int2* fin = par ? c->fr1.as<int2>() : c->fr0.as<int2>();
            int2* fout = par ? c->fr0.as<int2>() : c->fr1.as<int2>();
            walk_step_k<<<grid, WB, 0, s>>>(fin, fout, cnt, par, k, status, nv, theta, th2, c->m2l_pairs.as<int2>(),
                                            (int)cap_m2l, c->p2p_pairs.as<int2>(), (int)cap_p2p, (int)cap_fr,
                                            c->walk_spin_limit, c->walk_wait_never ? 0x40000000u : 0u);
            GB_LAUNCH("walk_step_k");
            walk_advance_k<<<1, 1, 0, s>>>(cnt, par, max_fr);
            GB_LAUNCH("walk_advance_k");
        }
        HostReads hr(c);
        const WalkCounters* hh = hr.read<WalkCounters>(cnt);
        const int* hhmax = hr.read<int>(max_fr);
        const int* hserr = hr.read<int>(sort_err(c));  // a sort of the build (node order by leaf size) that gave up
        hr.wait();
        WalkCounters h = *hh;
        int hmax = *hhmax, serr = *hserr;
        sort_err_throw(c, serr);
        if (h.err) throw FmmError{FMM_ERR_TIMEOUT, "walk: a frontier tile waited too long for the tiles before it"};
        if (h.nf[0] != 0 || h.nf[1] != 0) throw FmmError{FMM_ERR_CAPACITY, "walk did not finish in 2 x levels + 2 steps"};
        bool over = h.n_m2l > cap_m2l || h.n_p2p > cap_p2p || hmax > cap_fr;
        if (h.n_m2l < 0 || h.n_p2p < 0 || hmax < 0) throw FmmError{FMM_ERR_CAPACITY, "walk counters above 2^31"};
        if (over) {
            // a truncated frontier under-reports what the later steps need: grow each
            // overflowing buffer to at least twice its size and try again
            if (attempt >= 10) throw FmmError{FMM_ERR_CAPACITY, "walk buffers still overflow after 10 retries"};
            if (h.n_m2l > cap_m2l) c->cap_m2l = std::max<int64_t>(2 * cap_m2l, (int64_t)h.n_m2l + h.n_m2l / 8);
            if (h.n_p2p > cap_p2p) c->cap_p2p = std::max<int64_t>(2 * cap_p2p, (int64_t)h.n_p2p + h.n_p2p / 8);
            if (hmax > cap_fr) c->cap_fr = std::max<int64_t>(2 * cap_fr, (int64_t)hmax + hmax / 8);
            c->walk_retries++;
            continue;
        }
        n_m2l = h.n_m2l;
        n_p2p = h.n_p2p;
        break;
    }
    c->n_m2l = n_m2l;
    c->n_p2p = n_p2p;
    int bits = bits_for(nn);
    c->id_bits = bits;
    // M2L: per-target segments of source ids; binary64 also keeps every entry's
    // (pair << 1 | side) for the shared pair tensors of its M2L
    if (c->precision == FMM_FP64) {
        build_segments(c, c->m2l_pairs.as<int2>(), n_m2l, (int)nn, true, c->m2l_seg, c->m2l_dirp);
        ensure(c->m2l_dir, sizeof(uint32_t) * (size_t)(n_m2l > 0 ? 2 * n_m2l : 1));
        if (n_m2l > 0) {
            m2l_src_k<<<grid_for(2 * n_m2l, WB), WB, 0, s>>>(2 * n_m2l, c->m2l_dirp.as<uint32_t>(),
                                                            c->m2l_pairs.as<int2>(), c->m2l_dir.as<uint32_t>());
            GB_LAUNCH("m2l_src_k");
        }
    } else {
        build_segments(c, c->m2l_pairs.as<int2>(), n_m2l, (int)nn, false, c->m2l_seg, c->m2l_dir);
    }
    // P2P: per-target segments of (pair << 1 | side) in list order, then the partial
    // slots in that order (p2p_pbase: first slot of every target, [nn] the total;
    // p2p_off: first slot of every pair << 1 | side)
    build_segments(c, c->p2p_pairs.as<int2>(), n_p2p, (int)nn, true, c->p2p_seg, c->p2p_dval);
    int64_t ne_p = 2 * n_p2p;
    ensure(c->p2p_psize, sizeof(long long) * (size_t)(nn + 1));
    ensure(c->p2p_pbase, sizeof(long long) * (size_t)(nn + 1));
    ensure(c->p2p_off, sizeof(long long) * (size_t)(ne_p > 0 ? ne_p : 1));
    p2p_tslots_k<<<grid_for(nn, WB), WB, 0, s>>>(c->p2p_seg.as<long long>(), (int)nn, c->ncount.as<int>(),
                                                c->p2p_psize.as<long long>());
    GB_LAUNCH("p2p_tslots_k");
    scan_i64_from_i64(c, c->p2p_psize.as<long long>(), nn, c->p2p_pbase.as<long long>());
    if (ne_p > 0) {
        p2p_slot_of_k<<<grid_for(ne_p, WB), WB, 0, s>>>(c->seg_k.as<uint32_t>(), c->p2p_dval.as<uint32_t>(), ne_p,
                                                       (int)nn, c->p2p_seg.as<long long>(),
                                                       c->p2p_pbase.as<long long>(), c->ncount.as<int>(),
                                                       c->p2p_off.as<long long>());
        GB_LAUNCH("p2p_slot_of_k");
    }
    // work items: m2l_chunk M2L sources (default 32) and p2p_chunk P2P entries (64) per chunk
    build_item_sets(c, (int)nn, c->m2l_seg.as<long long>(), c->m2l_chunk, c->m2l_items, c->p2p_seg.as<long long>(),
                    c->p2p_chunk, c->p2p_items);
    c->list_theta = theta;
    c->walk_gen++;
    c->p2p_total_gen = c->walk_gen;  // read with the item totals
}

}  // namespace gbfmm
