// Internal state of a gbfmm context and the host-side launchers shared by the
// translation units of the CUDA library.  Not part of the public C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gbfmm.h"
#include "fmm_device.cuh"

namespace gbfmm {

// Grow-only device buffer.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    template <class T>
    T* as() const {
        return static_cast<T*>(p);
    }
};

// Error carried out of the launchers as a C++ exception and turned into a status
// code at the C boundary.
struct FmmError {
    int code;
    std::string msg;
};

void cuda_check(cudaError_t e, const char* what);
void count_launch();
#define GB_CUDA(call) ::gbfmm::cuda_check((call), #call)
#define GB_LAUNCH(what) (::gbfmm::count_launch(), ::gbfmm::cuda_check(cudaGetLastError(), what))

// Node arrays (breadth-first order); all device pointers.
struct NodeView {
    const int* first;
    const int* count;
    const int* parent;
    const int* child_first;
    const int* nchild;
    const double* Zx;
    const double* Zy;
    const double* Zz;
    const double* rmax;
    const float4* zh;  // (hi(Z), r_max rounded up) in binary32
    const float4* zl;  // (lo(Z), 0)
};

// Chunked work over per-cell segments (see build_item_sets in walk.cu).
struct ItemSet {
    DevBuf items;   // int4 (cell, entry begin, entry end, -)
    DevBuf fo, po;  // long long [n + 1]: full-chunk offsets, partial-chunk ranks
    int64_t n_full = 0, n_items = 0;
    int chunk = 0;
};

constexpr int M2L_CHUNK = 32;
constexpr int M2L_CHUNK_MIXED = 64;  // default in FMM_MIXED
constexpr int P2P_CHUNK = 64;
// polls of one status word before a walk tile gives up waiting for the tiles before it
// (~0.1-1 s; never reached in a correct run)
constexpr long long WALK_SPIN_LIMIT = 1ll << 22;

enum Stage {
    ST_BUILD = 0,   // bounding cube .. r_max
    ST_MOMENTS,     // P2M + M2M
    ST_WALK,        // dual-tree walk + list canonicalisation
    ST_M2L,         // M2L (target-major, both partners of every mutual pair)
    ST_L2L,         // L2L
    ST_P2P,         // mutual P2P tiles
    ST_L2P,         // L2P + particle reduction + unpermute
    ST_COUNT
};

}  // namespace gbfmm

struct fmm_ctx {
    int device = 0;
    int precision = FMM_FP64;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // particles
    int64_t N = 0;
    int leaf = 0;
    bool built = false;
    // systems of a batch: particles [off[s], off[s+1]) (one system for fmm_build)
    int n_sys = 1;
    std::vector<long long> sys_off_h;
    gbfmm::DevBuf sys_off, sys_k, sys_v, sys_diag;
    // device buffers (see the kernels for layouts)
    gbfmm::DevBuf x_stage, m_stage;           // host inputs staged on the device
    gbfmm::DevBuf keys0, keys1, vals0, vals1;  // sort ping-pong
    gbfmm::DevBuf xs, ys, zs, ms;              // sorted SoA positions and masses
    gbfmm::DevBuf perm;                        // sorted position -> input index (uint32)
    gbfmm::DevBuf flags, scan_out, scan_tmp, geom, errflag;
    gbfmm::DevBuf rs_hist;                     // radix sort digit totals, tickets and offsets
    gbfmm::DevBuf rs_status;                   // radix sort look-back words (tile x digit)
    gbfmm::DevBuf rs_err;                      // set by a radix sort tile whose wait gave up
    unsigned rs_epoch = 0;                     // last look-back tag handed out
    gbfmm::DevBuf leaf_of;                     // leaf of every sorted particle
    // nodes
    int64_t n_nodes = 0, cap_nodes = 0;
    int n_levels = 0;                          // levels 0 .. n_levels-1
    std::vector<int> level_start;              // size n_levels + 1
    gbfmm::DevBuf lvl_ctl, lvl_status;         // octree level table and look-back words (build)
    gbfmm::DevBuf nfirst, ncount, nlevel, nparent, nchildf, nnchild;
    gbfmm::DevBuf nM, nSx, nSy, nSz, nZx, nZy, nZz, nr2, nrmax;
    gbfmm::DevBuf nr2f;                        // binary32 estimate of r_max^2 (prefilter)
    gbfmm::DevBuf leaf_key, leaf_key2, leaf_order, leaf_order2;  // nodes by leaf size (per-leaf kernels)
    // expansions
    int mom_p = -1;
    gbfmm::DevBuf mom;   // n_nodes x nmi(p)
    gbfmm::DevBuf loc;   // n_nodes x (nmi(p) | 4 nmi(p-1))
    gbfmm::DevBuf locp;  // standard locals for potentials of the conserving form
    gbfmm::DevBuf locT, locpT;  // leaf locals in leaf units, pair-kernel type (scaled-mode L2P)
    // lists
    double list_theta = -1.0;
    int64_t n_m2l = 0, n_p2p = 0;
    gbfmm::DevBuf fr0, fr1, cnt, cnt_off;      // walk frontier and counters
    int64_t cap_fr = 1 << 16, cap_m2l = 1 << 16, cap_p2p = 1 << 16;   // walk buffer sizes (grow only)
    bool caps_user = false;                    // sizes set by fmm_set_walk_capacity
    int m2l_chunk = gbfmm::M2L_CHUNK;          // directed M2L entries per work item (fmm_set_tiles)
    int p2p_chunk = gbfmm::P2P_CHUNK;          // directed P2P entries per reduction item
    int64_t walk_retries = 0;                  // walks re-run after a buffer overflow
    long long walk_spin_limit = gbfmm::WALK_SPIN_LIMIT;  // polls per look-back wait (fmm_set_wait_limit)
    bool walk_wait_never = false;              // test of the timeout path: no wait is ever satisfied
    int schedule = FMM_SCHEDULE_LISTS;         // fmm_set_schedule
    double fused_theta = 0.0;                  // theta of the running fused evaluation
    gbfmm::DevBuf p2p_direct;                  // fused schedule: per-particle P2P sums (Quad<double>)
    gbfmm::DevBuf m2l_pairs, p2p_pairs;        // int2, walk order
    gbfmm::DevBuf m2l_dir;                     // uint32 source ids, per-target segments in list order
    gbfmm::DevBuf m2l_dirp;                    // uint32 (pair << 1 | side) of the same entries
    gbfmm::DevBuf m2l_pth, m2l_ptd;            // binary64 h and D tensors of every M2L pair
    int64_t pth_gen = -1, ptd_gen = -1;        // walk the pair tensors belong to ...
    int pth_p = -1, ptd_p = -1;                // ... and their order
    gbfmm::DevBuf m2l_seg;                     // int64 [n_nodes + 1] segment starts per target
    gbfmm::DevBuf p2p_dval;                    // uint32 (pair << 1 | side), per-target segments in list order
    gbfmm::DevBuf p2p_seg;                     // int64 [n_nodes + 1]
    gbfmm::DevBuf p2p_psize;                   // int64 partial slots per target node
    gbfmm::DevBuf seg_k, seg_k2, seg_v2;       // directed-entry keys of the list sort (+ scratch)
    gbfmm::DevBuf walk_status;                 // per-tile look-back words of the walk steps
    gbfmm::DevBuf seg_cnt;                     // per-segment chunk counts of the work items
    gbfmm::DevBuf p2p_off;                     // int64 [2 n_p2p] first partial slot of pair << 1 | side
    gbfmm::DevBuf p2p_part;                    // double4 partials
    gbfmm::ItemSet m2l_items, p2p_items;
    gbfmm::DevBuf m2l_part;                    // M2L partial locals per item
    gbfmm::DevBuf p2p_islot;                   // long long [items + 1]: slot offsets of P2P items
    gbfmm::DevBuf p2p_ipart;                   // double4 per (P2P item, slot)
    gbfmm::DevBuf cmom;                        // conserving source moments, n_nodes x 4 nmi(p-1)
    gbfmm::DevBuf m2m_tmp;                     // shifted child moments of one level
    gbfmm::DevBuf lf_x, lf_v, lf_m, lf_a, lf_diag;  // leapfrog state (input order)
    gbfmm::DevBuf tune_acc;                    // output of the autotuner's trial evaluations
    gbfmm::DevBuf pos4;                        // packed (x, y, z, m) per sorted particle, storage type
    gbfmm::DevBuf p2p_sep;                     // centre separation of every P2P pair, storage type
    gbfmm::DevBuf p2p_cls, p2p_cls2;           // ring-kernel class keys of the P2P pairs (+ sort scratch)
    gbfmm::DevBuf p2p_list, p2p_list2;         // P2P pair ids in class order (+ sort scratch)
    gbfmm::DevBuf p2p_tab;                     // ring class table: start, count, warp prefix per width
    gbfmm::DevBuf p2p_desc;                    // ring descriptors of the P2P pairs in class order (binary32)
    int64_t walk_gen = 0, p2p_cls_gen = -1;    // walks run so far; walk the classes belong to
    int64_t gather_gen = -1;                   // walk the P2P item slots and entry bases belong to
    int64_t p2p_total_gen = -1;                // walk p2p_total belongs to
    long long p2p_total = 0;                   // P2P partial slots of that walk
    // fmm_forces_graph: the recorded evaluation and what it was recorded for
    int64_t op_gen = 0;                        // builds and settings (change what a recorded graph assumes)
    cudaGraphExec_t graph_exec = nullptr;
    bool capturing = false;                    // inside the recording (stage timers off)
    int64_t graph_op_gen = -1, graph_walk_gen = -1;
    int graph_mom_p = -1;
    long long graph_reallocs = -1;
    int graph_p = 0, graph_variant = 0;
    double graph_theta = -1.0;
    double *graph_acc = nullptr, *graph_pot = nullptr;
    long long p2p_nslots = 0;                  // particle slots over all P2P reduction items
    gbfmm::DevBuf p2p_pbase;                   // int64 [n_nodes + 1] first partial slot of every target node
    bool pos_valid = false;
    gbfmm::DevBuf momT;                        // raw moments in the pair-kernel type (range-scaled, padded)
    gbfmm::DevBuf nk;                          // per-node moment unit exponent (scaled modes)
    gbfmm::DevBuf zhl;                         // double-float node centres: float4 hi[n] | lo[n] (build)
    gbfmm::DevBuf m2l_kpart;                   // per-item unit exponent of the M2L partials
    int id_bits = 0;
    // results (sorted order) and output staging
    gbfmm::DevBuf acc_s, pot_s;                // SoA: ax | ay | az
    gbfmm::DevBuf out_stage;
    gbfmm::DevBuf diag_tmp;
    bool have_forces = false;
    // second stream for stages that do not depend on each other (the moments beside the
    // walk; the pair kernels beside the far field), forked from and joined back into
    // `stream` by events
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    // page-locked host words for the small device values the host reads (list sizes,
    // status flags): copies into them are asynchronous, so one read point costs one stream
    // synchronisation however many values it reads (gbfmm::HostReads)
    void* hpin = nullptr;
    int overlap = FMM_OVERLAP_MOMENTS_WALK;    // fmm_set_overlap
    // timing
    cudaEvent_t ev[2 * gbfmm::ST_COUNT] = {};
    float stage_ms[gbfmm::ST_COUNT] = {};
    bool stage_valid[gbfmm::ST_COUNT] = {};
};

namespace gbfmm {

// buffers
void ensure(DevBuf& b, size_t bytes);                              // grow, contents lost
void ensure_keep(DevBuf& b, size_t bytes, cudaStream_t s);         // grow, contents kept
void release(DevBuf& b);
long long realloc_count();  // allocations and frees of DevBufs so far (all contexts)

// scans (launch.cu); out must hold n + 1 entries, out[n] = total
void scan_int(fmm_ctx* c, const int* in, int64_t n, int* out);
void scan_i64(fmm_ctx* c, const int* in, int64_t n, long long* out);
void scan_i64_from_i64(fmm_ctx* c, const long long* in, int64_t n, long long* out);
// radix sort of keys [+ values] on bits [0, bits); result in place
void radix_sort(fmm_ctx* c, DevBuf& keys, DevBuf& keys_tmp, DevBuf* vals, DevBuf* vals_tmp, int64_t n, int bits);
// the same on 32-bit keys
void radix_sort32(fmm_ctx* c, DevBuf& keys, DevBuf& keys_tmp, DevBuf* vals, DevBuf* vals_tmp, int64_t n, int bits);
// the sorts' wait-timeout flag (device int, zero until a look-back gives up), and the check
// of its value read at a host read point (throws FMM_ERR_TIMEOUT and clears it)
int* sort_err(fmm_ctx* c);
void sort_err_throw(fmm_ctx* c, int flag);

// tree (tree.cu)
int build_tree(fmm_ctx* c, const double* x_dev, const double* m_dev);

// walk (walk.cu)
void run_walk(fmm_ctx* c, double theta);

// expansions (expansion_p*.cu, dispatched in expansion.cu)
void run_moments(fmm_ctx* c, int p);
void run_far_field(fmm_ctx* c, int p, int variant, bool want_pot);

// particle-particle + final reduction (p2p.cu): set-up (positions, ring classes, partial
// buffer, separations; may read sizes on the host once per walk), then the pair kernels
void run_p2p(fmm_ctx* c, bool want_pot);
void run_p2p_prepare(fmm_ctx* c);
void run_p2p_kernels(fmm_ctx* c, bool want_pot);

// Small device values read on the host at one point: read() queues an asynchronous copy
// into the context's page-locked words and returns where the value will be; wait()
// synchronises the stream once, after which every returned pointer holds its value.
constexpr size_t HPIN_BYTES = 4096;
struct HostReads {
    fmm_ctx* c;
    size_t off = 0;
    explicit HostReads(fmm_ctx* ctx) : c(ctx) {}
    template <class T>
    T* read(const void* dev_src, size_t count = 1) {
        off = (off + 15) & ~(size_t)15;
        size_t bytes = sizeof(T) * count;
        if (off + bytes > HPIN_BYTES) throw FmmError{FMM_ERR_CAPACITY, "host read words exhausted"};
        T* dst = reinterpret_cast<T*>(static_cast<char*>(c->hpin) + off);
        off += bytes;
        cuda_check(cudaMemcpyAsync(dst, dev_src, bytes, cudaMemcpyDeviceToHost, c->stream), "host read");
        return dst;
    }
    void wait() { cuda_check(cudaStreamSynchronize(c->stream), "host read wait"); }
};

// The side stream: fork_side makes c->side wait for the work queued on c->stream so far;
// while a SideLaunches is alive, the launchers (which all queue on c->stream) queue on the
// side stream; join_side makes c->stream wait for the side stream's work.
void fork_side(fmm_ctx* c);
void join_side(fmm_ctx* c);
struct SideLaunches {
    fmm_ctx* c;
    cudaStream_t main;
    explicit SideLaunches(fmm_ctx* ctx);
    ~SideLaunches();
};
// the fused schedule's near field: per-particle P2P sums into c->p2p_direct (p2p.cu)
void run_p2p_fused(fmm_ctx* c, bool want_pot, double theta);
void run_p2p_gather(fmm_ctx* c);

// high-order (p = 7, 8) binary64 M2L into the item partials and L2L of one level
// (high_order.cu)
void m2l_generic_launch(fmm_ctx* c, int p, int variant, double* part);
void l2l_generic_launch(fmm_ctx* c, int p, int variant, int lo, int hi, double* loc);
void run_gather_out(fmm_ctx* c, int p, int variant, bool want_pot, double* acc_out, double* pot_out);
void run_diagnostics(fmm_ctx* c, double* out6_host);
void run_diagnostics_sys(fmm_ctx* c, double* out_dev);

void stage_begin(fmm_ctx* c, Stage s);
void stage_end(fmm_ctx* c, Stage s);

NodeView node_view(const fmm_ctx* c);

}  // namespace gbfmm
