// The C ABI of gbfmm (include/gbfmm.h): argument checks, host/device staging of inputs
// and outputs, the order of the stages, and the conversion of errors to status codes.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "fmm_device.cuh"
#include "fmm_internal.h"

namespace gbfmm {
long long launches();
void run_moments_dispatch(fmm_ctx* c, int p);
void run_far_field_dispatch(fmm_ctx* c, int p, int variant, bool want_pot);
void run_finish_dispatch(fmm_ctx* c, int p, int variant, bool want_pot, double* acc, double* pot);
}  // namespace gbfmm

using namespace gbfmm;

static thread_local std::string g_last_error;

namespace gbfmm {
void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace gbfmm

static int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

// true when ptr is device (or managed) memory
static bool is_device_ptr(const void* ptr) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d) {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <class F>
static int guarded(fmm_ctx* c, F&& f) {
    try {
        DeviceGuard g(c->device);
        return f();
    } catch (const FmmError& e) {
        return fail(e.code, e.msg);
    } catch (const std::bad_alloc&) {
        return fail(FMM_ERR_OOM, "host allocation failed");
    }
}

extern "C" {

const char* fmm_strerror(int status) {
    switch (status) {
        case FMM_OK: return "ok";
        case FMM_ERR_INVALID: return "invalid argument";
        case FMM_ERR_STATE: return "call out of order";
        case FMM_ERR_CUDA: return "CUDA runtime error";
        case FMM_ERR_OOM: return "out of device memory";
        case FMM_ERR_CAPACITY: return "internal size limit exceeded";
        case FMM_ERR_TIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

const char* fmm_last_error(void) { return g_last_error.c_str(); }

int64_t fmm_kernel_launches(void) { return (int64_t)launches(); }

int fmm_create(fmm_ctx** out, int device, int precision, void* cuda_stream) {
    if (!out) return fail(FMM_ERR_INVALID, "fmm_create: out is NULL");
    if (precision != FMM_FP64 && precision != FMM_MIXED && precision != FMM_DF64)
        return fail(FMM_ERR_INVALID, "fmm_create: unknown precision");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(FMM_ERR_CUDA, "fmm_create: no such CUDA device");
    }
    fmm_ctx* c = new (std::nothrow) fmm_ctx();
    if (!c) return fail(FMM_ERR_OOM, "fmm_create: host allocation failed");
    c->device = device;
    c->precision = precision;
    // the binary32 M2L is cheap next to the binary64 reduction of its item partials, so its
    // work items are longer (measured at N = 2^20: 32 entries is best in binary64, 64 in
    // binary32; double-float is indifferent)
    if (precision == FMM_MIXED) c->m2l_chunk = gbfmm::M2L_CHUNK_MIXED;
    int rc = guarded(c, [&]() -> int {
        if (cuda_stream) {
            c->stream = static_cast<cudaStream_t>(cuda_stream);
        } else {
            GB_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
            c->own_stream = true;
        }
        GB_CUDA(cudaMallocHost(&c->hpin, gbfmm::HPIN_BYTES));
        // the side stream and its fork/join events (independent stages of fmm_forces)
        GB_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
        GB_CUDA(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
        GB_CUDA(cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming));
        return FMM_OK;
    });
    if (rc != FMM_OK) {
        if (c->side) cudaStreamDestroy(c->side);
        if (c->fork_ev) cudaEventDestroy(c->fork_ev);
        if (c->join_ev) cudaEventDestroy(c->join_ev);
        if (c->hpin) cudaFreeHost(c->hpin);
        if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
        delete c;
        return rc;
    }
    *out = c;
    return FMM_OK;
}

int fmm_destroy(fmm_ctx* c) {
    if (!c) return FMM_OK;
    {
        DeviceGuard g(c->device);
        if (c->stream) cudaStreamSynchronize(c->stream);
        DevBuf* bufs[] = {&c->x_stage, &c->m_stage, &c->keys0, &c->keys1, &c->vals0, &c->vals1, &c->xs, &c->ys,
                          &c->zs, &c->ms, &c->perm, &c->flags, &c->scan_out, &c->scan_tmp, &c->geom, &c->errflag,
                          &c->rs_hist, &c->rs_status, &c->rs_err, &c->leaf_of, &c->nfirst, &c->ncount,
                          &c->nlevel, &c->nparent, &c->nchildf, &c->nnchild, &c->nM, &c->nSx, &c->nSy, &c->nSz,
                          &c->nZx, &c->nZy, &c->nZz, &c->nr2, &c->nr2f, &c->nrmax, &c->leaf_key, &c->leaf_key2, &c->leaf_order, &c->leaf_order2, &c->mom, &c->loc, &c->locp, &c->locT, &c->locpT, &c->fr0,
                          &c->fr1, &c->cnt, &c->cnt_off, &c->m2l_pairs, &c->p2p_pairs, &c->m2l_dir, &c->m2l_dirp, &c->m2l_pth, &c->m2l_ptd, &c->m2l_seg,
                          &c->p2p_dval, &c->p2p_psize, &c->p2p_pbase, &c->seg_k, &c->seg_k2, &c->seg_v2, &c->walk_status, &c->seg_cnt, &c->p2p_seg, &c->p2p_off, &c->p2p_part,
                          &c->acc_s, &c->pot_s, &c->out_stage, &c->diag_tmp, &c->m2l_items.items,
                          &c->m2l_items.fo, &c->m2l_items.po, &c->p2p_items.items, &c->p2p_items.fo,
                          &c->p2p_items.po, &c->m2l_part, &c->p2p_islot, &c->p2p_ipart, &c->cmom, &c->pos4,
                          &c->momT, &c->nk, &c->zhl, &c->m2l_kpart, &c->p2p_sep, &c->p2p_cls, &c->p2p_cls2, &c->p2p_list, &c->p2p_list2, &c->p2p_tab, &c->p2p_desc, &c->m2m_tmp,
                          &c->lf_x, &c->lf_v,
                          &c->lf_m, &c->lf_a, &c->lf_diag, &c->tune_acc, &c->lvl_ctl, &c->lvl_status, &c->p2p_direct, &c->sys_off, &c->sys_k, &c->sys_v, &c->sys_diag};
        for (DevBuf* b : bufs) release(*b);
        if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
        for (cudaEvent_t& e : c->ev)
            if (e) cudaEventDestroy(e);
        if (c->side) {
            cudaStreamSynchronize(c->side);
            cudaStreamDestroy(c->side);
        }
        if (c->fork_ev) cudaEventDestroy(c->fork_ev);
        if (c->join_ev) cudaEventDestroy(c->join_ev);
        if (c->hpin) cudaFreeHost(c->hpin);
        if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    }
    delete c;
    return FMM_OK;
}

int fmm_set_stream(fmm_ctx* c, void* cuda_stream) {
    if (!c) return fail(FMM_ERR_INVALID, "fmm_set_stream: NULL context");
    c->op_gen++;
    return guarded(c, [&]() -> int {
        GB_CUDA(cudaStreamSynchronize(c->stream));
        if (c->own_stream) GB_CUDA(cudaStreamDestroy(c->stream));
        c->own_stream = false;
        if (cuda_stream) {
            c->stream = static_cast<cudaStream_t>(cuda_stream);
        } else {
            GB_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
            c->own_stream = true;
        }
        return FMM_OK;
    });
}

static int build_common(fmm_ctx* c, const double* x, const double* m, int64_t N, int leaf_size,
                        const std::vector<long long>& off) {
    return guarded(c, [&]() -> int {
        for (int s = 0; s < ST_COUNT; s++) c->stage_valid[s] = false;
        c->built = false;
        c->have_forces = false;
        c->mom_p = -1;
        c->list_theta = -1.0;
        c->pos_valid = false;
        c->N = N;
        // walk buffers: start from sizes that fit the usual lists (the walk grows them)
        if (!c->caps_user) {
            c->cap_m2l = std::max<int64_t>(c->cap_m2l, 16 * N + 4096);
            c->cap_p2p = std::max<int64_t>(c->cap_p2p, 4 * N + 4096);
            c->cap_fr = std::max<int64_t>(c->cap_fr, 4 * N + 4096);
        }
        c->leaf = leaf_size;
        c->n_sys = (int)off.size() - 1;
        c->sys_off_h = off;
        ensure(c->sys_off, sizeof(long long) * off.size());
        GB_CUDA(cudaMemcpyAsync(c->sys_off.p, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice,
                                c->stream));
        const double* xd = x;
        const double* md = m;
        if (!is_device_ptr(x)) {
            ensure(c->x_stage, sizeof(double) * 3 * (size_t)N);
            GB_CUDA(cudaMemcpyAsync(c->x_stage.p, x, sizeof(double) * 3 * (size_t)N, cudaMemcpyHostToDevice,
                                    c->stream));
            xd = c->x_stage.as<double>();
        }
        if (!is_device_ptr(m)) {
            ensure(c->m_stage, sizeof(double) * (size_t)N);
            GB_CUDA(cudaMemcpyAsync(c->m_stage.p, m, sizeof(double) * (size_t)N, cudaMemcpyHostToDevice, c->stream));
            md = c->m_stage.as<double>();
        }
        stage_begin(c, ST_BUILD);
        int rc = build_tree(c, xd, md);
        if (rc != FMM_OK) return fail(rc, "fmm_build: non-finite position or mass, or negative mass");
        stage_end(c, ST_BUILD);
        c->built = true;
        return FMM_OK;
    });
}

int fmm_build(fmm_ctx* c, const double* x, const double* m, int64_t N, int leaf_size) {
    if (!c) return fail(FMM_ERR_INVALID, "fmm_build: NULL context");
    c->op_gen++;
    if (!x || !m) return fail(FMM_ERR_INVALID, "fmm_build: x and m are required");
    if (N < 1) return fail(FMM_ERR_INVALID, "fmm_build: N must be >= 1");
    if (N >= ((int64_t)1 << 31) - 1) return fail(FMM_ERR_CAPACITY, "fmm_build: N must be < 2^31 - 1");
    if (leaf_size < 1) return fail(FMM_ERR_INVALID, "fmm_build: leaf_size must be >= 1");
    return build_common(c, x, m, N, leaf_size, std::vector<long long>{0, (long long)N});
}

int fmm_build_batch(fmm_ctx* c, const double* x, const double* m, const int64_t* offsets, int n_sys,
                    int leaf_size) {
    if (!c) return fail(FMM_ERR_INVALID, "fmm_build_batch: NULL context");
    c->op_gen++;
    if (!x || !m || !offsets) return fail(FMM_ERR_INVALID, "fmm_build_batch: x, m and offsets are required");
    if (n_sys < 1) return fail(FMM_ERR_INVALID, "fmm_build_batch: n_sys must be >= 1");
    if (leaf_size < 1) return fail(FMM_ERR_INVALID, "fmm_build_batch: leaf_size must be >= 1");
    std::vector<long long> off((size_t)n_sys + 1);
    if (is_device_ptr(offsets)) {
        if (cudaMemcpy(off.data(), offsets, sizeof(int64_t) * off.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return fail(FMM_ERR_CUDA, "fmm_build_batch: reading offsets failed");
        }
    } else {
        for (size_t i = 0; i < off.size(); i++) off[i] = offsets[i];
    }
    if (off[0] != 0) return fail(FMM_ERR_INVALID, "fmm_build_batch: offsets[0] must be 0");
    for (int i = 0; i < n_sys; i++)
        if (off[i + 1] <= off[i]) return fail(FMM_ERR_INVALID, "fmm_build_batch: every system needs >= 1 particle");
    int64_t N = off[n_sys];
    if (N >= ((int64_t)1 << 31) - 1) return fail(FMM_ERR_CAPACITY, "fmm_build_batch: total N must be < 2^31 - 1");
    return build_common(c, x, m, N, leaf_size, off);
}

int fmm_forces(fmm_ctx* c, int p, double theta, int variant, double* acc, double* pot) {
    if (!c) return fail(FMM_ERR_INVALID, "fmm_forces: NULL context");
    if (!c->built) return fail(FMM_ERR_STATE, "fmm_forces: call fmm_build first");
    if (p < 1 || p > FMM_P_MAX) return fail(FMM_ERR_INVALID, "fmm_forces: p must be in [1, FMM_P_MAX]");
    if (!(theta >= 0.0 && theta < 1.0)) return fail(FMM_ERR_INVALID, "fmm_forces: theta must be in [0, 1)");
    if (c->precision == FMM_DF64 && p > FMM_DF64_P_MAX)
        return fail(FMM_ERR_INVALID, "fmm_forces: FMM_DF64 supports p <= FMM_DF64_P_MAX");
    if (c->precision == FMM_MIXED && p > FMM_MIXED_P_MAX)
        return fail(FMM_ERR_INVALID, "fmm_forces: FMM_MIXED supports p <= FMM_MIXED_P_MAX");
    if (variant != FMM_STANDARD && variant != FMM_CONSERVING && variant != FMM_CONSERVING_PAPER0)
        return fail(FMM_ERR_INVALID, "fmm_forces: unknown variant");
    if (variant == FMM_CONSERVING_PAPER0 && p != 1)
        return fail(FMM_ERR_INVALID, "fmm_forces: FMM_CONSERVING_PAPER0 needs p = 1");
    if (!acc) return fail(FMM_ERR_INVALID, "fmm_forces: acc is required");
    if (c->schedule == FMM_SCHEDULE_FUSED &&
        (c->precision != FMM_FP64 || p > 6 || variant == FMM_CONSERVING_PAPER0))
        return fail(FMM_ERR_INVALID, "fmm_forces: the fused schedule runs FMM_FP64, p <= 6, standard or conserving");
    // the literal order-0 form reads the second moments (eq. aaB0): expansion order 2
    if (variant == FMM_CONSERVING_PAPER0) p = 2;
    return guarded(c, [&]() -> int {
        for (int s = ST_MOMENTS; s < ST_COUNT; s++) c->stage_valid[s] = false;
        bool want_pot = pot != nullptr;
        size_t n = (size_t)c->N;
        bool fused = c->schedule == FMM_SCHEDULE_FUSED;
        bool need_mom = c->mom_p != p, need_walk = !fused && c->list_theta != theta;
        auto moments = [&]() {
            stage_begin(c, ST_MOMENTS);
            run_moments_dispatch(c, p);
            stage_end(c, ST_MOMENTS);
        };
        auto walk = [&]() {
            stage_begin(c, ST_WALK);
            run_walk(c, theta);
            stage_end(c, ST_WALK);
        };
        if (need_mom && need_walk && (c->overlap & FMM_OVERLAP_MOMENTS_WALK)) {
            // the moments (build -> P2M -> M2M) do not depend on the walk, and neither on
            // the other: the moments run on the side stream while the walk (with its host
            // reads of list sizes) runs on the context's stream
            c->mom_p = -1;
            fork_side(c);
            {
                SideLaunches side(c);
                moments();
            }
            walk();
            join_side(c);
            c->mom_p = p;
        } else {
            if (need_mom) {
                moments();
                c->mom_p = p;
            }
            if (need_walk) walk();
        }
        if (fused) {
            // no walk and no lists: every target node traverses for its own pairs
            c->list_theta = -1.0;
            c->fused_theta = theta;
            GB_CUDA(cudaMemsetAsync(c->errflag.as<int>() + 2, 0, sizeof(int), c->stream));
            run_far_field_dispatch(c, p, variant, want_pot);
            stage_begin(c, ST_P2P);
            run_p2p_fused(c, want_pot, theta);
            stage_end(c, ST_P2P);
        } else if (c->overlap & FMM_OVERLAP_NEAR_FAR) {
            // near field (pair kernels) beside the far field (M2L, L2L): independent until
            // the per-particle sums; the set-up (with its host read of the partial count,
            // once per walk) runs first on the context's stream
            run_p2p_prepare(c);
            fork_side(c);
            {
                SideLaunches side(c);
                run_p2p_kernels(c, want_pot);
            }
            run_far_field_dispatch(c, p, variant, want_pot);
            join_side(c);
        } else {
            run_far_field_dispatch(c, p, variant, want_pot);
            run_p2p(c, want_pot);
        }
        ensure(c->acc_s, sizeof(double) * 3 * n);
        ensure(c->pot_s, sizeof(double) * n);
        bool acc_dev = is_device_ptr(acc);
        bool pot_dev = want_pot && is_device_ptr(pot);
        ensure(c->out_stage, sizeof(double) * 4 * n);
        double* acc_d = acc_dev ? acc : c->out_stage.as<double>();
        double* pot_d = want_pot ? (pot_dev ? pot : c->out_stage.as<double>() + 3 * n) : nullptr;
        stage_begin(c, ST_L2P);
        if (!fused) run_p2p_gather(c);
        run_finish_dispatch(c, p, variant, want_pot, acc_d, pot_d);
        stage_end(c, ST_L2P);
        if (fused) {  // a traversal stack that would have overflowed (none is expected)
            HostReads hr(c);
            int* over = hr.read<int>(c->errflag.as<int>() + 2);
            hr.wait();
            if (*over) throw FmmError{FMM_ERR_CAPACITY, "fused schedule: traversal stack exceeded"};
        }
        if (!acc_dev)
            GB_CUDA(cudaMemcpyAsync(acc, acc_d, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
        if (want_pot && !pot_dev)
            GB_CUDA(cudaMemcpyAsync(pot, pot_d, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
        if (!acc_dev || (want_pot && !pot_dev)) GB_CUDA(cudaStreamSynchronize(c->stream));
        c->have_forces = true;
        return FMM_OK;
    });
}

int fmm_forces_graph(fmm_ctx* c, int p, double theta, int variant, double* acc, double* pot) {
    if (!c) return fail(FMM_ERR_INVALID, "fmm_forces_graph: NULL context");
    if (!c->built) return fail(FMM_ERR_STATE, "fmm_forces_graph: call fmm_build first");
    if (!acc || !is_device_ptr(acc) || (pot && !is_device_ptr(pot)))
        return fail(FMM_ERR_INVALID, "fmm_forces_graph: acc (and pot) must be device memory");
    if (c->schedule != FMM_SCHEDULE_LISTS)
        return fail(FMM_ERR_INVALID, "fmm_forces_graph: needs the list schedule");
    // the recording assumes the moments, lists and buffers it was made on: a direct
    // fmm_forces that formed none of them anew leaves it valid
    bool same = c->graph_exec && c->graph_p == p && c->graph_theta == theta && c->graph_variant == variant &&
                c->graph_acc == acc && c->graph_pot == pot && c->graph_op_gen == c->op_gen &&
                c->graph_walk_gen == c->walk_gen && c->graph_mom_p == c->mom_p &&
                c->graph_reallocs == realloc_count();
    if (!same) {
        if (c->graph_exec) {
            cudaGraphExecDestroy(c->graph_exec);
            c->graph_exec = nullptr;
        }
        // one direct evaluation forms the moments and lists and sizes every buffer; the
        // next one then has no host read and no allocation, and is recorded
        int rc = fmm_forces(c, p, theta, variant, acc, pot);
        if (rc != FMM_OK) return rc;
        long long before = realloc_count();
        rc = guarded(c, [&]() -> int {
            GB_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            return FMM_OK;
        });
        if (rc != FMM_OK) return rc;
        c->capturing = true;  // no stage timer events inside the recording
        rc = fmm_forces(c, p, theta, variant, acc, pot);
        c->capturing = false;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (rc == FMM_OK && (e != cudaSuccess || realloc_count() != before)) {
            cudaGetLastError();
            rc = fail(FMM_ERR_CUDA, "fmm_forces_graph: the evaluation could not be recorded");
        }
        if (rc == FMM_OK && cudaGraphInstantiate(&c->graph_exec, g, 0) != cudaSuccess) {
            cudaGetLastError();
            c->graph_exec = nullptr;
            rc = fail(FMM_ERR_CUDA, "fmm_forces_graph: graph instantiation failed");
        }
        if (g) cudaGraphDestroy(g);
        if (rc != FMM_OK) return rc;
        c->graph_p = p;
        c->graph_theta = theta;
        c->graph_variant = variant;
        c->graph_acc = acc;
        c->graph_pot = pot;
        c->graph_op_gen = c->op_gen;
        c->graph_walk_gen = c->walk_gen;
        c->graph_mom_p = c->mom_p;
        c->graph_reallocs = realloc_count();
    }
    return guarded(c, [&]() -> int {
        GB_CUDA(cudaGraphLaunch(c->graph_exec, c->stream));
        for (int s = 0; s < ST_COUNT; s++) c->stage_valid[s] = false;  // the replay times no stage
        c->have_forces = true;
        return FMM_OK;
    });
}

int fmm_forces_batch(fmm_ctx* c, int p, double theta, int variant, double* acc, double* pot, double* diag) {
    int rc = fmm_forces(c, p, theta, variant, acc, pot);
    if (rc != FMM_OK || !diag) return rc;
    return guarded(c, [&]() -> int {
        ensure(c->sys_diag, sizeof(double) * 6 * (size_t)c->n_sys);
        run_diagnostics_sys(c, c->sys_diag.as<double>());
        GB_CUDA(cudaMemcpyAsync(diag, c->sys_diag.p, sizeof(double) * 6 * (size_t)c->n_sys, cudaMemcpyDefault,
                                c->stream));
        GB_CUDA(cudaStreamSynchronize(c->stream));
        return FMM_OK;
    });
}

int fmm_diagnostics(fmm_ctx* c, double sum_ma[3], double sum_mxa[3]) {
    if (!c) return fail(FMM_ERR_INVALID, "fmm_diagnostics: NULL context");
    if (!c->have_forces) return fail(FMM_ERR_STATE, "fmm_diagnostics: call fmm_forces first");
    return guarded(c, [&]() -> int {
        double out[6];
        run_diagnostics(c, out);
        if (sum_ma)
            for (int d = 0; d < 3; d++) sum_ma[d] = out[d];
        if (sum_mxa)
            for (int d = 0; d < 3; d++) sum_mxa[d] = out[3 + d];
        return FMM_OK;
    });
}

int fmm_counts(fmm_ctx* c, int64_t* n_nodes, int64_t* n_m2l, int64_t* n_p2p, int32_t* n_levels) {
    if (!c) return fail(FMM_ERR_INVALID, "fmm_counts: NULL context");
    if (!c->built) return fail(FMM_ERR_STATE, "fmm_counts: call fmm_build first");
    if (n_nodes) *n_nodes = c->n_nodes;
    if (n_m2l) *n_m2l = c->list_theta >= 0 ? c->n_m2l : 0;
    if (n_p2p) *n_p2p = c->list_theta >= 0 ? c->n_p2p : 0;
    if (n_levels) *n_levels = c->n_levels;
    return FMM_OK;
}

// copy n elements of device array src to dst (host or device)
static void copy_out(fmm_ctx* c, void* dst, const void* src, size_t bytes) {
    if (!dst || bytes == 0) return;
    GB_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
}

int fmm_get_keys(fmm_ctx* c, uint64_t* keys_sorted, int64_t* perm, double* lo, double* side) {
    if (!c) return fail(FMM_ERR_INVALID, "fmm_get_keys: NULL context");
    if (!c->built) return fail(FMM_ERR_STATE, "fmm_get_keys: call fmm_build first");
    return guarded(c, [&]() -> int {
        size_t n = (size_t)c->N;
        copy_out(c, keys_sorted, c->keys0.p, sizeof(uint64_t) * n);
        std::vector<uint32_t> p32(perm ? n : 0);
        if (perm) copy_out(c, p32.data(), c->perm.p, sizeof(uint32_t) * n);
        double g[5];
        copy_out(c, g, c->geom.p, sizeof(double) * 5);
        GB_CUDA(cudaStreamSynchronize(c->stream));
        if (perm) {
            if (is_device_ptr(perm)) {
                std::vector<int64_t> p64(p32.begin(), p32.end());
                GB_CUDA(cudaMemcpy(perm, p64.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice));
            } else {
                for (size_t i = 0; i < n; i++) perm[i] = p32[i];
            }
        }
        if (lo) copy_out(c, lo, c->geom.p, sizeof(double) * 3);
        if (side) copy_out(c, side, c->geom.as<double>() + 3, sizeof(double));
        GB_CUDA(cudaStreamSynchronize(c->stream));
        return FMM_OK;
    });
}

int fmm_get_tree(fmm_ctx* c, int32_t* first, int32_t* count, int32_t* level, int32_t* parent, int32_t* child_first,
                 int32_t* nchild) {
    if (!c) return fail(FMM_ERR_INVALID, "fmm_get_tree: NULL context");
    if (!c->built) return fail(FMM_ERR_STATE, "fmm_get_tree: call fmm_build first");
    return guarded(c, [&]() -> int {
        size_t b = sizeof(int32_t) * (size_t)c->n_nodes;
        copy_out(c, first, c->nfirst.p, b);
        copy_out(c, count, c->ncount.p, b);
        copy_out(c, level, c->nlevel.p, b);
        copy_out(c, parent, c->nparent.p, b);
        copy_out(c, child_first, c->nchildf.p, b);
        copy_out(c, nchild, c->nnchild.p, b);
        GB_CUDA(cudaStreamSynchronize(c->stream));
        return FMM_OK;
    });
}

int fmm_get_geometry(fmm_ctx* c, double* M, double* Z, double* rmax) {
    if (!c) return fail(FMM_ERR_INVALID, "fmm_get_geometry: NULL context");
    if (!c->built) return fail(FMM_ERR_STATE, "fmm_get_geometry: call fmm_build first");
    return guarded(c, [&]() -> int {
        size_t nn = (size_t)c->n_nodes;
        copy_out(c, M, c->nM.p, sizeof(double) * nn);
        copy_out(c, rmax, c->nrmax.p, sizeof(double) * nn);
        if (Z) {
            std::vector<double> zx(nn), zy(nn), zz(nn), zall(3 * nn);
            copy_out(c, zx.data(), c->nZx.p, sizeof(double) * nn);
            copy_out(c, zy.data(), c->nZy.p, sizeof(double) * nn);
            copy_out(c, zz.data(), c->nZz.p, sizeof(double) * nn);
            GB_CUDA(cudaStreamSynchronize(c->stream));
            for (size_t i = 0; i < nn; i++) {
                zall[3 * i] = zx[i];
                zall[3 * i + 1] = zy[i];
                zall[3 * i + 2] = zz[i];
            }
            GB_CUDA(cudaMemcpy(Z, zall.data(), sizeof(double) * 3 * nn, cudaMemcpyDefault));
        }
        GB_CUDA(cudaStreamSynchronize(c->stream));
        return FMM_OK;
    });
}

int fmm_get_lists(fmm_ctx* c, int32_t* m2l, int32_t* p2p) {
    if (!c) return fail(FMM_ERR_INVALID, "fmm_get_lists: NULL context");
    if (c->list_theta < 0) return fail(FMM_ERR_STATE, "fmm_get_lists: call fmm_forces first");
    return guarded(c, [&]() -> int {
        size_t nn = (size_t)c->n_nodes;
        // the canonical list: for every target in increasing id, its partners above it
        // (at or above it for P2P, whose self pairs have one entry) in increasing id
        if (m2l && c->n_m2l > 0) {
            std::vector<long long> seg(nn + 1);
            std::vector<uint32_t> src(2 * (size_t)c->n_m2l);
            copy_out(c, seg.data(), c->m2l_seg.p, sizeof(long long) * seg.size());
            copy_out(c, src.data(), c->m2l_dir.p, sizeof(uint32_t) * src.size());
            GB_CUDA(cudaStreamSynchronize(c->stream));
            std::vector<int32_t> out;
            out.reserve(2 * (size_t)c->n_m2l);
            std::vector<int32_t> part;
            for (size_t t = 0; t < nn; t++) {
                part.clear();
                for (long long e = seg[t]; e < seg[t + 1]; e++)
                    if ((int64_t)src[e] > (int64_t)t) part.push_back((int32_t)src[e]);
                std::sort(part.begin(), part.end());
                for (int32_t q : part) {
                    out.push_back((int32_t)t);
                    out.push_back(q);
                }
            }
            GB_CUDA(cudaMemcpy(m2l, out.data(), sizeof(int32_t) * out.size(), cudaMemcpyDefault));
        }
        if (p2p && c->n_p2p > 0) {
            std::vector<long long> seg(nn + 1);
            std::vector<int2> pairs((size_t)c->n_p2p);
            copy_out(c, seg.data(), c->p2p_seg.p, sizeof(long long) * seg.size());
            GB_CUDA(cudaStreamSynchronize(c->stream));
            std::vector<uint32_t> val((size_t)seg[nn]);
            copy_out(c, val.data(), c->p2p_dval.p, sizeof(uint32_t) * val.size());
            copy_out(c, pairs.data(), c->p2p_pairs.p, sizeof(int2) * pairs.size());
            GB_CUDA(cudaStreamSynchronize(c->stream));
            std::vector<int32_t> out;
            out.reserve(2 * (size_t)c->n_p2p);
            std::vector<int32_t> part;
            for (size_t t = 0; t < nn; t++) {
                part.clear();
                for (long long e = seg[t]; e < seg[t + 1]; e++) {
                    int2 pr = pairs[val[e] >> 1];
                    int32_t partner = (val[e] & 1u) ? pr.x : pr.y;
                    if ((int64_t)partner >= (int64_t)t) part.push_back(partner);
                }
                std::sort(part.begin(), part.end());
                for (int32_t q : part) {
                    out.push_back((int32_t)t);
                    out.push_back(q);
                }
            }
            GB_CUDA(cudaMemcpy(p2p, out.data(), sizeof(int32_t) * out.size(), cudaMemcpyDefault));
        }
        return FMM_OK;
    });
}

int fmm_set_walk_capacity(fmm_ctx* c, int64_t frontier, int64_t m2l, int64_t p2p) {
    if (!c) return fail(FMM_ERR_INVALID, "fmm_set_walk_capacity: NULL context");
    c->op_gen++;
    if (frontier < 1 || m2l < 1 || p2p < 1) return fail(FMM_ERR_INVALID, "fmm_set_walk_capacity: sizes must be >= 1");
    c->cap_fr = frontier;
    c->cap_m2l = m2l;
    c->cap_p2p = p2p;
    c->caps_user = true;
    c->list_theta = -1.0;
    return FMM_OK;
}

int fmm_set_tiles(fmm_ctx* c, int m2l_chunk, int p2p_chunk) {
    if (!c) return fail(FMM_ERR_INVALID, "fmm_set_tiles: NULL context");
    c->op_gen++;
    if (m2l_chunk < 1 || m2l_chunk > 4096 || p2p_chunk < 1 || p2p_chunk > 4096)
        return fail(FMM_ERR_INVALID, "fmm_set_tiles: chunk lengths must be in [1, 4096]");
    if (c->m2l_chunk != m2l_chunk || c->p2p_chunk != p2p_chunk) c->list_theta = -1.0;
    c->m2l_chunk = m2l_chunk;
    c->p2p_chunk = p2p_chunk;
    return FMM_OK;
}

int fmm_autotune(fmm_ctx* c, const double* x, const double* m, int64_t N, const int64_t* offsets, int n_sys,
                 int p, double theta, int variant, const int* leaf_sizes, int n_leaf, const int* m2l_chunks,
                 int n_chunk, int reps, int* best_leaf, int* best_chunk, double* best_ms) {
    if (!c || !x || !m || !leaf_sizes || !m2l_chunks || !best_leaf || !best_chunk || !best_ms)
        return fail(FMM_ERR_INVALID, "fmm_autotune: NULL argument");
    if (n_leaf < 1 || n_chunk < 1 || reps < 1 || N < 1) return fail(FMM_ERR_INVALID, "fmm_autotune: empty search");
    for (int i = 0; i < n_leaf; i++)
        if (leaf_sizes[i] < 1) return fail(FMM_ERR_INVALID, "fmm_autotune: leaf sizes must be >= 1");
    int keep_p2p = c->p2p_chunk;
    double best = -1.0;
    int bl = leaf_sizes[0], bc = m2l_chunks[0];
    auto build = [&](int leaf) {
        return offsets ? fmm_build_batch(c, x, m, offsets, n_sys, leaf) : fmm_build(c, x, m, N, leaf);
    };
    for (int a = 0; a < n_leaf; a++) {
        for (int b = 0; b < n_chunk; b++) {
            int rc = fmm_set_tiles(c, m2l_chunks[b], keep_p2p);
            if (rc != FMM_OK) return rc;
            double* acc = nullptr;
            rc = guarded(c, [&]() -> int {
                ensure(c->tune_acc, sizeof(double) * 3 * (size_t)N);
                acc = c->tune_acc.as<double>();
                return FMM_OK;
            });
            if (rc != FMM_OK) return rc;
            // one untimed evaluation sizes every buffer, then reps timed ones
            rc = build(leaf_sizes[a]);
            if (rc == FMM_OK) rc = fmm_forces(c, p, theta, variant, acc, nullptr);
            if (rc != FMM_OK) return rc;
            float ms = 0.f;
            rc = guarded(c, [&]() -> int {
                cudaEvent_t e0, e1;
                GB_CUDA(cudaEventCreate(&e0));
                GB_CUDA(cudaEventCreate(&e1));
                GB_CUDA(cudaEventRecord(e0, c->stream));
                int r = FMM_OK;
                for (int k = 0; k < reps && r == FMM_OK; k++) {
                    r = build(leaf_sizes[a]);
                    if (r == FMM_OK) r = fmm_forces(c, p, theta, variant, acc, nullptr);
                }
                GB_CUDA(cudaEventRecord(e1, c->stream));
                GB_CUDA(cudaEventSynchronize(e1));
                GB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return r;
            });
            if (rc != FMM_OK) return rc;
            double t = (double)ms / reps;
            if (best < 0.0 || t < best) {
                best = t;
                bl = leaf_sizes[a];
                bc = m2l_chunks[b];
            }
        }
    }
    // leave the context built with the winner
    int rc = fmm_set_tiles(c, bc, keep_p2p);
    if (rc == FMM_OK) rc = build(bl);
    if (rc != FMM_OK) return rc;
    *best_leaf = bl;
    *best_chunk = bc;
    *best_ms = best;
    return FMM_OK;
}

int fmm_walk_retries(fmm_ctx* c, int64_t* retries) {
    if (!c || !retries) return fail(FMM_ERR_INVALID, "fmm_walk_retries: NULL argument");
    *retries = c->walk_retries;
    return FMM_OK;
}

int fmm_set_schedule(fmm_ctx* c, int schedule) {
    if (!c) return fail(FMM_ERR_INVALID, "fmm_set_schedule: NULL context");
    c->op_gen++;
    if (schedule != FMM_SCHEDULE_LISTS && schedule != FMM_SCHEDULE_FUSED)
        return fail(FMM_ERR_INVALID, "fmm_set_schedule: unknown schedule");
    c->schedule = schedule;
    c->list_theta = -1.0;
    return FMM_OK;
}

int fmm_set_overlap(fmm_ctx* c, int mask) {
    if (!c) return fail(FMM_ERR_INVALID, "fmm_set_overlap: NULL context");
    if (mask & ~(FMM_OVERLAP_MOMENTS_WALK | FMM_OVERLAP_NEAR_FAR))
        return fail(FMM_ERR_INVALID, "fmm_set_overlap: unknown bits in the mask");
    c->op_gen++;
    c->overlap = mask;
    return FMM_OK;
}

int fmm_set_wait_limit(fmm_ctx* c, int64_t polls, int never_satisfied) {
    if (!c) return fail(FMM_ERR_INVALID, "fmm_set_wait_limit: NULL context");
    c->op_gen++;
    if (polls < 0) return fail(FMM_ERR_INVALID, "fmm_set_wait_limit: polls must be >= 0");
    c->walk_spin_limit = polls > 0 ? (long long)polls : gbfmm::WALK_SPIN_LIMIT;
    c->walk_wait_never = never_satisfied != 0;
    c->list_theta = -1.0;   // the next fmm_forces walks again under these limits
    return FMM_OK;
}

int fmm_stage_times(fmm_ctx* c, double* ms, int n) {
    if (!c || !ms) return fail(FMM_ERR_INVALID, "fmm_stage_times: NULL argument");
    return guarded(c, [&]() -> int {
        GB_CUDA(cudaStreamSynchronize(c->stream));
        for (int s = 0; s < n && s < ST_COUNT; s++) {
            ms[s] = -1.0;
            if (c->stage_valid[s]) {
                float t = 0.f;
                GB_CUDA(cudaEventElapsedTime(&t, c->ev[2 * s], c->ev[2 * s + 1]));
                ms[s] = t;
            }
        }
        return FMM_OK;
    });
}

}  // extern "C"
