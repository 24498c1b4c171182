/*
 * gbfmm.h -- C ABI of the GB300 (sm_103a) symmetric Cartesian fast multipole method
 * for Newtonian gravity, standard and angular-momentum-conserving, after
 * Korobkin et al., "Conservation of Angular Momentum in the Fast Multipole Method"
 * (arXiv:2107.07166).
 *
 * Problem (Sec. 2, eq. jia): N particles at X_a with masses m_a; compute for every a
 *   acceleration a_a = -sum_{b != a} m_b (X_a - X_b) / |X_a - X_b|^3   (G = 1, no softening)
 *   potential   phi_a = -sum_{b != a} m_b / |X_a - X_b|
 * with the FMM of Sec. 2: an octree of nodes with centre of mass Z and radius r_max,
 * multipoles up to order p about Z, mutual cell-cell interactions for pairs passing the
 * acceptance test (r_A,max + r_B,max) / R <= theta (eq. mac_criterion, theta = tan of the
 * MAC angle), and exact particle-particle sums for the rest.  Coincident particles
 * (r = 0) exert nothing on each other.
 *
 * Order p is the multipole/potential order of Sec. 2.1 ("expansion up to 4-th order" is
 * p = 4); the paper's "zeroth order FMM" of Sec. 3.1 is p = 1.
 *
 * Conventions for every call:
 *   - return 0 (FMM_OK) or a negative FMM_ERR_* code; fmm_strerror() names it and
 *     fmm_last_error() gives the detail of the last failure on this thread;
 *   - on error no output buffer is written;
 *   - every array argument may be host memory or device memory of the context's
 *     device (detected with cudaPointerGetAttributes); the caller owns all arrays;
 *     inputs are copied, outputs are written in the caller's particle order;
 *   - work is queued on the context's stream; calls that return results on the host
 *     synchronise that stream first;
 *   - a context is not thread-safe.
 */
#ifndef GBFMM_H
#define GBFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_ctx fmm_ctx;

#if defined(__GNUC__)
#define GBFMM_API __attribute__((visibility("default")))
#else
#define GBFMM_API
#endif

/* highest multipole order compiled into the library (binary64), and into its FMM_MIXED
 * and FMM_DF64 modes */
#define FMM_P_MAX 8
#define FMM_MIXED_P_MAX 6
#define FMM_DF64_P_MAX 5

/* variants */
enum {
    FMM_STANDARD = 0,   /* Sec. 2: symmetric Taylor expansion (eq. taylor), forces a = -grad phi */
    FMM_CONSERVING = 1, /* Sec. 3.2: every approximated pair force realigned onto the line X_a - Y_b */
    FMM_CONSERVING_PAPER0 = 2 /* Sec. 3.2, eqs. realign2 and aaB0, p = 1 only: zeroth-order magnitude
                                 times the first-order expanded unit vector, summed into monopole,
                                 x_perp, (n.x) x and second-moment terms (moments carried to order 2) */
};

/* arithmetic of the pair kernels (M2L and P2P); tree, moments, translations (M2M, L2L),
 * L2P, accumulators and diagnostics are binary64 in every mode */
enum {
    FMM_FP64 = 0,  /* M2L and P2P in IEEE binary64; the P2P's r^-3 is refined in binary64 from a
                      binary32 seed (within 2 ulp, as a library reciprocal square root and cube) */
    FMM_MIXED = 1, /* M2L and P2P in binary32 (separations formed in double-float first),
                      per-pair and per-chunk partials summed in binary64 */
    FMM_DF64 = 2   /* M2L and P2P in double-float arithmetic on the binary32 units (two binary32
                      words, ~48-bit significand): binary64-level results at the binary32 issue rate */
};

/* schedules of the interaction stage (fmm_set_schedule) */
enum {
    FMM_SCHEDULE_LISTS = 0, /* the mutual walk stores its M2L and P2P pairs once, sorted by target, and
                               the pair kernels evaluate them (each P2P pair force formed once) */
    FMM_SCHEDULE_FUSED = 1  /* no lists: every target node walks the same recursion restricted to its
                               own pairs and evaluates them as it finds them (binary64 only) */
};

/* stages of fmm_forces that may run concurrently (fmm_set_overlap, a bit mask) */
enum {
    FMM_OVERLAP_MOMENTS_WALK = 1, /* P2M/M2M beside the dual-tree walk (the default) */
    FMM_OVERLAP_NEAR_FAR = 2      /* the P2P pair kernels beside M2L and L2L */
};

/* status codes */
enum {
    FMM_OK = 0,
    FMM_ERR_INVALID = -1,  /* bad argument: N < 1, leaf_size < 1, p not in [1,FMM_P_MAX], theta not in [0,1),
                              unknown variant, non-finite x or m, m < 0, NULL required pointer */
    FMM_ERR_STATE = -2,    /* call out of order (forces before build, diagnostics before forces) */
    FMM_ERR_CUDA = -3,     /* a CUDA runtime call failed */
    FMM_ERR_OOM = -4,      /* device allocation failed */
    FMM_ERR_CAPACITY = -5, /* an internal size limit was exceeded (N >= 2^31, > 2^31 list entries) */
    FMM_ERR_TIMEOUT = -6   /* a bounded device wait ran out (the walk's ordered output claims) */
};

/* Create a context on CUDA device `device` with arithmetic `precision` (FMM_FP64,
 * FMM_MIXED or FMM_DF64).
 * `cuda_stream` is the cudaStream_t to queue work on (cudaStreamLegacy and
 * cudaStreamPerThread are accepted), or NULL for a private non-blocking stream.  Device
 * outputs are complete once that stream has reached the end of the call's work. */
GBFMM_API int fmm_create(fmm_ctx **out, int device, int precision, void *cuda_stream);

/* Release the context and all device memory it holds.  NULL is accepted. */
GBFMM_API int fmm_destroy(fmm_ctx *c);

/* Re-target the context's work to another stream of the same device (NULL: private). */
GBFMM_API int fmm_set_stream(fmm_ctx *c, void *cuda_stream);

/* Build the tree (Sec. 2: nodes with COM Z and r_max, eq. mac_criterion).
 *   x: N x 3 row-major positions (float64); m: N masses (float64, >= 0, finite).
 *   leaf_size: a node with more than leaf_size particles is split into its non-empty
 *   octants, down to level 21 at most.
 * Steps: bounding cube, 63-bit Morton keys, stable radix sort, breadth-first octree,
 * centres of mass and exact r_max.  Invalidates previous moments, lists and forces. */
GBFMM_API int fmm_build(fmm_ctx *c, const double *x, const double *m, int64_t N, int leaf_size);

/* Build a batch of independent systems in one context (no force acts between systems).
 *   x: N x 3, m: N with the systems concatenated; offsets: n_sys + 1 entries (host or
 *   device), system s = particles [offsets[s], offsets[s+1]), offsets[0] = 0, every
 *   system non-empty, N = offsets[n_sys].
 * Every system gets its own bounding cube, keys and octree, exactly as fmm_build would
 * give it alone; the trees form one forest (system s owns root node s) and every later
 * stage processes all systems in the same launches.  fmm_get_keys reports the cube of
 * system 0. */
GBFMM_API int fmm_build_batch(fmm_ctx *c, const double *x, const double *m, const int64_t *offsets, int n_sys,
                              int leaf_size);

/* One force evaluation on the last built tree.
 *   p in [1,FMM_P_MAX]: multipole order (Sec. 2.1); theta in [0,1): acceptance parameter
 *   (eq. mac_criterion); variant: FMM_STANDARD, FMM_CONSERVING, or FMM_CONSERVING_PAPER0
 *   (which needs p = 1, else FMM_ERR_INVALID).
 *   acc: N x 3 row-major output accelerations (required).
 *   pot: N output potentials, or NULL to skip them.  For FMM_CONSERVING the potential
 *   is the standard order-p potential (a realigned force field has no potential); for
 *   FMM_CONSERVING_PAPER0 it is the standard order-2 potential of the moments it carries.
 * Steps: P2M/M2M (cached per p), dual-tree walk (cached per theta), M2L, L2L, L2P,
 * mutual P2P, deterministic reductions (no floating-point atomics).  Stages that do not
 * depend on each other may run concurrently on a second stream of the context
 * (fmm_set_overlap), forked from and joined back into the context's stream, so all work
 * of the call is ordered on that stream; the results do not depend on it (bitwise). */
GBFMM_API int fmm_forces(fmm_ctx *c, int p, double theta, int variant, double *acc, double *pot);

/* fmm_forces recorded once as a CUDA graph and replayed: the same evaluation (every
 * stage from M2L to the outputs, on the moments and lists of the last build and walk)
 * as one graph launch on the context's stream, with no host read.
 *   Arguments as fmm_forces; acc and pot (or NULL) must be device memory, and the context
 *   must use the list schedule (FMM_SCHEDULE_LISTS), else FMM_ERR_INVALID.
 *   The first call, and any call after a change of arguments, of the tree (fmm_build*),
 *   of a setting (fmm_set_*), after a direct fmm_forces that formed moments or lists anew
 *   (another p or theta), or after any device buffer of the library was allocated or
 *   freed, runs fmm_forces once (moments, walk, buffer sizes), then records a second
 *   evaluation and launches it; other calls only launch.
 *   Results are bitwise those of fmm_forces.  The replay does not synchronise the stream
 *   and times no stage (fmm_stage_times reports -1 after it).  FMM_ERR_CUDA if the
 *   evaluation could not be recorded. */
GBFMM_API int fmm_forces_graph(fmm_ctx *c, int p, double theta, int variant, double *acc, double *pot);

/* fmm_forces for a batch, plus per-system diagnostics: diag (n_sys x 6, host or device, or
 * NULL) receives [sum m a, sum m X x a] of every system, summed in a fixed order. */
GBFMM_API int fmm_forces_batch(fmm_ctx *c, int p, double theta, int variant, double *acc, double *pot,
                               double *diag);

/* Kick-drift-kick leapfrog with this context's forces, for momentum-drift runs.
 *   x, v: N x 3 row-major positions and velocities (host or device), advanced in place;
 *   m: N masses.  Every step: v += a dt/2, x += v dt, rebuild (leaf_size), forces
 *   (p, theta, variant), v += a dt/2.  All state stays on the device between steps.
 *   diag: (nsteps + 1) x 6 doubles (host or device, or NULL): total linear momentum
 *   sum m v and angular momentum sum m x x v before the first step and after each step,
 *   summed in a fixed order.  Leaves the context built on the final positions. */
GBFMM_API int fmm_leapfrog(fmm_ctx *c, double *x, double *v, const double *m, int64_t N, int leaf_size, int p,
                           double theta, int variant, double dt, int nsteps, double *diag);

/* Diagnostics of the last fmm_forces (eqs. netforce, total_torque), float64,
 * summed in a fixed order:  sum_ma = sum_a m_a acc_a,  sum_mxa = sum_a m_a X_a x acc_a. */
GBFMM_API int fmm_diagnostics(fmm_ctx *c, double sum_ma[3], double sum_mxa[3]);

/* Sizes of the last build/walk: nodes, mutual M2L pairs, P2P pairs (self pairs included),
 * number of tree levels.  Any pointer may be NULL. */
GBFMM_API int fmm_counts(fmm_ctx *c, int64_t *n_nodes, int64_t *n_m2l, int64_t *n_p2p, int32_t *n_levels);

/* Parity exports (copies into caller buffers of the sizes given by fmm_counts). */
/* keys_sorted[N]: Morton keys in sorted order; perm[N]: input index of each sorted particle;
 * lo[3], side[1]: the bounding cube (either may be NULL). */
GBFMM_API int fmm_get_keys(fmm_ctx *c, uint64_t *keys_sorted, int64_t *perm, double *lo, double *side);
/* breadth-first node arrays, n_nodes each: first sorted particle, particle count, level,
 * parent (-1 for the root), first child (-1 for leaves), number of children */
GBFMM_API int fmm_get_tree(fmm_ctx *c, int32_t *first, int32_t *count, int32_t *level, int32_t *parent,
                 int32_t *child_first, int32_t *nchild);
/* node mass M[n], centre of mass Z[n x 3], radius rmax[n] */
GBFMM_API int fmm_get_geometry(fmm_ctx *c, double *M, double *Z, double *rmax);
/* canonical lists of the last walk: pairs (min id, max id) in lexicographic order,
 * m2l[n_m2l x 2], p2p[n_p2p x 2] (self pairs (A, A) included) */
GBFMM_API int fmm_get_lists(fmm_ctx *c, int32_t *m2l, int32_t *p2p);

/* Initial sizes (entries) of the dual-tree walk's buffers: frontier, M2L pairs, P2P pairs.
 * Without this call they start at 4N, 16N and 4N.  A walk that outgrows a buffer is run
 * again with larger buffers (see fmm_walk_retries); the results do not depend on the
 * sizes.  Invalidates cached lists. */
GBFMM_API int fmm_set_walk_capacity(fmm_ctx *c, int64_t frontier, int64_t m2l, int64_t p2p);
/* Tile shapes: directed M2L entries per M2L work item (default 32; 64 in FMM_MIXED) and
 * directed P2P entries per reduction item (default 64), each in [1, 4096].  Results change
 * only in summation order.  Invalidates cached lists. */
GBFMM_API int fmm_set_tiles(fmm_ctx *c, int m2l_chunk, int p2p_chunk);

/* Autotuner: times build + forces (p, theta, variant, no potentials) on the given input
 * for every leaf size in leaf_sizes[n_leaf] and M2L chunk length in m2l_chunks[n_chunk]
 * (one untimed evaluation, then reps timed ones, CUDA events on the context's stream) and
 * returns the fastest pair in *best_leaf, *best_chunk with its time per evaluation in
 * *best_ms.  x, m (N particles) and offsets (n_sys + 1 entries, or NULL for one system,
 * as in fmm_build_batch) may be host or device memory.  The context is left built with
 * the winning leaf size and tiles.  Errors of the trial builds or evaluations are
 * returned as they occur. */
GBFMM_API int fmm_autotune(fmm_ctx *c, const double *x, const double *m, int64_t N, const int64_t *offsets,
                           int n_sys, int p, double theta, int variant, const int *leaf_sizes, int n_leaf,
                           const int *m2l_chunks, int n_chunk, int reps, int *best_leaf, int *best_chunk,
                           double *best_ms);

/* Number of walks this context has re-run after a buffer overflow. */
GBFMM_API int fmm_walk_retries(fmm_ctx *c, int64_t *retries);

/* Schedule of the interactions of later fmm_forces calls (FMM_SCHEDULE_LISTS, the default,
 * or FMM_SCHEDULE_FUSED).  Both evaluate exactly the pairs of the mutual walk of Sec. 2
 * (eq. mac_criterion); results differ only in summation order.  The fused schedule keeps no
 * interaction list: every target node runs the walk's recursion restricted to the pairs
 * that contain one of its ancestors, evaluates its M2L sources and P2P partners as it finds
 * them and writes each result once (no list sort, no partial buffers, no gather).  It forms
 * every particle-pair force from both sides, so it does about 1.5x the binary64 P2P work of
 * the list schedule.  It runs in FMM_FP64 for p <= 6 and the FMM_STANDARD and FMM_CONSERVING
 * variants; other combinations return FMM_ERR_INVALID from fmm_forces.  fmm_get_lists needs
 * the list schedule.  Invalidates cached lists. */
GBFMM_API int fmm_set_schedule(fmm_ctx *c, int schedule);

/* Which independent stages of later fmm_forces calls run concurrently: a mask of
 * FMM_OVERLAP_MOMENTS_WALK (the moments on a second stream while the walk runs on the
 * context's stream) and FMM_OVERLAP_NEAR_FAR (the P2P pair kernels on the second stream
 * while M2L and L2L run; the list schedule only).  The default is FMM_OVERLAP_MOMENTS_WALK.
 * Measured on one GB300: the moments beside the walk take 0.8-3% off an evaluation; the
 * near field beside the far field takes another 3% off in FMM_MIXED, whose pair kernels
 * are latency-bound, and adds 3% in FMM_FP64, whose pair kernels both keep the binary64
 * units busy.  Results are bitwise the same for every mask.  FMM_ERR_INVALID for other
 * bits.  The paper has no counterpart: this is a scheduling setting. */
GBFMM_API int fmm_set_overlap(fmm_ctx *c, int mask);

/* Limit of the walk's only device-side wait, for tests of its failure path.  Each walk
 * step places its outputs after those of the tiles before it (eq. mac_criterion decides
 * the pairs; the order of the lists is fixed by the tree), so a tile polls a status word
 * of its predecessors; after `polls` polls (0: the default, about 4 million, far beyond
 * any correct run) it gives up, the remaining steps do nothing, and fmm_forces returns
 * FMM_ERR_TIMEOUT with no output written.  never_satisfied != 0 makes every such wait
 * look for a status that no tile publishes, so the limit is reached whenever a step has
 * more than one tile of 1024 frontier pairs.  The context stays usable; the next
 * fmm_forces walks again.  Invalidates cached lists. */
GBFMM_API int fmm_set_wait_limit(fmm_ctx *c, int64_t polls, int never_satisfied);

/* Device time in milliseconds of each stage of the last build/forces call, measured
 * with CUDA events on the stream each stage ran on: [build, moments, walk, m2l, l2l, p2p,
 * l2p].  Stages that ran concurrently (fmm_set_overlap) overlap in time, so the stage
 * times of one call can add up to more than its duration.  A stage that did not run in
 * that call reports -1. */
GBFMM_API int fmm_stage_times(fmm_ctx *c, double *ms, int n);

/* Largest N accepted by fmm_morton_sort_noalloc. */
#define FMM_NOALLOC_MAX_N 131072

/* Bounding cube, Morton keys and stable sort of fmm_build, for callers that cannot
 * allocate device memory.  The paper has no counterpart: this is a service entry point.
 *
 * Who needs it: hosts that hand out all device memory from their own pool or budget it
 * up front, and code that must not call cudaMalloc/cudaFree because those calls can
 * synchronise the whole device.  The call allocates nothing: its scratch is one fixed
 * array of about 2.2 MiB in the library's device image, which every GPU that loads the
 * library holds until the process exits.
 *
 *   x: N x 3 row-major positions, device memory of the current device (or managed
 *   memory); 1 <= N <= FMM_NOALLOC_MAX_N.
 *   keys_sorted[N] (device): the 63-bit Morton keys in stable sorted order.
 *   perm[N] (device): input index of each sorted particle.
 *   lo[3], side[1] (device, either may be NULL): the bounding cube.
 *   cuda_stream: stream to queue the work on (NULL: the legacy default stream).
 * The call synchronises that stream before it returns: it reads back a flag that says
 * whether every coordinate was finite.  Only that stream is waited for, not the device.
 * Results equal those of fmm_build followed by fmm_get_keys on the same positions.
 * Returns FMM_ERR_CAPACITY for N above the maximum; FMM_ERR_INVALID for NULL arrays,
 * host arrays, arrays of another device, N < 1, or a non-finite coordinate (outputs are
 * then unspecified); FMM_ERR_CUDA with the failing step in fmm_last_error().
 * The first call on each device looks up the scratch array's address there; make that
 * first call before any stream capture.  All calls share the one array, so calls whose
 * GPU work overlaps (different streams or threads) race: serialise them. */
GBFMM_API int fmm_morton_sort_noalloc(const double *x, int64_t N, uint64_t *keys_sorted, int64_t *perm,
                                      double *lo, double *side, void *cuda_stream);

/* Measured fused multiply-add rate of device `device` in TFLOP/s (an FMA counted as two
 * flops): binary64 for precision FMM_FP64, binary32 for FMM_MIXED.  A kernel of eight
 * independent FMA chains per thread, four blocks of 256 threads per SM, timed with CUDA
 * events (best of three after a warm-up run, about 20 ms each).  The paper has no
 * counterpart: this is the measured peak against which the ALU-bound pair kernels (M2L,
 * P2P) are rated.  Synchronises the device's work on a private stream; allocates 16 bytes. */
GBFMM_API int fmm_probe_fma_rate(int device, int precision, double *tflops);

/* Number of CUDA kernels this library has launched in this process so far (all contexts). */
GBFMM_API int64_t fmm_kernel_launches(void);

GBFMM_API const char *fmm_strerror(int status);
GBFMM_API const char *fmm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GBFMM_H */
