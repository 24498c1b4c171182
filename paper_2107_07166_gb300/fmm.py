"""Python binding of the gbfmm C ABI (``include/gbfmm.h``): argument marshalling only.

Every step of the method runs in the CUDA library ``libgbfmm.so``; this module
converts numpy arrays / torch tensors (host or CUDA) into pointers and sizes and turns
status codes into exceptions.  It raises if the library is missing: there is no CPU
fallback.

    from paper_2107_07166_gb300 import fmm
    f = fmm.FMM(device=0)
    f.build(x, m, leaf_size=32)                # x: (N, 3) float64, m: (N,) float64
    f.forces(p=4, theta=0.6, variant=fmm.CONSERVING, acc=acc, pot=None)
    sum_ma, sum_mxa = f.diagnostics()
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbfmm.so")

STANDARD, CONSERVING, CONSERVING_PAPER0 = 0, 1, 2
FP64, MIXED, DF64 = 0, 1, 2
SCHEDULE_LISTS, SCHEDULE_FUSED = 0, 1
OVERLAP_MOMENTS_WALK, OVERLAP_NEAR_FAR = 1, 2
P_MAX = 8
MIXED_P_MAX = 6
DF64_P_MAX = 5
STAGES = ("build", "moments", "walk", "m2l", "l2l", "p2p", "l2p")
EXPORTS = ("fmm_create", "fmm_destroy", "fmm_set_stream", "fmm_build", "fmm_build_batch", "fmm_forces",
           "fmm_forces_graph", "fmm_forces_batch", "fmm_diagnostics",
           "fmm_counts", "fmm_get_keys", "fmm_get_tree", "fmm_get_geometry", "fmm_get_lists",
           "fmm_stage_times", "fmm_leapfrog", "fmm_set_walk_capacity", "fmm_set_tiles", "fmm_autotune",
           "fmm_walk_retries", "fmm_set_wait_limit", "fmm_set_schedule", "fmm_set_overlap", "fmm_probe_fma_rate", "fmm_morton_sort_noalloc", "fmm_kernel_launches", "fmm_strerror",
           "fmm_last_error")
NOALLOC_MAX_N = 131072

_lock = threading.Lock()
_lib = None


class FMMError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status}: {detail}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load libgbfmm.so (raises OSError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise OSError(f"gbfmm CUDA library not built: {path} (run __graft_entry__.build())")
        lib = C.CDLL(path)
        P, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
        sig = {
            "fmm_create": (i32, [C.POINTER(C.c_void_p), i32, i32, P]),
            "fmm_destroy": (i32, [P]),
            "fmm_set_stream": (i32, [P, P]),
            "fmm_build": (i32, [P, P, P, i64, i32]),
            "fmm_forces": (i32, [P, i32, dbl, i32, P, P]),
            "fmm_forces_graph": (i32, [P, i32, dbl, i32, P, P]),
            "fmm_build_batch": (i32, [P, P, P, P, i32, i32]),
            "fmm_forces_batch": (i32, [P, i32, dbl, i32, P, P, P]),
            "fmm_diagnostics": (i32, [P, P, P]),
            "fmm_counts": (i32, [P, P, P, P, P]),
            "fmm_get_keys": (i32, [P, P, P, P, P]),
            "fmm_get_tree": (i32, [P] * 7),
            "fmm_get_geometry": (i32, [P, P, P, P]),
            "fmm_get_lists": (i32, [P, P, P]),
            "fmm_stage_times": (i32, [P, P, i32]),
            "fmm_set_walk_capacity": (i32, [P, i64, i64, i64]),
            "fmm_set_tiles": (i32, [P, i32, i32]),
            "fmm_autotune": (i32, [P, P, P, i64, P, i32, i32, dbl, i32, P, i32, P, i32, i32, P, P, P]),
            "fmm_leapfrog": (i32, [P, P, P, P, i64, i32, i32, dbl, i32, dbl, i32, P]),
            "fmm_walk_retries": (i32, [P, P]),
            "fmm_set_wait_limit": (i32, [P, i64, i32]),
            "fmm_set_schedule": (i32, [P, i32]),
            "fmm_set_overlap": (i32, [P, i32]),
            "fmm_probe_fma_rate": (i32, [i32, i32, P]),
            "fmm_morton_sort_noalloc": (i32, [P, i64, P, P, P, P, P]),
            "fmm_kernel_launches": (i64, []),
            "fmm_strerror": (C.c_char_p, [i32]),
            "fmm_last_error": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def probe_fma_rate(device: int = 0, precision: int = FP64) -> float:
    """Measured FMA rate (TFLOP/s) of the binary64 (FP64) or binary32 (MIXED) units."""
    out = np.zeros(1)
    _check(load().fmm_probe_fma_rate(int(device), int(precision), _ptr(out)), "fmm_probe_fma_rate")
    return float(out[0])


def kernel_launches() -> int:
    """CUDA kernels launched by the library in this process so far."""
    return int(load().fmm_kernel_launches())


def _ptr(a, dtype=None):
    """Raw pointer of a numpy array or torch tensor (host or device), checked contiguous."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):      # torch.Tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None and str(a.dtype).replace("torch.", "") != np.dtype(dtype).name:
            raise TypeError(f"tensor dtype {a.dtype}, expected {np.dtype(dtype).name}")
        return C.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or not a.flags.c_contiguous:
        raise ValueError("expected a C-contiguous numpy array or torch tensor")
    if dtype is not None and a.dtype != np.dtype(dtype):
        raise TypeError(f"array dtype {a.dtype}, expected {np.dtype(dtype).name}")
    return a.ctypes.data_as(C.c_void_p)


def _check(rc: int, where: str):
    if rc != 0:
        lib = load()
        raise FMMError(rc, where, f"{lib.fmm_strerror(rc).decode()} ({lib.fmm_last_error().decode()})")


class FMM:
    """One gbfmm context (fmm_create ... fmm_destroy)."""

    def __init__(self, device: int = 0, precision: int = FP64, stream=None):
        self.lib = load()
        h = C.c_void_p()
        _check(self.lib.fmm_create(C.byref(h), int(device), int(precision), self._stream_ptr(stream)),
               "fmm_create")
        self.h = h
        self.N = 0

    @staticmethod
    def _stream_ptr(stream):
        """None -> private library stream; a torch stream or raw handle otherwise.  The
        legacy default stream (handle 0) is passed as cudaStreamLegacy (1), because a NULL
        handle asks the library for a private stream."""
        if stream is None:
            return None
        h = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        return C.c_void_p(h if h != 0 else 1)

    def close(self):
        if getattr(self, "h", None):
            self.lib.fmm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream):
        _check(self.lib.fmm_set_stream(self.h, self._stream_ptr(stream)), "fmm_set_stream")

    def build(self, x, m, leaf_size: int):
        n = int(x.shape[0])
        if tuple(x.shape) != (n, 3) or tuple(m.shape) != (n,):
            raise ValueError("x must be (N, 3) and m (N,)")
        _check(self.lib.fmm_build(self.h, _ptr(x, np.float64), _ptr(m, np.float64), n, int(leaf_size)),
               "fmm_build")
        self.N = n

    def build_batch(self, x, m, offsets, leaf_size: int):
        """Independent systems concatenated in x, m; offsets (n_sys + 1,) int64."""
        off = np.ascontiguousarray(offsets, dtype=np.int64) if not hasattr(offsets, "data_ptr") else offsets
        n = int(x.shape[0])
        if tuple(x.shape) != (n, 3) or tuple(m.shape) != (n,):
            raise ValueError("x must be (N, 3) and m (N,)")
        _check(self.lib.fmm_build_batch(self.h, _ptr(x, np.float64), _ptr(m, np.float64), _ptr(off, np.int64),
                                        int(off.shape[0]) - 1, int(leaf_size)), "fmm_build_batch")
        self.N = n
        self.n_sys = int(off.shape[0]) - 1

    def forces_batch(self, p: int, theta: float, variant: int, acc, pot=None):
        """Forces of every system; returns the (n_sys, 6) per-system [sum m a, sum m X x a]."""
        diag = np.zeros((self.n_sys, 6))
        _check(self.lib.fmm_forces_batch(self.h, int(p), float(theta), int(variant), _ptr(acc, np.float64),
                                         _ptr(pot, np.float64), _ptr(diag)), "fmm_forces_batch")
        return diag

    def forces(self, p: int, theta: float, variant: int, acc, pot=None):
        if self.N and (tuple(acc.shape) != (self.N, 3) or (pot is not None and tuple(pot.shape) != (self.N,))):
            raise ValueError("acc must be (N, 3) and pot (N,)")
        _check(self.lib.fmm_forces(self.h, int(p), float(theta), int(variant), _ptr(acc, np.float64),
                                   _ptr(pot, np.float64)), "fmm_forces")

    def forces_graph(self, p: int, theta: float, variant: int, acc, pot=None):
        """fmm_forces replayed as one recorded CUDA graph (device outputs only)."""
        if self.N and (tuple(acc.shape) != (self.N, 3) or (pot is not None and tuple(pot.shape) != (self.N,))):
            raise ValueError("acc must be (N, 3) and pot (N,)")
        _check(self.lib.fmm_forces_graph(self.h, int(p), float(theta), int(variant), _ptr(acc, np.float64),
                                         _ptr(pot, np.float64)), "fmm_forces_graph")

    def diagnostics(self):
        f = np.zeros(3)
        t = np.zeros(3)
        _check(self.lib.fmm_diagnostics(self.h, _ptr(f), _ptr(t)), "fmm_diagnostics")
        return f, t

    def counts(self):
        nn, nm, npp = (np.zeros(1, np.int64) for _ in range(3))
        nl = np.zeros(1, np.int32)
        _check(self.lib.fmm_counts(self.h, _ptr(nn), _ptr(nm), _ptr(npp), _ptr(nl)), "fmm_counts")
        return dict(n_nodes=int(nn[0]), n_m2l=int(nm[0]), n_p2p=int(npp[0]), n_levels=int(nl[0]))

    def get_keys(self):
        keys = np.zeros(self.N, np.uint64)
        perm = np.zeros(self.N, np.int64)
        lo = np.zeros(3)
        side = np.zeros(1)
        _check(self.lib.fmm_get_keys(self.h, _ptr(keys), _ptr(perm), _ptr(lo), _ptr(side)), "fmm_get_keys")
        return keys, perm, lo, float(side[0])

    def get_tree(self):
        nn = self.counts()["n_nodes"]
        names = ("first", "count", "level", "parent", "child_first", "nchild")
        t = {k: np.zeros(nn, np.int32) for k in names}
        _check(self.lib.fmm_get_tree(self.h, *[_ptr(t[k]) for k in names]), "fmm_get_tree")
        return t

    def get_geometry(self):
        nn = self.counts()["n_nodes"]
        M = np.zeros(nn)
        Z = np.zeros((nn, 3))
        r = np.zeros(nn)
        _check(self.lib.fmm_get_geometry(self.h, _ptr(M), _ptr(Z), _ptr(r)), "fmm_get_geometry")
        return M, Z, r

    def get_lists(self):
        c = self.counts()
        m2l = np.zeros((c["n_m2l"], 2), np.int32)
        p2p = np.zeros((c["n_p2p"], 2), np.int32)
        _check(self.lib.fmm_get_lists(self.h, _ptr(m2l), _ptr(p2p)), "fmm_get_lists")
        return m2l, p2p

    def leapfrog(self, x, v, m, leaf_size: int, p: int, theta: float, variant: int, dt: float, nsteps: int,
                 diag=None):
        """nsteps kick-drift-kick steps; x and v (N x 3) are advanced in place.  Returns the
        (nsteps + 1) x 6 momenta [sum m v, sum m x x v] as numpy if diag is None."""
        n = int(x.shape[0])
        out = np.zeros((nsteps + 1, 6)) if diag is None else diag
        _check(self.lib.fmm_leapfrog(self.h, _ptr(x, np.float64), _ptr(v, np.float64), _ptr(m, np.float64), n,
                                     int(leaf_size), int(p), float(theta), int(variant), float(dt), int(nsteps),
                                     _ptr(out, np.float64)), "fmm_leapfrog")
        self.N = n
        return out

    def set_walk_capacity(self, frontier: int, m2l: int, p2p: int):
        _check(self.lib.fmm_set_walk_capacity(self.h, int(frontier), int(m2l), int(p2p)), "fmm_set_walk_capacity")

    def set_tiles(self, m2l_chunk: int, p2p_chunk: int = 64):
        _check(self.lib.fmm_set_tiles(self.h, int(m2l_chunk), int(p2p_chunk)), "fmm_set_tiles")

    def autotune(self, x, m, p: int, theta: float, variant: int, leaf_sizes=(16, 24, 32, 48, 64),
                 m2l_chunks=(16, 32, 64), offsets=None, reps: int = 3):
        """Fastest (leaf size, M2L chunk) for build + forces on this input; the context is
        left built with it.  Returns (leaf_size, m2l_chunk, ms per evaluation)."""
        n = int(x.shape[0])
        leaves = np.ascontiguousarray(leaf_sizes, dtype=np.int32)
        chunks = np.ascontiguousarray(m2l_chunks, dtype=np.int32)
        off = None if offsets is None else np.ascontiguousarray(offsets, dtype=np.int64)
        bl, bc = np.zeros(1, np.int32), np.zeros(1, np.int32)
        ms = np.zeros(1)
        _check(self.lib.fmm_autotune(self.h, _ptr(x, np.float64), _ptr(m, np.float64), n, _ptr(off, np.int64),
                                     0 if off is None else int(off.shape[0]) - 1, int(p), float(theta), int(variant),
                                     _ptr(leaves), int(leaves.shape[0]), _ptr(chunks), int(chunks.shape[0]),
                                     int(reps), _ptr(bl), _ptr(bc), _ptr(ms)), "fmm_autotune")
        self.N = n
        if off is not None:
            self.n_sys = int(off.shape[0]) - 1
        return int(bl[0]), int(bc[0]), float(ms[0])

    def walk_retries(self) -> int:
        r = np.zeros(1, np.int64)
        _check(self.lib.fmm_walk_retries(self.h, _ptr(r)), "fmm_walk_retries")
        return int(r[0])

    def set_schedule(self, schedule: int):
        """SCHEDULE_LISTS (default) or SCHEDULE_FUSED (no interaction lists; binary64)."""
        _check(self.lib.fmm_set_schedule(self.h, int(schedule)), "fmm_set_schedule")

    def set_overlap(self, mask: int):
        """Mask of OVERLAP_MOMENTS_WALK (default) and OVERLAP_NEAR_FAR: independent stages of
        fmm_forces run on a second stream."""
        _check(self.lib.fmm_set_overlap(self.h, int(mask)), "fmm_set_overlap")

    def set_wait_limit(self, polls: int = 0, never_satisfied: bool = False):
        """Limit of the walk's look-back wait (0: default); never_satisfied for tests of the
        FMM_ERR_TIMEOUT path."""
        _check(self.lib.fmm_set_wait_limit(self.h, int(polls), int(bool(never_satisfied))), "fmm_set_wait_limit")

    def stage_times(self):
        ms = np.zeros(len(STAGES))
        _check(self.lib.fmm_stage_times(self.h, _ptr(ms), len(STAGES)), "fmm_stage_times")
        return dict(zip(STAGES, ms.tolist()))
