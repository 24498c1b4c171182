"""FP64 CPU oracle of the symmetric Cartesian FMM (standard and angular-momentum
conserving forms of arXiv:2107.07166).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package smoke check and by
the CPU-baseline leg of ``bench.py``.  The CUDA library never imports, links or
calls it, and it shares no code with the CUDA path.  The arithmetic lives in
``fmm_oracle.c`` (plain C, single thread, compiled with ``-ffp-contract=off``); this
module only compiles it and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

STANDARD, CONSERVING, CONSERVING_PAPER0 = 0, 1, 2


def expansion_order(p: int, variant: int) -> int:
    """Order of the moments (and standard locals) a run carries: p, except for the
    literal order-0 realigned form, which needs the second moments of eq. aaB0."""
    return 2 if variant == CONSERVING_PAPER0 else p


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (gcc, -O2, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P = C.c_void_p
        i64, i32, dbl = C.c_int64, C.c_int, C.c_double
        lib.orc_run.restype = P
        lib.orc_run.argtypes = [P, P, i64, i32, i32, dbl, i32, i32]
        lib.orc_free.argtypes = [P]
        for f in ("orc_n_nodes", "orc_n_m2l", "orc_n_p2p", "orc_n_trace"):
            getattr(lib, f).restype = i64
            getattr(lib, f).argtypes = [P]
        lib.orc_get_keys.argtypes = [P, P, P, P, P]
        lib.orc_get_tree.argtypes = [P] * 7
        lib.orc_get_geometry.argtypes = [P] * 4
        lib.orc_get_moments.argtypes = [P, P]
        lib.orc_get_locals.argtypes = [P, P, P]
        lib.orc_get_locals.restype = i32
        lib.orc_get_lists.argtypes = [P, P, P]
        lib.orc_set_trace.argtypes = [i32]
        lib.orc_counts.argtypes = [P, P, i64, i32, dbl, P]
        lib.orc_stage_seconds.argtypes = [P, P]
        lib.orc_get_trace.argtypes = [P, P]
        lib.orc_get_result.argtypes = [P, P, P]
        lib.orc_nmi.argtypes = [i32]
        lib.orc_nmi.restype = i32
        lib.orc_multi_index.argtypes = [i32, P]
        lib.orc_dtensor.argtypes = [i32, P, P]
        lib.orc_htensor.argtypes = [i32, P, P]
        lib.orc_bbox.argtypes = [P, i64, P, P]
        lib.orc_keys.argtypes = [P, i64, P, dbl, P]
        lib.orc_sort.argtypes = [P, i64, P, P]
        lib.orc_direct.argtypes = [P, P, i64, P, P]
        lib.orc_direct_targets.argtypes = [P, P, i64, P, i64, P, P]
        lib.orc_pair_taylor.argtypes = [i32, i32, P, P, i64, P, P, P, i64, P, P]
        lib.orc_cell_pair.argtypes = [i32, i32, P, P, i64, P, P, P, i64, P, P]
        lib.orc_p2m.argtypes = [i32, P, P, P, i64, P]
        lib.orc_m2m.argtypes = [i32, P, P, P, P]
        lib.orc_l2l.argtypes = [i32, P, P, P]
        _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def nmi(p: int) -> int:
    """Number of multi-indices with |alpha| <= p."""
    return int(_load().orc_nmi(p))


def multi_indices(p: int) -> np.ndarray:
    """Multi-index table (nmi(p) x 3) in the oracle's order."""
    lib = _load()
    out = np.zeros((nmi(p), 3), dtype=np.int32)
    a = np.zeros(3, dtype=np.int32)
    for k in range(nmi(p)):
        lib.orc_multi_index(k, _p(a))
        out[k] = a
    return out


def dtensor(p: int, R) -> np.ndarray:
    """D_alpha = d^alpha(-1/r) at R for |alpha| <= p."""
    R = _f64(R, (3,))
    out = np.zeros(nmi(p))
    _load().orc_dtensor(p, _p(R), _p(out))
    return out


def htensor(p: int, R) -> np.ndarray:
    """h_alpha = d^alpha(-|r|^-3) at R for |alpha| <= p."""
    R = _f64(R, (3,))
    out = np.zeros(nmi(p))
    _load().orc_htensor(p, _p(R), _p(out))
    return out


def bbox(x):
    x = _f64(x, (-1, 3))
    lo = np.zeros(3)
    side = np.zeros(1)
    _load().orc_bbox(_p(x), x.shape[0], _p(lo), _p(side))
    return lo, float(side[0])


def keys(x, lo, side):
    x = _f64(x, (-1, 3))
    lo = _f64(lo, (3,))
    out = np.zeros(x.shape[0], dtype=np.uint64)
    _load().orc_keys(_p(x), x.shape[0], _p(lo), float(side), _p(out))
    return out


def sort(k):
    k = np.ascontiguousarray(k, dtype=np.uint64)
    sk = np.zeros_like(k)
    perm = np.zeros(k.shape[0], dtype=np.int64)
    _load().orc_sort(_p(k), k.shape[0], _p(sk), _p(perm))
    return sk, perm


def direct(x, m, want_pot=True):
    """O(N^2) direct sum: accelerations (N x 3) and potentials (N)."""
    x = _f64(x, (-1, 3))
    m = _f64(m)
    N = x.shape[0]
    acc = np.zeros((N, 3))
    pot = np.zeros(N) if want_pot else None
    _load().orc_direct(_p(x), _p(m), N, _p(acc), _p(pot))
    return acc, pot


def direct_targets(x, m, targets):
    x = _f64(x, (-1, 3))
    m = _f64(m)
    t = np.ascontiguousarray(targets, dtype=np.int64)
    acc = np.zeros((t.shape[0], 3))
    pot = np.zeros(t.shape[0])
    _load().orc_direct_targets(_p(x), _p(m), x.shape[0], _p(t), t.shape[0], _p(acc), _p(pot))
    return acc, pot


def pair_taylor(p, variant, ZA, XA, ZB, YB, mB):
    """Per-pair truncated Taylor accelerations/potentials of cluster B on cluster A."""
    ZA, ZB = _f64(ZA, (3,)), _f64(ZB, (3,))
    XA, YB, mB = _f64(XA, (-1, 3)), _f64(YB, (-1, 3)), _f64(mB)
    acc = np.zeros((XA.shape[0], 3))
    pot = np.zeros(XA.shape[0])
    _load().orc_pair_taylor(p, variant, _p(ZA), _p(XA), XA.shape[0], _p(ZB), _p(YB), _p(mB), YB.shape[0],
                            _p(acc), _p(pot))
    return acc, pot


def cell_pair(p, variant, ZA, XA, ZB, YB, mB):
    """Cluster B on cluster A through P2M -> M2L -> L2P (one mutual cell pair, one side)."""
    ZA, ZB = _f64(ZA, (3,)), _f64(ZB, (3,))
    XA, YB, mB = _f64(XA, (-1, 3)), _f64(YB, (-1, 3)), _f64(mB)
    acc = np.zeros((XA.shape[0], 3))
    pot = np.zeros(XA.shape[0])
    _load().orc_cell_pair(p, variant, _p(ZA), _p(XA), XA.shape[0], _p(ZB), _p(YB), _p(mB), YB.shape[0],
                          _p(acc), _p(pot))
    return acc, pot


def p2m(p, Z, Y, m):
    Z, Y, m = _f64(Z, (3,)), _f64(Y, (-1, 3)), _f64(m)
    out = np.zeros(nmi(p))
    _load().orc_p2m(p, _p(Z), _p(Y), _p(m), Y.shape[0], _p(out))
    return out


def m2m(p, Zc, Zp, Mc):
    Zc, Zp, Mc = _f64(Zc, (3,)), _f64(Zp, (3,)), _f64(Mc)
    out = np.zeros(nmi(p))
    _load().orc_m2m(p, _p(Zc), _p(Zp), _p(Mc), _p(out))
    return out


def l2l(p, s, Lp):
    s, Lp = _f64(s, (3,)), _f64(Lp)
    out = np.zeros(nmi(p))
    _load().orc_l2l(p, _p(s), _p(Lp), _p(out))
    return out


def counts(x, m, leaf_size, theta):
    """Walk counts without expansions: (nodes, mutual M2L pairs, P2P pairs, particle pairs)."""
    x = _f64(x, (-1, 3))
    m = _f64(m)
    out = np.zeros(4, dtype=np.int64)
    _load().orc_counts(_p(x), _p(m), x.shape[0], int(leaf_size), float(theta), _p(out))
    return tuple(int(v) for v in out)


class Result:
    """Everything one oracle evaluation produced (numpy copies)."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


# decisions of the walk trace
WALK_SELF_SPLIT, WALK_M2L, WALK_P2P, WALK_SPLIT_A, WALK_SPLIT_B = 0, 1, 2, 3, 4


def run(x, m, leaf_size, p, theta, variant=STANDARD, want_pot=True, want_internals=True,
        want_trace=False) -> Result:
    """One full FMM evaluation (steps a1..a13): returns accelerations and potentials in
    input order plus, if requested, keys, permutation, tree, geometry, moments, lists and locals.
    want_trace adds ``trace``: every pair the walk visited, in visiting order, as rows
    (A, B, decision) with the WALK_* decisions above."""
    lib = _load()
    x = _f64(x, (-1, 3))
    m = _f64(m)
    N = x.shape[0]
    with _lock:
        lib.orc_set_trace(int(bool(want_trace)))
        h = lib.orc_run(_p(x), _p(m), N, int(leaf_size), int(p), float(theta), int(variant), int(bool(want_pot)))
        lib.orc_set_trace(0)
    if not h:
        raise ValueError("oracle rejected the arguments")
    try:
        nn, nm2l, np2p = lib.orc_n_nodes(h), lib.orc_n_m2l(h), lib.orc_n_p2p(h)
        acc = np.zeros((N, 3))
        pot = np.zeros(N) if want_pot else None
        lib.orc_get_result(h, _p(acc), _p(pot))
        st = np.zeros(6)
        lib.orc_stage_seconds(h, _p(st))
        r = Result(acc=acc, pot=pot, n_nodes=nn, n_m2l=nm2l, n_p2p=np2p,
                   stage_seconds=dict(zip(("tree", "moments", "walk", "m2l", "l2l_l2p", "p2p"), st.tolist())))
        if want_trace:
            tr = np.zeros((lib.orc_n_trace(h), 3), dtype=np.int32)
            lib.orc_get_trace(h, _p(tr))
            r.trace = tr
        if want_internals:
            keys_s = np.zeros(N, dtype=np.uint64)
            perm = np.zeros(N, dtype=np.int64)
            lo = np.zeros(3)
            side = np.zeros(1)
            lib.orc_get_keys(h, _p(keys_s), _p(perm), _p(lo), _p(side))
            tree = {k: np.zeros(nn, dtype=np.int32)
                    for k in ("first", "count", "level", "parent", "child_first", "nchild")}
            lib.orc_get_tree(h, *[_p(tree[k]) for k in
                                  ("first", "count", "level", "parent", "child_first", "nchild")])
            M = np.zeros(nn)
            Z = np.zeros((nn, 3))
            rmax = np.zeros(nn)
            lib.orc_get_geometry(h, _p(M), _p(Z), _p(rmax))
            pe = expansion_order(p, variant)
            mom = np.zeros((nn, nmi(pe)))
            lib.orc_get_moments(h, _p(mom))
            m2l = np.zeros((nm2l, 2), dtype=np.int32)
            p2p = np.zeros((np2p, 2), dtype=np.int32)
            lib.orc_get_lists(h, _p(m2l), _p(p2p))
            L = np.zeros((nn, nmi(pe)))
            SU = np.zeros((nn, 4 * nmi(pe - 1)))
            got = lib.orc_get_locals(h, _p(L), _p(SU))
            r.__dict__.update(keys=keys_s, perm=perm, lo=lo, side=float(side[0]), tree=tree, M=M, Z=Z,
                              rmax=rmax, moments=mom, m2l=m2l, p2p=p2p,
                              L=L if got & 1 else None, SU=SU if got & 2 else None)
        return r
    finally:
        lib.orc_free(h)
