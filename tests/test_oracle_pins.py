"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: the closed forms
printed in Sec. 2.1 (eqs. D..Dijkl, quad_mom, octo_mom, hexa_mom), finite
differences, harmonicity, exact polynomial identities, the O(N^2) direct sum
(eq. jia), the conservation statements of Sec. 2 (eq. netforce) and Sec. 3, and
closed-form Plummer/Hernquist energies."""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2107_07166_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def alpha_of(idx):
    a = [0, 0, 0]
    for i in idx:
        a[i] += 1
    return tuple(a)


def index_map(orc, p):
    mi = orc.multi_indices(p)
    return {tuple(int(v) for v in a): k for k, a in enumerate(mi)}


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


# ---------------------------------------------------------------- tensors

def test_dtensor_golden_R122(orc):
    """D..D_ijkl at R=(1,2,2) equal the paper's closed forms (exact rationals)."""
    im = index_map(orc, 4)
    D = orc.dtensor(4, [1.0, 2.0, 2.0])
    n = 0
    with open(os.path.join(GOLD, "dtensor_R122.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            idx, num, den = line.split()
            a = (0, 0, 0) if idx == "-" else alpha_of(int(c) for c in idx.split(","))
            want = float(Fraction(int(num), int(den)))
            assert D[im[a]] == pytest.approx(want, rel=1e-14, abs=1e-16), (idx, D[im[a]], want)
            n += 1
    assert n == 1 + 3 + 9 + 27 + 81


def _paper_D(R, idx):
    """Closed forms of Sec. 2.1 for orders <= 4 in floating point."""
    R = np.asarray(R, float)
    R2 = R @ R
    r = math.sqrt(R2)
    dl = lambda i, j: 1.0 if i == j else 0.0
    n = len(idx)
    if n == 0:
        return -1 / r
    if n == 1:
        return R[idx[0]] / r ** 3
    if n == 2:
        i, j = idx
        return (-3 * R[i] * R[j] + dl(i, j) * R2) / r ** 5
    if n == 3:
        i, j, k = idx
        return (15 * R[i] * R[j] * R[k] - 3 * R2 * (dl(i, j) * R[k] + dl(j, k) * R[i] + dl(i, k) * R[j])) / r ** 7
    i, j, k, l = idx
    t = -105 * R[i] * R[j] * R[k] * R[l]
    t += 15 * R2 * (dl(i, j) * R[k] * R[l] + dl(i, l) * R[j] * R[k] + dl(i, k) * R[j] * R[l]
                    + dl(j, l) * R[i] * R[k] + dl(j, k) * R[i] * R[l] + dl(l, k) * R[i] * R[j])
    t -= 3 * R2 * R2 * (dl(i, j) * dl(k, l) + dl(i, k) * dl(j, l) + dl(i, l) * dl(j, k))
    return t / r ** 9


@pytest.mark.parametrize("seed", range(5))
def test_dtensor_closed_forms_random(orc, seed):
    rng = np.random.default_rng(seed)
    R = rng.normal(size=3) * (0.3 + 3 * rng.random())
    im = index_map(orc, 4)
    D = orc.dtensor(4, R)
    for n in range(5):
        for idx in itertools.product(range(3), repeat=n):
            want = _paper_D(R, idx)
            got = D[im[alpha_of(idx)]]
            scale = np.linalg.norm(R) ** -(n + 1)
            assert abs(got - want) <= 1e-13 * scale, (idx, got, want)


@pytest.mark.parametrize("which", ["d", "h"])
def test_tensor_finite_differences(orc, which):
    """Order n+1 components equal central differences of order n components (n <= 7)."""
    rng = np.random.default_rng(11)
    R = np.array([0.7, -1.1, 0.4])
    f = orc.dtensor if which == "d" else orc.htensor
    im = index_map(orc, 8)
    T = f(8, R)
    h = 1e-5
    for a, k in im.items():
        if sum(a) >= 8:
            continue
        for i in range(3):
            e = np.zeros(3)
            e[i] = h
            fd = (f(8, R + e)[k] - f(8, R - e)[k]) / (2 * h)
            b = list(a)
            b[i] += 1
            exact = T[im[tuple(b)]]
            assert abs(fd - exact) <= 1e-6 * max(1.0, abs(exact)), (a, i, fd, exact)


def test_dtensor_traceless(orc):
    """1/r is harmonic: sum_i D_{alpha + 2 e_i} = 0 for every alpha."""
    R = np.array([0.3, 1.7, -0.9])
    im = index_map(orc, 8)
    D = orc.dtensor(8, R)
    for a, k in im.items():
        if sum(a) > 6:
            continue
        s = 0.0
        mag = 0.0
        for i in range(3):
            b = list(a)
            b[i] += 2
            s += D[im[tuple(b)]]
            mag += abs(D[im[tuple(b)]])
        assert abs(s) <= 1e-13 * mag


def test_htensor_low_orders(orc):
    """h = -r^-3: h_i = 3 R_i r^-5, h_ij = 3 d_ij r^-5 - 15 R_i R_j r^-7."""
    R = np.array([1.3, -0.2, 0.8])
    r = np.linalg.norm(R)
    im = index_map(orc, 2)
    H = orc.htensor(2, R)
    assert H[im[(0, 0, 0)]] == pytest.approx(-r ** -3, rel=1e-15)
    for i in range(3):
        a = [0, 0, 0]
        a[i] = 1
        assert H[im[tuple(a)]] == pytest.approx(3 * R[i] * r ** -5, rel=1e-14)
        for j in range(3):
            b = list(a)
            b[j] += 1
            want = 3 * (i == j) * r ** -5 - 15 * R[i] * R[j] * r ** -7
            assert H[im[tuple(b)]] == pytest.approx(want, rel=1e-13, abs=1e-15)


# ---------------------------------------------------------------- moments and shifts

def test_moments_match_paper_QHX(orc):
    """Raw moments reproduce the paper's traceless Q, H, X (eqs. quad_mom, octo_mom, hexa_mom)."""
    rng = np.random.default_rng(3)
    Y = rng.normal(size=(17, 3))
    m = rng.random(17)
    Z = (m[:, None] * Y).sum(0) / m.sum()
    im = index_map(orc, 4)
    Mr = orc.p2m(4, Z, Y, m)

    def raw(idx):     # sum_b m_b y^i y^j ... from M_alpha = sum m (-y)^alpha / alpha!
        a = alpha_of(idx)
        fac = math.factorial(a[0]) * math.factorial(a[1]) * math.factorial(a[2])
        return Mr[im[a]] * fac * (-1) ** len(idx)

    y = Y - Z
    q2 = (y * y).sum(1)
    dl = np.eye(3)
    assert Mr[im[(0, 0, 0)]] == pytest.approx(m.sum(), rel=1e-15)
    for i in range(3):            # dipole vanishes about the COM
        a = [0, 0, 0]
        a[i] = 1
        assert abs(Mr[im[tuple(a)]]) < 1e-14
    tr2 = sum(raw((l, l)) for l in range(3))
    for i, j in itertools.product(range(3), repeat=2):
        Q = (m * (3 * y[:, i] * y[:, j] - dl[i, j] * q2)).sum()
        assert 3 * raw((i, j)) - dl[i, j] * tr2 == pytest.approx(Q, rel=1e-12, abs=1e-13)
    for i, j, k in itertools.product(range(3), repeat=3):
        H = (m * (15 * y[:, i] * y[:, j] * y[:, k]
                  - 3 * q2 * (dl[i, j] * y[:, k] + dl[j, k] * y[:, i] + dl[i, k] * y[:, j]))).sum()
        tr = lambda u: sum(raw((l, l, u)) for l in range(3))
        got = 15 * raw((i, j, k)) - 3 * (dl[i, j] * tr(k) + dl[j, k] * tr(i) + dl[i, k] * tr(j))
        assert got == pytest.approx(H, rel=1e-12, abs=1e-12)
    for i, j, k, l in itertools.product(range(3), repeat=4):
        X = (m * (105 * y[:, i] * y[:, j] * y[:, k] * y[:, l]
                  - 15 * q2 * (dl[i, j] * y[:, k] * y[:, l] + dl[i, l] * y[:, j] * y[:, k]
                               + dl[i, k] * y[:, j] * y[:, l] + dl[j, l] * y[:, i] * y[:, k]
                               + dl[j, k] * y[:, i] * y[:, l] + dl[l, k] * y[:, i] * y[:, j])
                  + 3 * q2 * q2 * (dl[i, j] * dl[k, l] + dl[i, k] * dl[j, l] + dl[i, l] * dl[j, k]))).sum()
        t2 = lambda u, v: sum(raw((s, s, u, v)) for s in range(3))
        t4 = sum(raw((s, s, u, u)) for s in range(3) for u in range(3))
        got = (105 * raw((i, j, k, l))
               - 15 * (dl[i, j] * t2(k, l) + dl[i, l] * t2(j, k) + dl[i, k] * t2(j, l)
                       + dl[j, l] * t2(i, k) + dl[j, k] * t2(i, l) + dl[l, k] * t2(i, j))
               + 3 * t4 * (dl[i, j] * dl[k, l] + dl[i, k] * dl[j, l] + dl[i, l] * dl[j, k]))
        assert got == pytest.approx(X, rel=1e-11, abs=1e-11)


@pytest.mark.parametrize("p", [1, 2, 4, 6, 8])
def test_m2m_equals_direct_p2m(orc, p):
    """Shifting child moments to the parent centre equals P2M about the parent centre."""
    rng = np.random.default_rng(p)
    Y = rng.normal(size=(23, 3)) * 0.3
    m = rng.random(23)
    Zc = (m[:, None] * Y).sum(0) / m.sum()
    Zp = Zc + rng.normal(size=3) * 0.4
    shifted = orc.m2m(p, Zc, Zp, orc.p2m(p, Zc, Y, m))
    direct = orc.p2m(p, Zp, Y, m)
    assert np.allclose(shifted, direct, rtol=1e-12, atol=1e-13 * np.abs(direct).max())


@pytest.mark.parametrize("p", [2, 4, 7])
def test_l2l_is_polynomial_shift(orc, p):
    """The shifted local polynomial evaluated at x equals the original at x + s."""
    rng = np.random.default_rng(100 + p)
    n = orc.nmi(p)
    mi = orc.multi_indices(p)
    Lp = rng.normal(size=n)
    s = rng.normal(size=3) * 0.5
    Lc = orc.l2l(p, s, Lp)
    fact = np.array([math.factorial(a) * math.factorial(b) * math.factorial(c) for a, b, c in mi])
    ev = lambda L, x: (L * np.prod(x[None, :] ** mi, axis=1) / fact).sum()
    for _ in range(5):
        x = rng.normal(size=3) * 0.3
        assert ev(Lc, x) == pytest.approx(ev(Lp, x + s), rel=1e-12, abs=1e-12)
    back = orc.l2l(p, -s, Lc)
    assert np.allclose(back, Lp, rtol=1e-11, atol=1e-11)


# ---------------------------------------------------------------- M2L / L2P algebra

@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 6, 8])
def test_multipole_route_equals_pair_taylor(orc, p, variant):
    """P2M -> M2L -> L2P equals the per-pair truncated Taylor sum of eq. taylor
    (standard) or of the realigned pair force (conserving), to rounding."""
    rng = np.random.default_rng(7 * p + variant)
    XA = rng.normal(size=(9, 3)) * 0.25
    YB = rng.normal(size=(13, 3)) * 0.3 + np.array([2.5, -1.0, 0.7])
    mB = rng.random(13)
    ZA = XA.mean(0) + 0.05
    ZB = (mB[:, None] * YB).sum(0) / mB.sum()
    a1, p1 = orc.cell_pair(p, variant, ZA, XA, ZB, YB, mB)
    a2, p2 = orc.pair_taylor(p, variant, ZA, XA, ZB, YB, mB)
    assert rel(a1, a2) < 1e-13
    assert rel(p1, p2) < 1e-13


@pytest.mark.parametrize("variant", [0, 1])
def test_pair_taylor_converges_to_newton(orc, variant):
    """The truncated pair series converges to the exact force as p grows (|d|/R < 1)."""
    rng = np.random.default_rng(5)
    XA = rng.normal(size=(6, 3)) * 0.2
    YB = rng.normal(size=(6, 3)) * 0.2 + np.array([2.0, 0.0, 0.0])
    mB = rng.random(6)
    ZA, ZB = XA.mean(0), YB.mean(0)
    x = np.concatenate([XA, YB])
    mm = np.concatenate([np.zeros(6), mB])
    exact, _ = orc.direct(x, mm)
    errs = []
    for p in range(1, 9):
        a, _ = orc.pair_taylor(p, variant, ZA, XA, ZB, YB, mB)
        errs.append(rel(a, exact[:6]))
    # odd and even orders can tie (offsets nearly normal to R cancel odd terms), so
    # require a decrease over every two orders
    assert all(errs[i + 2] < errs[i] for i in range(len(errs) - 2)), errs
    assert errs[-1] < 1e-3 * errs[0]


def test_conserving_pair_force_is_central(orc):
    """Each realigned pair force is parallel to X_a - Y_b (eq. realign): single-particle B."""
    rng = np.random.default_rng(9)
    XA = rng.normal(size=(5, 3)) * 0.2
    YB = np.array([[2.1, 0.3, -0.4]])
    for p in (1, 2, 4, 8):
        a, _ = orc.pair_taylor(p, 1, XA.mean(0), XA, YB[0] + 0.05, YB, np.array([1.0]))
        d = XA - YB
        cr = np.cross(a, d)
        assert np.abs(cr).max() <= 1e-15 * np.abs(a).max() * np.abs(d).max() * 10


# ---------------------------------------------------------------- keys, sort, tree, walk

def _exact_quantised(x, lo, side):
    """q = min(floor((x - lo) 2^21 / side), 2^21 - 1) in exact rational arithmetic, and the
    distance of the exact t from the nearest integer (where the binary64 rounding of t
    may decide the floor, the pin does not apply)."""
    q = np.zeros(x.shape, dtype=np.int64)
    near = np.zeros(x.shape, dtype=bool)
    S = Fraction(side)
    for i in range(x.shape[0]):
        for d in range(3):
            t = (Fraction(float(x[i, d])) - Fraction(float(lo[d]))) * (1 << 21) / S
            f = math.floor(t)
            # t = 0 (the minimum, exact in binary64 too) and t near 2^21 (the largest
            # extent, clamped to the last cell either way) decide nothing
            near[i, d] = (min(t - f, f + 1 - t) < Fraction(1, 10 ** 8) and t != 0
                          and abs(t - (1 << 21)) > Fraction(1, 10 ** 8))
            q[i, d] = min(f, (1 << 21) - 1)
    return q, near


def _deinterleave(k):
    """(qx, qy, qz) of 63-bit keys: bit 3b + 2 = x bit b, 3b + 1 = y bit b, 3b = z bit b"""
    q = np.zeros((k.shape[0], 3), dtype=np.int64)
    ki = k.astype(np.int64)
    for b in range(21):
        for d in range(3):
            q[:, d] |= ((ki >> (3 * b + 2 - d)) & 1) << b
    return q


def test_keys_quantise_positions(orc):
    """Morton quantisation of the tree's cube (reading A12): the cube is the per-axis
    minimum and the largest extent, and every coordinate maps to exactly
    min(floor((x - lo) 2^21 / side), 2^21 - 1) -- the floor of the exact rational, not a
    rounding of it -- except within 1e-8 of a cell boundary, where binary64 rounding of t
    may decide (none of the drawn points lies there)."""
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(size=(300, 3)), rng.uniform(-3, 5, size=(200, 3))])
    lo, side = orc.bbox(x)
    assert np.array_equal(lo, x.min(0))
    assert side == (x.max(0) - x.min(0)).max()
    k = orc.keys(x, lo, side)
    assert np.all(k < 2 ** 63)
    q = _deinterleave(k)
    want, near = _exact_quantised(x, lo, side)
    assert near.sum() == 0
    assert np.array_equal(q, want)
    # the extreme points: the minimum maps to cell 0, the maximum of the longest axis to
    # the last cell (the clamp), and about half of all coordinates sit in the upper half
    # of their cell, where rounding instead of the floor would move them up by one
    ax = int(np.argmax(x.max(0) - x.min(0)))
    assert q[np.argmax(x[:, ax]), ax] == 2 ** 21 - 1
    assert np.all(q[np.argmin(x, axis=0), np.arange(3)] == 0)


def test_keys_quantise_cell_boundaries(orc):
    """Points placed exactly on and just inside cell boundaries of a dyadic cube (side 8,
    lo 0: one cell is 2^-18) quantise to the cell that starts there."""
    cell = 8.0 / 2 ** 21
    base = np.array([0.0, 1.0, 3.5, 7.25, 4.0 - cell, 8.0])
    x = np.stack([base, base[::-1], np.full(6, 2.0)], axis=1)
    x[0, 2] = 0.0
    x[1, 2] = 8.0
    lo, side = orc.bbox(x)
    assert np.array_equal(lo, [0.0, 0.0, 0.0]) and side == 8.0
    q = _deinterleave(orc.keys(x, lo, side))
    want = np.minimum(np.floor(x / cell).astype(np.int64), 2 ** 21 - 1)
    assert np.array_equal(q, want)
    assert q[4, 0] == 2 ** 20 - 1 and q[5, 0] == 2 ** 21 - 1 and q[2, 0] == 7 * 2 ** 17


def test_sort_is_stable(orc):
    rng = np.random.default_rng(2)
    k = rng.integers(0, 50, 500).astype(np.uint64)
    sk, perm = orc.sort(k)
    ref = np.argsort(k, kind="stable")
    assert np.array_equal(perm, ref)
    assert np.array_equal(sk, k[ref])


def check_tree(r, N, leaf):
    t = r.tree
    nn = r.n_nodes
    assert t["parent"][0] == -1 and t["first"][0] == 0 and t["count"][0] == N
    assert np.all(np.diff(t["level"]) >= 0)                        # breadth-first
    for n in range(nn):
        nc, c0 = t["nchild"][n], t["child_first"][n]
        if nc == 0:
            assert c0 == -1
            assert t["count"][n] <= leaf or t["level"][n] == 21
        else:
            assert t["count"][n] > leaf
            ch = np.arange(c0, c0 + nc)
            assert np.all(t["parent"][ch] == n)
            assert t["first"][ch[0]] == t["first"][n]
            assert np.all(t["first"][ch[1:]] == t["first"][ch[:-1]] + t["count"][ch[:-1]])
            assert t["count"][ch].sum() == t["count"][n]
            assert np.all(t["level"][ch] == t["level"][n] + 1)
    leaves = t["nchild"] == 0
    assert t["count"][leaves].sum() == N
    k = r.keys
    assert np.all(k[1:] >= k[:-1])
    # a node at level l is a key prefix of 3 l bits: its particles share it, and its
    # children are its non-empty octants at level l + 1, in increasing octant order
    for n in range(nn):
        f, c, lv = t["first"][n], t["count"][n], t["level"][n]
        assert c >= 1
        if lv > 0:
            s = np.uint64(63 - 3 * lv)
            assert k[f] >> s == k[f + c - 1] >> s
        if t["nchild"][n] > 0:
            ch = np.arange(t["child_first"][n], t["child_first"][n] + t["nchild"][n])
            dig = (k[t["first"][ch]] >> np.uint64(60 - 3 * lv)) & np.uint64(7)
            assert np.all(dig[1:] > dig[:-1])


@pytest.mark.parametrize("case", ["plummer", "coincident", "leaf1"])
def test_tree_is_the_octree_of_the_keys(orc, case):
    """The tree is the octree of the sorted keys: breadth-first, children the non-empty
    octants in Morton order, split while count > leaf below level 21."""
    rng = np.random.default_rng(8)
    if case == "plummer":
        x, m = synth.plummer(4000, 9)
        leaf = 16
    elif case == "coincident":
        x = np.concatenate([rng.normal(size=(400, 3)), np.repeat(rng.normal(size=(2, 3)), 30, axis=0)])
        m = rng.random(x.shape[0])
        leaf = 8
    else:
        x, m = synth.hernquist(600, 10)
        leaf = 1
    r = orc.run(x, m, leaf, 1, 0.5, 0, want_pot=False)
    check_tree(r, x.shape[0], leaf)
    if case == "coincident":
        deep = (r.tree["level"] == 21) & (r.tree["nchild"] == 0)
        assert np.any(r.tree["count"][deep] > leaf)


@pytest.mark.parametrize("variant", [0, 1])
def test_walk_covers_every_pair_once(orc, variant):
    x, m = synth.plummer(3000, 4)
    r = orc.run(x, m, 8, 3, 0.5, variant)
    check_tree(r, 3000, 8)
    c = r.tree["count"]
    m2l, p2p = r.m2l, r.p2p
    assert np.all(m2l[:, 0] < m2l[:, 1])
    assert np.all(p2p[:, 0] <= p2p[:, 1])
    for L in (m2l, p2p):
        key = L[:, 0].astype(np.int64) * 2 ** 32 + L[:, 1]
        assert np.all(np.diff(key) > 0)                               # canonical, unique
    leaf = r.tree["nchild"] == 0
    assert np.all(leaf[p2p[:, 0]]) and np.all(leaf[p2p[:, 1]])
    selfp = p2p[:, 0] == p2p[:, 1]
    total = (c[m2l[:, 0]].astype(np.int64) * c[m2l[:, 1]]).sum()
    total += np.where(selfp, c[p2p[:, 0]].astype(np.int64) * (c[p2p[:, 0]] - 1) // 2,
                      c[p2p[:, 0]].astype(np.int64) * c[p2p[:, 1]]).sum()
    assert total == 3000 * 2999 // 2
    # every particle pair is covered exactly once: mark (particle, particle) coverage
    leaf_of = np.empty(3000, dtype=np.int64)
    anc = {}
    for n in range(r.n_nodes):
        anc[n] = (r.tree["first"][n], r.tree["first"][n] + c[n])
    cover = np.zeros((3000, 3000), dtype=np.int8)
    for A, B in np.concatenate([m2l, p2p]):
        a0, a1 = anc[A]
        b0, b1 = anc[B]
        cover[a0:a1, b0:b1] += 1
        if A != B:
            cover[b0:b1, a0:a1] += 1
    np.fill_diagonal(cover, 1)
    assert np.all(cover == 1)
    # MAC holds for every accepted pair (eq. mac_criterion)
    Z, rm = r.Z, r.rmax
    d = Z[m2l[:, 0]] - Z[m2l[:, 1]]
    R = np.sqrt((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2])
    assert np.all(rm[m2l[:, 0]] + rm[m2l[:, 1]] <= 0.5 * R)
    # and every P2P pair between two leaves fails it (a pair that passes is never
    # evaluated directly)
    q = p2p[p2p[:, 0] != p2p[:, 1]]
    d = Z[q[:, 0]] - Z[q[:, 1]]
    R = np.sqrt((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2])
    assert not np.any((R > 0) & (rm[q[:, 0]] + rm[q[:, 1]] <= 0.5 * R))


def _read_walk_cases():
    cases, cur = [], None
    with open(os.path.join(GOLD, "walk_hand.txt")) as f:
        for line in f:
            w = line.split()
            if not w or w[0].startswith("#"):
                continue
            if w[0] == "case":
                cur = {"name": w[1], "tree": [], "m2l": [], "p2p": []}
            elif w[0] == "x":
                cur["x"] = np.array([float(v) for v in w[1:]])
            elif w[0] == "tree":
                cur["tree"].append([int(v) for v in w[1:]])
            elif w[0] in ("m2l", "p2p"):
                cur[w[0]].append([int(w[1]), int(w[2])])
            elif w[0] == "end":
                cases.append(cur)
    return cases


WALK_CASES = _read_walk_cases()


@pytest.mark.parametrize("case", WALK_CASES, ids=[c["name"] for c in WALK_CASES])
def test_walk_hand_worked_lists(orc, case):
    """Trees and lists worked out by hand (tests/golden/walk_hand.txt) for collinear unit
    masses with exact dyadic geometry: the split of the larger r_max, the tie-breaks by
    count and then by id, and the "<=" of eq. mac_criterion on a pair that sits exactly
    on r_A + r_B = theta R."""
    n = case["x"].shape[0]
    x = np.zeros((n, 3))
    x[:, 0] = case["x"]
    r = orc.run(x, np.ones(n), 2, 2, 0.5, 1, want_pot=False)
    t = np.array(case["tree"], dtype=np.int32)
    names = ("first", "count", "level", "parent", "child_first", "nchild")
    assert r.n_nodes == t.shape[0]
    for j, k in enumerate(names):
        assert np.array_equal(r.tree[k], t[:, j]), k
    assert np.array_equal(r.m2l, np.array(case["m2l"], dtype=np.int32).reshape(-1, 2))
    assert np.array_equal(r.p2p, np.array(case["p2p"], dtype=np.int32).reshape(-1, 2))


def test_walk_hand_worked_boundary_needs_le(orc):
    """The tie_by_id case with theta just below 1/2: the pair (4,5), which sits exactly on
    r_A + r_B = theta R at theta = 1/2, is no longer accepted and becomes P2P."""
    case = WALK_CASES[0]
    n = case["x"].shape[0]
    x = np.zeros((n, 3))
    x[:, 0] = case["x"]
    r = orc.run(x, np.ones(n), 2, 2, 0.5 - 2 ** -40, 1, want_pot=False)
    assert [4, 5] not in r.m2l.tolist() and [4, 5] in r.p2p.tolist()


def _check_trace(r, theta):
    """Every pair the walk visited was decided by eq. mac_criterion and reading A10, and
    the visited pairs are exactly Self(roots) plus the children of every split."""
    t = r.tree
    leaf = t["nchild"] == 0
    Z, rm, cnt = r.Z, r.rmax, t["count"]
    tr = r.trace
    A, B, dec = tr[:, 0].astype(np.int64), tr[:, 1].astype(np.int64), tr[:, 2]
    selfv = A == B
    assert np.all(dec[selfv & leaf[A]] == 2)                 # Self(leaf) -> P2P
    assert np.all(dec[selfv & ~leaf[A]] == 0)                # Self(inner) -> children
    d = Z[A] - Z[B]
    R = np.sqrt((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2])
    acc = (R > 0) & (rm[A] + rm[B] <= theta * R)
    pr = ~selfv
    assert np.all(dec[pr & acc] == 1)                        # accepted -> M2L
    assert np.all(acc[pr & (dec == 1)])
    both = leaf[A] & leaf[B]
    assert np.all(dec[pr & ~acc & both] == 2)                # rejected leaves -> P2P
    spl = pr & ~acc & ~both
    assert np.all((dec[spl] == 3) | (dec[spl] == 4))
    sa = dec == 3
    sb = dec == 4
    assert not np.any(sa & leaf[A]) and not np.any(sb & leaf[B])   # a leaf is never split
    inner = spl & ~leaf[A] & ~leaf[B]
    # the larger r_max is split; ties: the larger count, then the lower id
    want_a = np.where(rm[A] != rm[B], rm[A] > rm[B], np.where(cnt[A] != cnt[B], cnt[A] > cnt[B], A < B))
    assert np.array_equal(sa[inner], want_a[inner])
    # completeness: every visited pair is Self(root) or a child of exactly one split
    expect = [(0, 0)]
    for a, b, dd in zip(A.tolist(), B.tolist(), dec.tolist()):
        if dd == 0:
            c0, nc = t["child_first"][a], t["nchild"][a]
            for i in range(nc):
                for j in range(i, nc):
                    expect.append((c0 + i, c0 + j))
        elif dd in (3, 4):
            s = a if dd == 3 else b
            for c in range(t["child_first"][s], t["child_first"][s] + t["nchild"][s]):
                expect.append((c, b) if dd == 3 else (a, c))
    assert sorted(expect) == sorted(zip(A.tolist(), B.tolist()))
    # the lists are the M2L and P2P decisions, nothing else
    m2l = sorted((min(a, b), max(a, b)) for a, b, dd in zip(A.tolist(), B.tolist(), dec.tolist()) if dd == 1)
    p2p = sorted((min(a, b), max(a, b)) for a, b, dd in zip(A.tolist(), B.tolist(), dec.tolist()) if dd == 2)
    assert m2l == [tuple(v) for v in r.m2l.tolist()]
    assert p2p == [tuple(v) for v in r.p2p.tolist()]


@pytest.mark.parametrize("case", ["plummer", "hernquist-leaf1", "coincident"])
def test_walk_decisions_follow_the_rule(orc, case):
    """The oracle's walk trace, checked pair by pair: P2P only for leaf pairs that fail
    the acceptance test, splits only of pairs that fail it, the split node chosen by
    reading A10, and no pair visited that the recursion does not produce."""
    rng = np.random.default_rng(4)
    if case == "plummer":
        x, m = synth.plummer(3000, 4)
        leaf, theta = 8, 0.5
    elif case == "hernquist-leaf1":
        x, m = synth.hernquist(700, 10)
        leaf, theta = 1, 0.6
    else:
        x = np.concatenate([rng.normal(size=(300, 3)), np.repeat(rng.normal(size=(2, 3)), 20, axis=0)])
        m = rng.random(x.shape[0])
        leaf, theta = 4, 0.7
    r = orc.run(x, m, leaf, 2, theta, 0, want_pot=False, want_trace=True)
    _check_trace(r, theta)


def test_walk_counts_match_the_full_run(orc):
    """oracle.counts (tree and walk only, used to extrapolate the oracle's time to sizes it
    is not run at) gives the node, pair and particle-pair counts of the full evaluation."""
    x, m = synth.hernquist(5000, 21)
    r = orc.run(x, m, 12, 2, 0.55, 1, want_pot=False)
    c = r.tree["count"].astype(np.int64)
    P = r.p2p
    npp = int(np.where(P[:, 0] == P[:, 1], c[P[:, 0]] * (c[P[:, 0]] - 1) // 2, c[P[:, 0]] * c[P[:, 1]]).sum())
    assert orc.counts(x, m, 12, 0.55) == (r.n_nodes, r.n_m2l, r.n_p2p, npp)


def test_geometry_matches_definition(orc):
    x, m = synth.hernquist(2000, 6)
    r = orc.run(x, m, 12, 2, 0.5, 0)
    xs, ms = x[r.perm], m[r.perm]
    for n in range(r.n_nodes):
        f, c = r.tree["first"][n], r.tree["count"][n]
        M = ms[f:f + c].sum()
        Z = (ms[f:f + c, None] * xs[f:f + c]).sum(0) / M
        assert r.M[n] == pytest.approx(M, rel=1e-13)
        assert np.allclose(r.Z[n], Z, rtol=1e-12, atol=1e-14)
        rmax = np.sqrt(((xs[f:f + c] - r.Z[n]) ** 2).sum(1).max())
        assert r.rmax[n] == pytest.approx(rmax, rel=1e-13, abs=1e-15)


# ---------------------------------------------------------------- whole method

@pytest.mark.parametrize("variant", [0, 1])
def test_theta_zero_is_direct_sum(orc, variant):
    """At theta = 0 only zero-size cells pass the MAC, where the expansion is exact."""
    x, m = synth.plummer(1500, 8)
    r = orc.run(x, m, 6, 3, 0.0, variant)
    a, ph = orc.direct(x, m)
    assert rel(r.acc, a) < 1e-13
    assert rel(r.pot, ph) < 1e-13


def test_direct_two_body(orc):
    x = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [2.0, 0.0, 0.0]])
    m = np.array([3.0, 1.0, 0.5])
    a, ph = orc.direct(x, m)
    assert np.allclose(a[0], [1.5 / 4, 0, 0])
    assert np.allclose(a[1], [-3.0 / 4, 0, 0])      # coincident partner ignored
    assert ph[0] == pytest.approx(-1.5 / 2)


def _net(x, m, a):
    F = (m[:, None] * a).sum(0)
    T = (m[:, None] * np.cross(x, a)).sum(0)
    fs = (m * np.linalg.norm(a, axis=1)).sum()
    ts = (m * np.linalg.norm(x, axis=1) * np.linalg.norm(a, axis=1)).sum()
    return np.linalg.norm(F) / fs, np.linalg.norm(T) / ts


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_conservation(orc, p):
    """Net force vanishes for both forms (eq. netforce); net torque vanishes for the
    realigned form at every p and for the standard form at p = 1 (Sec. 3.1), and is
    far from zero for the standard form at p >= 2 (eq. total_torque)."""
    x, m = synth.plummer(4096, 1)
    for variant in (0, 1):
        r = orc.run(x, m, 16, p, 0.5, variant, want_pot=False, want_internals=False)
        f, t = _net(x, m, r.acc)
        assert f < 1e-14
        if variant == 1 or p == 1:
            assert t < 1e-14, (variant, p, t)
        else:
            assert t > 1e-8, (variant, p, t)


@pytest.mark.parametrize("variant", [0, 1])
def test_convergence_in_p_and_theta(orc, variant):
    x, m = synth.plummer(4096, 1)
    a, _ = orc.direct(x, m, want_pot=False)
    e = {}
    for p in (1, 2, 4, 6):
        for th in (0.3, 0.5, 0.7):
            r = orc.run(x, m, 16, p, th, variant, want_pot=False, want_internals=False)
            e[p, th] = rel(r.acc, a)
    for th in (0.3, 0.5, 0.7):
        assert e[1, th] > e[2, th] > e[4, th] > e[6, th]
    for p in (1, 2, 4, 6):
        assert e[p, 0.3] < e[p, 0.5] < e[p, 0.7]
    assert e[6, 0.3] < 1e-4


def test_plummer_energy(orc):
    """Potential energy W = 1/2 sum m phi of a unit Plummer sphere is -3 pi / 32."""
    x, m = synth.plummer(16384, 21)
    r = orc.run(x, m, 16, 4, 0.5, 0, want_pot=True, want_internals=False)
    W = 0.5 * (m * r.pot).sum()
    assert W == pytest.approx(-3 * math.pi / 32, rel=0.03)


def test_hernquist_energy(orc):
    """W = -1/(6a) for a unit-mass Hernquist sphere (a = 1); the u <= 0.999 cut lowers |W| slightly."""
    x, m = synth.hernquist(16384, 22)
    r = orc.run(x, m, 16, 4, 0.5, 0, want_pot=True, want_internals=False)
    W = 0.5 * (m * r.pot).sum()
    assert W == pytest.approx(-1.0 / 6.0, rel=0.05)


def test_plummer_potential_profile(orc):
    """The FMM potential follows Phi(r) = -1/sqrt(r^2 + 1) (shell averages)."""
    x, m = synth.plummer(16384, 23)
    r = orc.run(x, m, 16, 4, 0.5, 0, want_pot=True, want_internals=False)
    rad = np.linalg.norm(x, axis=1)
    for lo, hi in ((0.2, 0.4), (0.5, 0.8), (1.0, 1.5), (2.0, 3.0)):
        s = (rad > lo) & (rad < hi)
        want = (-1 / np.sqrt(rad[s] ** 2 + 1)).mean()
        assert r.pot[s].mean() == pytest.approx(want, rel=0.02)


# ---------------------------------------------------------------- literal order-0 realigned form

def _paper0_pairwise(ZA, XA, ZB, YB, mB):
    """Per-pair sum of eqs. realign2 and nab-expansion: a_a = sum_b -(m_b/R^2) (n + delta)
    (1 - n.delta), delta = ((X_a - Z_A) - (Y_b - Z_B)) / R, n = R/|R|, R = Z_A - Z_B."""
    R = ZA - ZB
    r = np.linalg.norm(R)
    n = R / r
    out = np.zeros_like(XA)
    for a in range(XA.shape[0]):
        delta = ((XA[a] - ZA)[None, :] - (YB - ZB)) / r
        nd = delta @ n
        out[a] = (-(mB / r ** 2)[:, None] * (n[None, :] + delta) * (1.0 - nd)[:, None]).sum(0)
    return out


@pytest.mark.parametrize("seed", range(4))
def test_paper0_closed_form_equals_pairwise_expansion(orc, seed):
    """The cell form of eq. aaB0 (monopole, x_perp, (n.x)x and Qbar terms) equals the
    particle-by-particle sum of the expanded realigned pair forces it was derived from,
    given that Z_B is the centre of mass of B (the dipole vanishes)."""
    rng = np.random.default_rng(40 + seed)
    XA = rng.normal(size=(7, 3)) * 0.3
    YB = rng.normal(size=(11, 3)) * 0.4 + rng.normal(size=3) * 3.0 + np.array([4.0, 0.0, 0.0])
    mB = rng.random(11) + 0.1
    ZA = XA.mean(0) + 0.03
    ZB = (mB[:, None] * YB).sum(0) / mB.sum()
    a1, _ = orc.cell_pair(1, 2, ZA, XA, ZB, YB, mB)
    a2 = _paper0_pairwise(ZA, XA, ZB, YB, mB)
    assert rel(a1, a2) < 1e-13


def test_paper0_single_source_is_central_and_first_order(orc):
    """With one source particle (Qbar = 0) every force lies on X_a - Y_b, and its error
    against Newton falls linearly with the separation (the expansion is of order 0 in
    magnitude and 1 in direction)."""
    rng = np.random.default_rng(3)
    XA = rng.normal(size=(6, 3)) * 0.2
    errs = []
    for dist in (4.0, 8.0, 16.0, 32.0):
        YB = np.array([[dist, 0.3, -0.2]])
        mB = np.array([1.7])
        a, _ = orc.cell_pair(1, 2, XA.mean(0), XA, YB[0], YB, mB)
        d = XA - YB
        assert np.abs(np.cross(a, d)).max() <= 1e-14 * np.abs(a).max() * np.abs(d).max()
        exact = -mB[0] * d / (np.linalg.norm(d, axis=1) ** 3)[:, None]
        errs.append(rel(a, exact))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(1.7 < q < 2.3 for q in ratios), ratios


def test_paper0_run_conserves_momenta(orc):
    """The literal order-0 realigned form conserves linear and angular momentum in the
    full FMM (pair forces central and antisymmetric), at roundoff."""
    x, m = synth.plummer(3000, 11)
    a, _ = orc.direct(x, m, want_pot=False)
    errs = []
    for th in (0.3, 0.6):
        r = orc.run(x, m, 16, 1, th, 2, want_pot=False, want_internals=False)
        f, t = _net(x, m, r.acc)
        assert f < 1e-14 and t < 1e-14, (th, f, t)
        s = orc.run(x, m, 16, 1, th, 0, want_pot=False, want_internals=False)
        errs.append(rel(r.acc, a))
        # same order as the standard monopole expansion (Sec. 3.1 vs Sec. 3.2)
        assert rel(s.acc, a) < errs[-1] < 2 * rel(s.acc, a), (th, errs[-1], rel(s.acc, a))
    assert errs[0] < errs[1]


def test_paper0_requires_order_one(orc):
    x, m = synth.plummer(100, 1)
    with pytest.raises(ValueError):
        orc.run(x, m, 16, 2, 0.5, 2)
