"""Host checks of the arithmetic the binary64 pair kernel's r^-3 rests on (eq. `jia`).

The kernel seeds y0 ~ s^(-1/2) with a binary32 reciprocal square root, forms t = y0^2 and
y0^3 from y0's 24-bit integer significand, e = 1 - s t with one fused multiply-add, the e^2
terms of the binomial series in binary32, and r^-3 = y0^3 (1 + 3/2 e + 15/8 e^2).  These
tests restate those steps with Python integers and numpy and check:

* the integer square and cube equal the binary64 products y0*y0 and (y0*y0)*y0 bit for bit
  (round to nearest, ties to even), so moving them off the binary64 unit changes nothing;
* the whole refinement stays within 2 ulp of s^(-3/2) (and 1 ulp of s^(-1/2)), with a
  seed perturbed by a few binary32 ulps, as the approximate binary32 instruction may be.
"""
import struct

import numpy as np
import pytest


def _f64(bits):
    return struct.unpack("<d", struct.pack("<Q", bits & (2**64 - 1)))[0]


def _square_cube(m, ey):
    """t = y0^2 and RN(y0^3) for y0 = m 2^(ey - 23), m the 24-bit significand."""
    m2 = m * m
    h2 = m2 >> 47
    t = _f64(((2 * ey + h2 + 1023) << 52) | ((m2 << (6 - h2)) & (2**52 - 1)))
    p = m2 * m
    lo, hi = p & (2**64 - 1), p >> 64
    lead = 64 + hi.bit_length() - 1
    sh = lead - 52
    sig = ((hi << (64 - sh)) & (2**64 - 1)) | (lo >> sh)
    rem, half = lo & ((1 << sh) - 1), 1 << (sh - 1)
    if rem > half or (rem == half and sig & 1):
        sig += 1
    ew = 3 * ey - 69 + lead
    if sig >> 53:
        sig >>= 1
        ew += 1
    return t, _f64(((ew + 1023) << 52) | (sig & (2**52 - 1)))


def test_integer_square_and_cube_are_the_binary64_products():
    rng = np.random.default_rng(11)
    ms = list(rng.integers(2**23, 2**24, 20000)) + [2**23, 2**23 + 1, 2**24 - 1, 2**24 - 2]
    eys = list(rng.integers(-301, 301, len(ms)))
    for m, ey in zip(ms, eys):
        m, ey = int(m), int(ey)
        y0 = m * 2.0 ** (ey - 23)
        t, w0 = _square_cube(m, ey)
        assert t == y0 * y0, (m, ey)
        assert w0 == (y0 * y0) * y0, (m, ey)


def test_ties_to_even_in_the_cube():
    # m^3 drops 17..19 bits; an exact half-ulp remainder needs 3 v2(m) = 18 with 19 bits
    # dropped, i.e. m = 64 o (o odd) and m^3 >= 2^71.  Every such tie must round to the even
    # significand, as the binary64 product does.
    o = (int(2 ** (71 / 3)) + 64) // 64 | 1  # the first odd o with (64 o)^3 >= 2^71
    ties = 0
    for m in range(64 * o, 2**24, 128)[:5000]:
        p = m * m * m
        assert p.bit_length() == 72
        sh = p.bit_length() - 53
        assert p & ((1 << sh) - 1) == 1 << (sh - 1)  # an exact tie
        y0 = m * 2.0**-23
        assert _square_cube(m, 0)[1] == (y0 * y0) * y0, m
        ties += 1
    assert ties == 5000


def _seeded_rinv(s, perturb, rng):
    """the kernel's steps on binary64 arrays s (float64), in numpy; fused multiply-adds in
    extended precision, rounded once"""
    L = np.longdouble
    b = s.view(np.int64)
    e = (b >> 52) - 1023
    k = e >> 1
    sb = (((e - 2 * k + 127) << 23) | ((b >> 29) & 0x7FFFFF)).astype(np.uint32)
    y = (1.0 / np.sqrt(sb.view(np.float32).astype(np.float64))).astype(np.float32)
    for _ in range(perturb):  # up to `perturb` binary32 ulps either way
        y = np.nextafter(y, np.float32(2) * rng.integers(0, 2, len(y)).astype(np.float32), dtype=np.float32)
    yb = y.view(np.uint32).astype(np.int64)
    y0 = ((((yb >> 23) - 127 - k + 1023) << 52) | ((yb & 0x7FFFFF) << 29)).view(np.float64)
    t = y0 * y0
    w0 = t * y0
    er = (L(1) - L(s) * L(t)).astype(np.float64)
    # e from its high word as binary32 (20 significand bits), e^2 terms in binary32
    hi = er.view(np.int64) >> 32
    ef = ((hi >> 20) & 0x7FF) - 896
    fb = ((hi & 0x80000000) | (np.maximum(ef, 0) << 23) | ((hi & 0xFFFFF) << 3)).astype(np.uint32)
    erf = np.where(ef > 0, fb.view(np.float32), np.float32(0))
    q3 = ((np.float32(1.875) * erf).astype(np.float32) * erf).astype(np.float32).astype(np.float64)
    q1 = ((np.float32(0.375) * erf).astype(np.float32) * erf).astype(np.float32).astype(np.float64)
    c3 = (L(er) * L(1.5) + L(q3)).astype(np.float64)
    c1 = (L(er) * L(0.5) + L(q1)).astype(np.float64)
    w3 = (L(w0) * L(c3) + L(w0)).astype(np.float64)
    ir = (L(y0) * L(c1) + L(y0)).astype(np.float64)
    return w3, ir


@pytest.mark.skipif(np.finfo(np.longdouble).nmant < 60, reason="needs an extended-precision long double")
def test_seeded_r3_within_two_ulp():
    rng = np.random.default_rng(3)
    # separations squared over the kernel's fast range |log2 s| <= 600 and the unit scale
    s = np.concatenate([2.0 ** rng.uniform(-600, 600, 40000), rng.uniform(0.25, 4.0, 40000)])
    L = np.longdouble
    for perturb in (0, 3):
        w3, ir = _seeded_rinv(s, perturb, rng)
        ref3 = L(s) ** L(-1.5)
        ref1 = L(s) ** L(-0.5)
        ok = np.isfinite(w3) & (ref3 < L(1e300)) & (ref3 > L(1e-300))
        err3 = (np.abs((L(w3) - ref3) / ref3).astype(np.float64) / 2.0**-53)[ok]
        err1 = (np.abs((L(ir) - ref1) / ref1).astype(np.float64) / 2.0**-53)
        assert ok.sum() > 60000
        assert err3.max() < 2.0, err3.max()
        assert err1.max() < 1.01, err1.max()
