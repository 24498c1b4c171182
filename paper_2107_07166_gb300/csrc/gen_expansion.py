"""Emits the unrolled expansion operators of the CUDA path, one header per order p.

The paper (Sec. 5) points at symbolic generation for higher-order multipole
operators; this script is that generator.  For each p in 1..8 it writes
``gen/exp_p{p}.cuh`` with straight-line device code, templated on the arithmetic type
T (double, or float in mixed precision), for:

  dtensor  D_alpha = d^alpha(-1/r) at R, |alpha| <= p, from the closed form
           d^alpha f(r) = sum_k prod_d [alpha_d! / (2^k_d k_d! (alpha_d - 2k_d)!)] R^(alpha-2k) f_(|alpha|-|k|)
           with the radial derivatives f_m = (r^-1 d/dr)^m f:
              f = -1/r   : f_m = -(-1)^m (2m-1)!! r^-(2m+1)
              h = -r^-3  : h_m = -(-1)^m (2m+1)!! r^-(2m+3)
  htensor  h_alpha for |alpha| <= p-1 (kernel of the realigned force)
  m2l_std  L_gamma += sum_{|beta|+|gamma|<=p} M_beta D_{beta+gamma}       (eq. taylor)
  m2l_con  S_gamma += s_gamma,  U_gamma += R s_gamma + w_gamma with
           s_gamma = sum M_beta h_{beta+gamma},  w_{i,gamma} = sum (beta_i+1) M_{beta+e_i} h_{beta+gamma};
           the (beta_i+1) M_{beta+e_i} factors are formed once per cell (con_moments) and R is
           folded into them per pair, so U_{i,gamma} += sum_beta (C_{i,beta} + R_i M_beta) h_{beta+gamma}
  m2l_con_o  the same without the per-pair fold: the source factors are formed once per
           cell about its system's root centre, Q_{i,beta} = C_{i,beta} - z_i M_beta with
           z = Z_cell - Z_root (con_moments_o), so U_{i,gamma} += sum_beta Q_{i,beta} h_{beta+gamma},
           and z_tgt,i S_gamma is added once per target cell after the sum over its sources
           (R = z_tgt - z_src makes the two forms equal in exact arithmetic)
  p2m      M_alpha += m (-y)^alpha / alpha!
  m2m      M^P_alpha += sum_{beta<=alpha} M^c_{alpha-beta} (-c)^beta / beta!
  l2l      L'_gamma += sum_beta L_{gamma+beta} s^beta / beta!
  l2p      standard: a_i = -sum_{|g|<=p-1} L_{g+e_i} x^g/g!, phi = sum L_g x^g/g!
           conserving: a = x S(x) + U(x)

Multi-indices are ordered by degree, then alpha_x descending, then alpha_y descending.
The generator is self-contained (no table is shared with any other component).
"""
from __future__ import annotations

import math
import os
import sys
from fractions import Fraction

PMAX = 8  # orders compiled into the library (M2L of p = 7, 8: the table-driven m2l_generic.cu)
MIXED_PMAX = 6  # highest order of the binary32 M2L (p = 7, 8 run in binary64 only)
DF64_PMAX = 5  # highest order of the double-float M2L (p = 6 takes minutes to compile)


def mis(p):
    out = []
    for n in range(p + 1):
        for ax in range(n, -1, -1):
            for ay in range(n - ax, -1, -1):
                out.append((ax, ay, n - ax - ay))
    return out


def nmi(p):
    return (p + 1) * (p + 2) * (p + 3) // 6 if p >= 0 else 0


def idx(a):
    """position of multi-index a in the ordering above (closed form)."""
    n = sum(a)
    j = n - a[0]
    return n * (n + 1) * (n + 2) // 6 + j * (j + 1) // 2 + (j - a[1])


def fact(a):
    return math.factorial(a[0]) * math.factorial(a[1]) * math.factorial(a[2])


def lit(v: Fraction) -> str:
    """C literal of a rational constant in type T."""
    v = Fraction(v)
    if v.denominator == 1:
        return f"T({v.numerator}.0)"
    return f"T({float(v)!r})"


def mono_name(a):
    return f"m{a[0]}{a[1]}{a[2]}"


def emit_monomials(lines, var, p, name="m", scale_fact=False):
    """Emit T {name}{ax}{ay}{az} = var^a (optionally / a!) for all |a| <= p."""
    vx, vy, vz = var
    lines.append(f"  T {name}px[{p + 1}], {name}py[{p + 1}], {name}pz[{p + 1}];")
    lines.append(f"  {name}px[0] = T(1); {name}py[0] = T(1); {name}pz[0] = T(1);")
    for k in range(1, p + 1):
        if scale_fact:
            lines.append(f"  {name}px[{k}] = {name}px[{k - 1}] * {vx} * T({1.0 / k!r});")
            lines.append(f"  {name}py[{k}] = {name}py[{k - 1}] * {vy} * T({1.0 / k!r});")
            lines.append(f"  {name}pz[{k}] = {name}pz[{k - 1}] * {vz} * T({1.0 / k!r});")
        else:
            lines.append(f"  {name}px[{k}] = {name}px[{k - 1}] * {vx};")
            lines.append(f"  {name}py[{k}] = {name}py[{k - 1}] * {vy};")
            lines.append(f"  {name}pz[{k}] = {name}pz[{k - 1}] * {vz};")


def mono_expr(name, a):
    parts = []
    if a[0]:
        parts.append(f"{name}px[{a[0]}]")
    if a[1]:
        parts.append(f"{name}py[{a[1]}]")
    if a[2]:
        parts.append(f"{name}pz[{a[2]}]")
    if not parts:
        return "T(1)"
    return " * ".join(parts)


def radial_tensor(p, kind):
    """Device function computing the derivative tensor up to order p.
    kind 'd': f = -1/r ; kind 'h': f = -r^-3."""
    L = []
    fn = "dtensor" if kind == "d" else "htensor"
    L.append(f"  /* {'D_alpha = d^alpha(-1/r)' if kind == 'd' else 'h_alpha = d^alpha(-r^-3)'} at R, |alpha| <= {p} */")
    L.append(f"  template <class T> __device__ __forceinline__ static void {fn}(T rx, T ry, T rz, T* __restrict__ D) {{")
    L.append("    T r2 = rx * rx + ry * ry + rz * rz;")
    L.append("    T ri = rsqrt_t(r2);")
    L.append("    T ri2 = ri * ri;")
    # radial derivatives
    if kind == "d":
        L.append("    T g0 = -ri;")
        for m in range(1, p + 1):
            L.append(f"    T g{m} = g{m - 1} * ri2 * T({-(2 * m - 1)}.0);")
    else:
        L.append("    T g0 = -ri * ri2;")
        for m in range(1, p + 1):
            L.append(f"    T g{m} = g{m - 1} * ri2 * T({-(2 * m + 1)}.0);")
    body = []
    emit_monomials(body, ("rx", "ry", "rz"), p, name="q")
    L += ["  " + b for b in body]
    for a in mis(p):
        terms = {}
        for kx in range(a[0] // 2 + 1):
            for ky in range(a[1] // 2 + 1):
                for kz in range(a[2] // 2 + 1):
                    k = (kx, ky, kz)
                    c = Fraction(1)
                    for d in range(3):
                        c *= Fraction(math.factorial(a[d]),
                                      2 ** k[d] * math.factorial(k[d]) * math.factorial(a[d] - 2 * k[d]))
                    mexp = sum(a) - sum(k)
                    rest = (a[0] - 2 * kx, a[1] - 2 * ky, a[2] - 2 * kz)
                    terms.setdefault(mexp, []).append((c, rest))
        expr = []
        for mexp, tl in sorted(terms.items()):
            poly = " + ".join(
                (f"{lit(c)} * {mono_expr('q', r)}" if c != 1 else mono_expr("q", r)) for c, r in tl)
            expr.append(f"g{mexp} * ({poly})")
        L.append(f"    D[{idx(a)}] = {' + '.join(expr)};")
    L.append("  }")
    return L


def m2l_std(p):
    L = ["  /* L_gamma += sum_{|beta|+|gamma|<=p} M_beta D_{beta+gamma} */",
         "  template <class T, class A> __device__ __forceinline__ static void m2l_std(const T* __restrict__ M, const T* __restrict__ D, A* __restrict__ Lc) {"]
    for b in mis(p):
        rem = p - sum(b)
        L.append(f"    {{ const T mb = M[{idx(b)}];")
        for g in mis(rem):
            s = (b[0] + g[0], b[1] + g[1], b[2] + g[2])
            L.append(f"      Lc[{idx(g)}] = fma_t(mb, D[{idx(s)}], Lc[{idx(g)}]);")
        L.append("    }")
    L.append("  }")
    return L


def m2l_std_s(p):
    """m2l_std with the source moments rescaled on load: M_beta * f[|beta|]."""
    L = ["  /* as m2l_std, with every moment multiplied on load by f[|beta|] (a power of two) */",
         "  template <class T, class A> __device__ __forceinline__ static void m2l_std_s(const T* __restrict__ M, const float* __restrict__ f, const T* __restrict__ D, A* __restrict__ Lc) {"]
    for b in mis(p):
        rem = p - sum(b)
        L.append(f"    {{ const T mb = scale_t(M[{idx(b)}], f[{sum(b)}]);")
        for g in mis(rem):
            s = (b[0] + g[0], b[1] + g[1], b[2] + g[2])
            L.append(f"      Lc[{idx(g)}] = fma_t(mb, D[{idx(s)}], Lc[{idx(g)}]);")
        L.append("    }")
    L.append("  }")
    return L


def con_moments(p):
    q = p - 1
    nq = nmi(q)
    L = ["  /* conserving source moments: [M_b | (b_x+1) M_{b+e_x} | (b_y+1) M_{b+e_y} | (b_z+1) M_{b+e_z}], |b| <= p-1 */",
         "  template <class T> __device__ __forceinline__ static void con_moments(const T* __restrict__ M, T* __restrict__ C) {"]
    for b in mis(q):
        bi = idx(b)
        L.append(f"    C[{bi}] = M[{bi}];")
        L.append(f"    C[{nq + bi}] = T({b[0] + 1}.0) * M[{idx((b[0] + 1, b[1], b[2]))}];")
        L.append(f"    C[{2 * nq + bi}] = T({b[1] + 1}.0) * M[{idx((b[0], b[1] + 1, b[2]))}];")
        L.append(f"    C[{3 * nq + bi}] = T({b[2] + 1}.0) * M[{idx((b[0], b[1], b[2] + 1))}];")
    L.append("  }")
    return L


def m2l_con(p):
    q = p - 1
    nq = nmi(q)
    L = ["  /* conserving M2L from conserving moments C (see con_moments): with the per-pair",
         "     M''_{i,b} = C_{i,b} + R_i M_b,  S_g += sum_b M_b h_{b+g},  U_{i,g} += sum_b M''_{i,b} h_{b+g}",
         "     (= R_i s_g + w_{i,g}).  SU layout: [S (nq) | Ux | Uy | Uz] */",
         "  template <class T, class A> __device__ __forceinline__ static void m2l_con(const T* __restrict__ C, const T* __restrict__ H, T rx, T ry, T rz, A* __restrict__ SU) {"]
    for b in mis(q):
        bi = idx(b)
        rem = q - sum(b)
        L.append(f"    {{ const T m = C[{bi}];")
        L.append(f"      const T mx = fma_t(rx, m, C[{nq + bi}]), my = fma_t(ry, m, C[{2 * nq + bi}]), mz = fma_t(rz, m, C[{3 * nq + bi}]);")
        for g in mis(rem):
            gi = idx(g)
            hb = f"H[{idx((b[0] + g[0], b[1] + g[1], b[2] + g[2]))}]"
            L.append(f"      SU[{gi}] = fma_t(m, {hb}, SU[{gi}]); SU[{nq + gi}] = fma_t(mx, {hb}, SU[{nq + gi}]);"
                     f" SU[{2 * nq + gi}] = fma_t(my, {hb}, SU[{2 * nq + gi}]); SU[{3 * nq + gi}] = fma_t(mz, {hb}, SU[{3 * nq + gi}]);")
        L.append("    }")
    L.append("  }")
    return L


def con_moments_o(p):
    q = p - 1
    nq = nmi(q)
    L = ["  /* conserving source moments about the system's root centre: [M_b | (b_i+1) M_{b+e_i} - z_i M_b],",
         "     |b| <= p-1, z = Z_cell - Z_root */",
         "  template <class T> __device__ __forceinline__ static void con_moments_o(const T* __restrict__ M, T zx, T zy, T zz, T* __restrict__ C) {"]
    for b in mis(q):
        bi = idx(b)
        L.append(f"    C[{bi}] = M[{bi}];")
        L.append(f"    C[{nq + bi}] = fma_t(-zx, M[{bi}], T({b[0] + 1}.0) * M[{idx((b[0] + 1, b[1], b[2]))}]);")
        L.append(f"    C[{2 * nq + bi}] = fma_t(-zy, M[{bi}], T({b[1] + 1}.0) * M[{idx((b[0], b[1] + 1, b[2]))}]);")
        L.append(f"    C[{3 * nq + bi}] = fma_t(-zz, M[{bi}], T({b[2] + 1}.0) * M[{idx((b[0], b[1], b[2] + 1))}]);")
    L.append("  }")
    return L


def m2l_con_o(p):
    q = p - 1
    nq = nmi(q)
    L = ["  /* conserving M2L from the root-relative source moments of con_moments_o: S_g += sum_b Q_b h_{b+g},",
         "     U_{i,g} += sum_b Q_{i,b} h_{b+g}; the target's z_i S_g is added once after all its sources */",
         "  template <class T, class A> __device__ __forceinline__ static void m2l_con_o(const T* __restrict__ C, const T* __restrict__ H, A* __restrict__ SU) {"]
    for b in mis(q):
        bi = idx(b)
        rem = q - sum(b)
        L.append(f"    {{ const T m = C[{bi}], mx = C[{nq + bi}], my = C[{2 * nq + bi}], mz = C[{3 * nq + bi}];")
        for g in mis(rem):
            gi = idx(g)
            hb = f"H[{idx((b[0] + g[0], b[1] + g[1], b[2] + g[2]))}]"
            L.append(f"      SU[{gi}] = fma_t(m, {hb}, SU[{gi}]); SU[{nq + gi}] = fma_t(mx, {hb}, SU[{nq + gi}]);"
                     f" SU[{2 * nq + gi}] = fma_t(my, {hb}, SU[{2 * nq + gi}]); SU[{3 * nq + gi}] = fma_t(mz, {hb}, SU[{3 * nq + gi}]);")
        L.append("    }")
    L.append("  }")
    return L


def m2l_con_s(p):
    """m2l_con with the conserving moments rescaled on load: the M_b block by f[|b|], the
    (b_i + 1) M_{b+e_i} blocks by f[|b| + 1]."""
    q = p - 1
    nq = nmi(q)
    L = ["  /* as m2l_con, with C_b multiplied on load by f[|b|] and C_{i,b} by f[|b|+1] (powers of two) */",
         "  template <class T, class A> __device__ __forceinline__ static void m2l_con_s(const T* __restrict__ C, const float* __restrict__ f, const T* __restrict__ H, T rx, T ry, T rz, A* __restrict__ SU) {"]
    for b in mis(q):
        bi = idx(b)
        rem = q - sum(b)
        nb, nb1 = sum(b), sum(b) + 1
        L.append(f"    {{ const T m = scale_t(C[{bi}], f[{nb}]);")
        L.append(f"      const T mx = fma_t(rx, m, scale_t(C[{nq + bi}], f[{nb1}])), my = fma_t(ry, m, scale_t(C[{2 * nq + bi}], f[{nb1}])),"
                 f" mz = fma_t(rz, m, scale_t(C[{3 * nq + bi}], f[{nb1}]));")
        for g in mis(rem):
            gi = idx(g)
            hb = f"H[{idx((b[0] + g[0], b[1] + g[1], b[2] + g[2]))}]"
            L.append(f"      SU[{gi}] = fma_t(m, {hb}, SU[{gi}]); SU[{nq + gi}] = fma_t(mx, {hb}, SU[{nq + gi}]);"
                     f" SU[{2 * nq + gi}] = fma_t(my, {hb}, SU[{2 * nq + gi}]); SU[{3 * nq + gi}] = fma_t(mz, {hb}, SU[{3 * nq + gi}]);")
        L.append("    }")
    L.append("  }")
    return L


def m2l_con_m(p):
    """Conserving M2L that forms the conserving moments from the raw moments on load:
    C_b = M_b f[|b|], C_{i,b} = (b_i + 1) M_{b+e_i} f[|b|+1] (f powers of two).  Reads nmi(p)
    values per source instead of 4 nmi(p-1)."""
    q = p - 1
    nq = nmi(q)
    L = ["  /* as m2l_con, reading the raw moments M (|a| <= p): C_b = M_b f[|b|] and",
         "     C_{i,b} = (b_i+1) M_{b+e_i} f[|b|+1] are formed on load */",
         "  template <class T, class A> __device__ __forceinline__ static void m2l_con_m(const T* __restrict__ M, const float* __restrict__ f, const T* __restrict__ H, T rx, T ry, T rz, A* __restrict__ SU) {"]
    def w(b, d):
        e = list(b)
        e[d] += 1
        c = b[d] + 1
        n = sum(b) + 1
        if c == 1:
            return f"scale_t(M[{idx(tuple(e))}], f[{n}])"
        return f"scale_c_t(M[{idx(tuple(e))}], f[{n}], {c}.f)"
    for b in mis(q):
        bi = idx(b)
        rem = q - sum(b)
        L.append(f"    {{ const T m = scale_t(M[{bi}], f[{sum(b)}]);")
        L.append(f"      const T mx = fma_t(rx, m, {w(b, 0)}), my = fma_t(ry, m, {w(b, 1)}), mz = fma_t(rz, m, {w(b, 2)});")
        for g in mis(rem):
            gi = idx(g)
            hb = f"H[{idx((b[0] + g[0], b[1] + g[1], b[2] + g[2]))}]"
            L.append(f"      SU[{gi}] = fma_t(m, {hb}, SU[{gi}]); SU[{nq + gi}] = fma_t(mx, {hb}, SU[{nq + gi}]);"
                     f" SU[{2 * nq + gi}] = fma_t(my, {hb}, SU[{2 * nq + gi}]); SU[{3 * nq + gi}] = fma_t(mz, {hb}, SU[{3 * nq + gi}]);")
        L.append("    }")
    L.append("  }")
    return L


def p2m(p):
    L = ["  /* M_alpha += m (-y)^alpha / alpha!,  y = Y - Z */",
         "  template <class T> __device__ __forceinline__ static void p2m(T m, T yx, T yy, T yz, T* __restrict__ M) {"]
    body = []
    emit_monomials(body, ("(-yx)", "(-yy)", "(-yz)"), p, name="w", scale_fact=True)
    L += ["  " + b for b in body]
    for a in mis(p):
        L.append(f"    M[{idx(a)}] = fma_t(m, {mono_expr('w', a)}, M[{idx(a)}]);")
    L.append("  }")
    return L


def _axis_pass(L, src, dst, p, axis, w, up):
    """One axis of a separable shift over all multi-indices of degree <= p:
    dst[g] = sum_k src[g +- k e_axis] w[k] (k = 0 ... while the index stays inside),
    with + (up: locals, the index rises) or - (moments, the index falls)."""
    for g in mis(p):
        kmax = (p - sum(g)) if up else g[axis]
        expr = f"{src}[{idx(g)}]"
        for k in range(1, kmax + 1):
            h = list(g)
            h[axis] += k if up else -k
            expr = f"fma_t({src}[{idx(tuple(h))}], {w}[{k}], {expr})"
        L.append(f"    {dst}[{idx(g)}] = {expr};")


def m2m(p):
    """M^P_alpha += sum_{beta<=alpha} M^c_{alpha-beta} (-c)^beta/beta!, as three one-axis
    shifts: (-c)^beta/beta! factors over the axes, so the sum over beta is a sum over
    beta_x, then beta_y, then beta_z (about half the multiply-adds of the direct sum at
    p = 4, a third at p = 8)."""
    n = nmi(p)
    L = ["  /* M^P_alpha += sum_{beta<=alpha} M^c_{alpha-beta} (-c)^beta/beta!,  c = Z_child - Z_parent,",
         "     one axis at a time */",
         "  template <class T> __device__ __forceinline__ static void m2m(const T* __restrict__ Mc, T cx, T cy, T cz, T* __restrict__ Mp) {"]
    body = []
    emit_monomials(body, ("(-cx)", "(-cy)", "(-cz)"), p, name="w", scale_fact=True)
    L += ["  " + b for b in body]
    L.append(f"    T A[{n}], B[{n}];")
    _axis_pass(L, "Mc", "A", p, 0, "wpx", False)
    _axis_pass(L, "A", "B", p, 1, "wpy", False)
    _axis_pass(L, "B", "A", p, 2, "wpz", False)
    for g in mis(p):
        L.append(f"    Mp[{idx(g)}] = Mp[{idx(g)}] + A[{idx(g)}];")
    L.append("  }")
    return L


def l2l_poly(p, name):
    """L'_gamma += sum_beta L_{gamma+beta} s^beta/beta!, as three one-axis shifts (the
    factor s^beta/beta! splits over the axes)."""
    n = nmi(p)
    L = [f"  /* L'_gamma += sum_beta L_{{gamma+beta}} s^beta/beta!  (|gamma+beta| <= {p}), one axis at a time */",
         f"  template <class T> __device__ __forceinline__ static void {name}(const T* __restrict__ Lp, T sx, T sy, T sz, T* __restrict__ Lc) {{"]
    body = []
    emit_monomials(body, ("sx", "sy", "sz"), p, name="w", scale_fact=True)
    L += ["  " + b for b in body]
    L.append(f"    T A[{n}], B[{n}];")
    _axis_pass(L, "Lp", "A", p, 0, "wpx", True)
    _axis_pass(L, "A", "B", p, 1, "wpy", True)
    _axis_pass(L, "B", "A", p, 2, "wpz", True)
    for g in mis(p):
        L.append(f"    Lc[{idx(g)}] = Lc[{idx(g)}] + A[{idx(g)}];")
    L.append("  }")
    return L


def l2p_std(p):
    L = ["  /* standard L2P: a_i = -sum_{|g|<=p-1} L_{g+e_i} x^g/g!;  phi = sum_g L_g x^g/g! */",
         "  template <class T> __device__ __forceinline__ static void l2p_std(const T* __restrict__ Lc, T xx, T xy, T xz, T& ax, T& ay, T& az, T& phi) {"]
    body = []
    emit_monomials(body, ("xx", "xy", "xz"), p, name="w", scale_fact=True)
    L += ["  " + b for b in body]
    L.append("    T sx = T(0), sy = T(0), sz = T(0), sp = T(0);")
    for g in mis(p - 1):
        w = mono_expr("w", g)
        L.append(f"    {{ const T wg = {w};")
        L.append(f"      sx = fma_t(Lc[{idx((g[0] + 1, g[1], g[2]))}], wg, sx);")
        L.append(f"      sy = fma_t(Lc[{idx((g[0], g[1] + 1, g[2]))}], wg, sy);")
        L.append(f"      sz = fma_t(Lc[{idx((g[0], g[1], g[2] + 1))}], wg, sz); }}")
    for g in mis(p):
        L.append(f"    sp = fma_t(Lc[{idx(g)}], {mono_expr('w', g)}, sp);")
    L.append("    ax = -sx; ay = -sy; az = -sz; phi = sp;")
    L.append("  }")
    return L


def l2p_con(p):
    q = p - 1
    nq = nmi(q)
    L = ["  /* conserving L2P: a = x S(x) + U(x) */",
         "  template <class T> __device__ __forceinline__ static void l2p_con(const T* __restrict__ SU, T xx, T xy, T xz, T& ax, T& ay, T& az) {"]
    body = []
    emit_monomials(body, ("xx", "xy", "xz"), max(q, 0), name="w", scale_fact=True)
    L += ["  " + b for b in body]
    L.append("    T s = T(0), ux = T(0), uy = T(0), uz = T(0);")
    for g in mis(q):
        w = mono_expr("w", g)
        gi = idx(g)
        L.append(f"    {{ const T wg = {w};")
        L.append(f"      s = fma_t(SU[{gi}], wg, s);")
        L.append(f"      ux = fma_t(SU[{nq + gi}], wg, ux);")
        L.append(f"      uy = fma_t(SU[{2 * nq + gi}], wg, uy);")
        L.append(f"      uz = fma_t(SU[{3 * nq + gi}], wg, uz); }}")
    L.append("    ax = fma_t(xx, s, ux); ay = fma_t(xy, s, uy); az = fma_t(xz, s, uz);")
    L.append("  }")
    return L


def header(p):
    q = p - 1
    out = [f"// generated by gen_expansion.py -- expansion operators of order p = {p}",
           "#pragma once",
           '#include "../fmm_math.cuh"',
           "namespace gbfmm {",
           f"template <> struct Exp<{p}> {{",
           f"  static constexpr int P = {p};",
           f"  static constexpr int NM = {nmi(p)};   // moments / standard locals",
           f"  static constexpr int NMP = {(nmi(p) + 7) // 8 * 8};   // moments padded to 32 bytes (binary32 storage)",
           f"  static constexpr int NQ = {nmi(q)};   // conserving scalar local S (|gamma| <= p-1)",
           f"  static constexpr int NSU = {4 * nmi(q)};  // conserving locals S, Ux, Uy, Uz"]
    out += radial_tensor(p, "d")
    out += radial_tensor(q, "h")
    out += m2l_std(p)
    out += m2l_std_s(p)
    out += con_moments(p)
    out += con_moments_o(p)
    out += m2l_con(p)
    out += m2l_con_o(p)
    out += m2l_con_s(p)
    out += m2l_con_m(p)
    out += p2m(p)
    out += m2m(p)
    out += l2l_poly(p, "l2l")
    out += l2l_poly(q, "l2l_q")
    out += l2p_std(p)
    out += l2p_con(p)
    out.append("};")
    out.append("}  // namespace gbfmm")
    return "\n".join(out) + "\n"


def _write(path, txt):
    if not os.path.exists(path) or open(path).read() != txt:
        with open(path, "w") as f:
            f.write(txt)


def main(outdir):
    """Writes gen/exp_p{p}.cuh and the translation units that instantiate them:
    expansion_p{p}.cu (moments, translations, L2P) and expansion_p{p}_{type}.cu (M2L of one
    arithmetic type), so that the heavy instantiations compile in parallel."""
    os.makedirs(outdir, exist_ok=True)
    for p in range(1, PMAX + 1):
        _write(os.path.join(outdir, f"exp_p{p}.cuh"), header(p))
        inc = f'#include "exp_p{p}.cuh"\n#include "../expansion_impl.cuh"\n'
        _write(os.path.join(outdir, f"expansion_p{p}.cu"),
               f"// generated: expansion stages of order p = {p}\n" + inc +
               f"namespace gbfmm {{\nGBFMM_INSTANTIATE({p})\n}}\n")
        for tname, t in (("f64", "double"), ("f32", "float"), ("df64", "df64")):
            if (t == "df64" and p > DF64_PMAX) or (t == "float" and p > MIXED_PMAX):
                continue
            _write(os.path.join(outdir, f"expansion_p{p}_{tname}.cu"),
                   f"// generated: M2L of order p = {p} in {t}\n" + inc +
                   f"namespace gbfmm {{\nGBFMM_INSTANTIATE_M2L({p}, {t})\n}}\n")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)), "gen"))
