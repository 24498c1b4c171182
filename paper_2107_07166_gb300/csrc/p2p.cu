// a12 mutual particle-particle interactions (eq. jia and its gradient) and a14 diagnostics.
//
// One warp per leaf pair (A, B) of the P2P list (A == B: a leaf with itself).  The
// nA x nB particle pairs are spread flat over the 32 lanes, so lanes stay busy whatever
// the leaf sizes (leaves hold ~10 particles on average): lane t of a round takes pair
// (a, b) = (t / ncol, t % ncol) of a column panel, forms d = X_a - X_b, r^-1 and d r^-3
// and stores them in a shared-memory panel.  Two passes then sum the panel with one lane
// per (particle, component): rows give a_a = -sum_b m_b d r^-3 (phi_a = -sum_b m_b r^-1),
// columns give a_b = +sum_a m_a d r^-3 (phi_b = -sum_a m_a r^-1).  Each pair force is
// formed once and applied to both partners (action = reaction).  A self pair keeps a < b.
// Results go to a per-(pair, side, slot) partial buffer that the final per-particle
// kernels sum in list order: no floating-point atomics, run-to-run identical.
#include <type_traits>

#include "fmm_device.cuh"
#include "fmm_internal.h"
#include "fmm_math.cuh"
#include "fused_traverse.cuh"
#include "prec.cuh"

namespace gbfmm {

constexpr int PB = 128;                 // 4 warps
constexpr int PW = PB / 32;
// panel columns: 8-byte types use 8 columns so that four warps of panels leave room for
// four blocks per SM; 4-byte types use 16
template <class T>
struct Panel {
    static constexpr int COLS = sizeof(T) == 4 ? 16 : 8;
    static constexpr int ROW = COLS * 4 + 4;  // elements per panel row: [col][comp], padded (stride = 4 mod 16)
    static constexpr int SIZE = 32 * ROW;     // elements per warp panel
};

// Row stride and per-warp shared elements of p2p_k.  With 8-byte elements a warp's row
// reads (lane = (row a, component c)) need 2 wavefronts at best; a stride of 4 mod 16 does
// that for 4 components per row task, 3 mod 16 for 3 (the stride 36 with 3-component tasks
// put rows a and a + 4 on the same banks: 3 wavefronts per read).  Binary64 folds the
// masses into the pair terms (FOLD): the panel holds [d_x, d_y, d_z, m_b r^-3] per pair,
// then come [a][column] arrays of m_a r^-3 and, with potentials, of r^-1.
template <class T, bool POT>
struct PanelRow {
    static constexpr bool FOLD = std::is_same<T, double>::value;
    static constexpr int ROW = (sizeof(T) == 8 && !POT) ? Panel<T>::COLS * 4 + 3 : Panel<T>::ROW;
    static constexpr int AUX = FOLD ? (POT ? 2 : 1) : 0;
    static constexpr int WARP = FOLD ? 32 * ROW + 32 * Panel<T>::COLS * AUX : Panel<T>::SIZE;
};

// Columns per panel for an nA x nB leaf pair.  A panel of k columns costs
// ceil(nA k / 32) lane rounds of pair terms (about 17 arithmetic steps each), then rows
// (ceil(NC nA / 32) rounds of k steps) and columns (ceil(NC k / 32) rounds of nA steps);
// the width with the fewest lane rounds over all panels wins, ties to the wider panel.
// Leaves hold ~9 particles on average, so a fixed width of 8 leaves the last pair round
// of most panels partly idle.
template <int NC>
__device__ __forceinline__ int panel_cols(int nA, int nB, int cmax) {
    constexpr int KC = 17;
    int best = 1, bcost = 0x7fffffff;
    for (int k = min(cmax, nB); k >= 1; k--) {
        int full = nB / k, rem = nB - full * k;
        int ck = ((nA * k + 31) >> 5) * KC + ((NC * nA + 31) >> 5) * k + ((NC * k + 31) >> 5) * nA;
        int cr = rem ? ((nA * rem + 31) >> 5) * KC + ((NC * nA + 31) >> 5) * rem + ((NC * rem + 31) >> 5) * nA : 0;
        int cost = full * ck + cr;
        if (cost < bcost) {
            bcost = cost;
            best = k;
        }
    }
    return best;
}

// r^2 == 0 (coincident particles) without a floating-point compare: r^2 is a sum of squares,
// so it is +0 exactly when its bit pattern is 0 (binary64: keeps the test off the FP64 unit)
__device__ __forceinline__ bool r2_zero(double v) { return __double_as_longlong(v) == 0ll; }
__device__ __forceinline__ bool r2_zero(float v) { return __float_as_uint(v) == 0u; }
__device__ __forceinline__ bool r2_zero(df64 v) { return is_zero(v); }

// a binary32 value v >= 0 as binary64, by integer rebiasing (no binary64 instruction);
// zero and subnormal v give 0
__device__ __forceinline__ double sq_to_f64(float v) {
    unsigned b = __float_as_uint(v);
    int e = (int)(b >> 23);
    return e > 0 ? __hiloint2double(((e + (1023 - 127)) << 20) | (int)((b & 0x7fffff) >> 3), (int)((b & 7u) << 29))
                 : 0.0;
}

// s^(-3/2) (and, if IR, s^(-1/2)) for a binary64 s > 0: three binary64 operations for
// s^(-3/2), where the library reciprocal square root and the cube take seven.  The seed
// y0 ~ s^(-1/2) is the binary32 reciprocal square root of the mantissa of s rescaled into
// [1, 4), taken back to s's scale by integer exponent arithmetic, so the seed costs no
// binary64 instruction (relative error below 2^-21).  With t = y0^2 (exact: y0 has 24
// significant bits) and e = 1 - s t (one rounding, |e| < 2^-20),
//   s^(-3/2) = y0^3 (1 - e)^(-3/2) = y0^3 (1 + 3/2 e + 15/8 e^2 + ...),
//   s^(-1/2) = y0 (1 - e)^(-1/2)   = y0 (1 + 1/2 e + 3/8 e^2 + ...):
// the binomial series cut after e^2 leave remainders below 2^-58, under binary64's own
// rounding.  The e^2 terms are below 2^-40 of the result and need only ~12 correct bits,
// so they are formed in binary32 (host emulation with a seed perturbed by a few ulp: the
// same 1.96-ulp maximum error as the all-binary64 form).  t and y0^3 come from y0's 24-bit
// integer significand by integer products, exactly the values of the binary64 products
// y0 y0 and t y0 (host check on random significands and on exact ties:
// tests/test_rinv_arith.py).  That leaves e = 1 - s t and the two fused multiply-adds of
// the series to the binary64 unit.  Exponents far from 0 (|e| > 600: subnormal, huge or
// non-finite s) take the library path.
template <bool IR>
__device__ __forceinline__ void rinv_f64(double s, double& w3, double& ir) {
    long long b = __double_as_longlong(s);
    int e = (int)(b >> 52) - 1023;  // s > 0: no sign bit
    if (e < -600 || e > 600) {  // |e| <= 600 keeps y0^2 and y0^3 below normal binary64 numbers
        double r = rsqrt(s);
        w3 = r * r * r;
        if (IR) ir = r;
        return;
    }
    int k = e >> 1;  // s = 2^(2k) s', s' in [1, 4)
    unsigned sb = ((unsigned)(e - 2 * k + 127) << 23) | (unsigned)((b >> 29) & 0x7fffff);
    unsigned yb = __float_as_uint(rsqrtf(__uint_as_float(sb)));  // ~ s'^(-1/2), in (0.5, 1]
    int ey = (int)(yb >> 23) - 127 - k;  // y0 = m 2^(ey - 23), m the 24-bit significand
    long long y0b = ((long long)(ey + 1023) << 52) | ((long long)(yb & 0x7fffff) << 29);
    double y0 = __longlong_as_double(y0b);  // 2^-k s'^(-1/2) ~ s^(-1/2), exactly the binary32 value
    // t = y0^2 and w0 = y0^3 rounded to nearest (what two binary64 products give) from the
    // integer significand: m^2 < 2^48 is exact, m^3 < 2^72 is rounded to 53 bits, ties to even
    unsigned long long m = (unsigned long long)((yb & 0x7fffffu) | 0x800000u);
    unsigned long long m2 = m * m;
    int h2 = (int)(m2 >> 47);  // m^2 in [2^46, 2^48): its leading bit is 46 + h2
    double t = __longlong_as_double(((long long)(2 * ey + h2 + 1023) << 52) |
                                    (long long)((m2 << (6 - h2)) & 0xfffffffffffffull));
    unsigned long long lo = m2 * m, hi = __umul64hi(m2, m);  // m^3 = hi 2^64 + lo, hi in [2^5, 2^8)
    int L = 127 - __clzll((long long)hi);                      // leading bit of m^3: 69..71
    int sh = L - 52;
    unsigned long long sig = (hi << (64 - sh)) | (lo >> sh), rem = lo & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    sig += (rem > half || (rem == half && (sig & 1ull))) ? 1ull : 0ull;
    int ew = 3 * ey - 69 + L;
    if (sig >> 53) {  // rounded up to the next power of two
        sig >>= 1;
        ew++;
    }
    double w0 = __longlong_as_double(((long long)(ew + 1023) << 52) | (long long)(sig & 0xfffffffffffffull));
    double er = fma(-s, t, 1.0);
    // the e^2 terms (below 2^-40 of the result) in binary32 from e's high word: e rebiased
    // to binary32 by integer arithmetic, two binary32 products, and the product rebiased
    // back (exact); |e| < 2^-126 leaves e^2 far below binary64 rounding and drops it
    int eh = __double2hiint(er);
    int ef = ((eh >> 20) & 0x7ff) - (1023 - 127);
    float erf = ef > 0 ? __int_as_float((eh & (int)0x80000000) | (ef << 23) | ((eh & 0xfffff) << 3)) : 0.f;
    w3 = fma(w0, fma(er, 1.5, sq_to_f64(1.875f * erf * erf)), w0);
    if (IR) ir = fma(y0, fma(er, 0.5, sq_to_f64(0.375f * erf * erf)), y0);
}


template <class S>
struct PState {
    S x, y, z, m;
};

// Leaves above 32 particles (only at the deepest level): one side at a time, lane = target
// particle, sources in increasing order.
template <class T, bool POT>
__device__ __forceinline__ void p2p_generic(int lane, bool self, int fA, int nA, int fB, int nB, long long oA,
                                            long long oB,
                                            typename Prec<T>::S rx, typename Prec<T>::S ry,
                                            typename Prec<T>::S rz,
                                            const PState<typename Prec<T>::S>* __restrict__ pos,
                                            Quad<T>* __restrict__ part) {
    using S = typename Prec<T>::S;
    for (int side = 0; side < (self ? 1 : 2); side++) {
        int fT = side ? fB : fA, nT = side ? nB : nA, fS = side ? fA : fB, nS = side ? nA : nB;
        long long oT = side ? oB : oA;
        S sx = side ? -rx : rx, sy = side ? -ry : ry, sz = side ? -rz : rz;
        for (int t = lane; t < nT; t += 32) {
            PState<S> pt = pos[fT + t];
            pt = PState<S>{sx + pt.x, sy + pt.y, sz + pt.z, pt.m};
            T ax = T(0), ay = T(0), az = T(0), ph = T(0);
            for (int u = 0; u < nS; u++) {
                if (self && u == t) continue;
                PState<S> ps = pos[fS + u];
                T dx = Prec<T>::sep(pt.x, ps.x), dy = Prec<T>::sep(pt.y, ps.y);
                T dz = Prec<T>::sep(pt.z, ps.z);
                T r2 = dx * dx + dy * dy + dz * dz;
                if (!is_zero(r2)) {
                    T ir = rsqrt_t(r2);
                    T fb = Prec<T>::mass(ps.m) * (ir * ir * ir);
                    ax = fma_t(-fb, dx, ax);
                    ay = fma_t(-fb, dy, ay);
                    az = fma_t(-fb, dz, az);
                    ph = fma_t(-Prec<T>::mass(ps.m), ir, ph);
                }
            }
            part[oT + t] = Quad<T>{Prec<T>::fin(ax), Prec<T>::fin(ay), Prec<T>::fin(az),
                                   POT ? Prec<T>::fin(ph) : T(0)};
        }
    }
}

// The pair kernel in arithmetic T over positions stored as S = Prec<T>::S.
template <class T, bool POT>
__global__ void __launch_bounds__(PB) p2p_k(int64_t npairs, const int2* __restrict__ pairs,
                                            const long long* __restrict__ pslot, const int* __restrict__ nfirst,
                                            const int* __restrict__ ncount,
                                            const PState<typename Prec<T>::S>* __restrict__ pos,
                                            const typename Prec<T>::S* __restrict__ sep,
                                            Quad<T>* __restrict__ part) {
    using S = typename Prec<T>::S;
    // panel layout and row stride: PanelRow
    constexpr int PCOL = Panel<T>::COLS;
    constexpr int PROW = PanelRow<T, POT>::ROW;
    // binary64: the masses are folded into the pair terms (FOLD)
    constexpr bool FOLD = PanelRow<T, POT>::FOLD;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ PState<S> sA[PW][32], sB[PW][32];
    __shared__ Quad<T> cacc[PW][32];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* F = reinterpret_cast<T*>(smem_raw) + (size_t)w * PanelRow<T, POT>::WARP;
    T* WA = F + 32 * PROW;    // FOLD: m_a r^-3 of the panel's pairs, [a][column]
    T* IRR = WA + 32 * PCOL;  // FOLD with potentials: r^-1, [a][column]
    T* cac = reinterpret_cast<T*>(&cacc[w][0]);
    int64_t gw = (int64_t)blockIdx.x * PW + w, nw = (int64_t)gridDim.x * PW;
    for (int64_t k = gw; k < npairs; k += nw) {
        int2 pr = pairs[k];
        int A = pr.x, B = pr.y;
        int nA = ncount[A], nB = ncount[B], fA = nfirst[A], fB = nfirst[B];
        bool self = A == B;
        long long oA = pslot[2 * k], oB = self ? 0 : pslot[2 * k + 1];  // first slots of A's and B's partials
        // positions are stored relative to their leaf's centre; the pair's centre
        // separation R = Z_A - Z_B (formed in binary64 by p2p_sep_k) is folded into the A side
        S rx = sep[3 * k], ry = sep[3 * k + 1], rz = sep[3 * k + 2];
        if (nA <= 32 && nB <= 32) {
            if (lane < nA) {
                PState<S> q = pos[fA + lane];
                sA[w][lane] = PState<S>{rx + q.x, ry + q.y, rz + q.z, q.m};
            }
            if (lane < nB) sB[w][lane] = pos[fB + lane];
            cacc[w][lane] = Quad<T>{T(0), T(0), T(0), T(0)};
            // row task tau = lane + 32 q: (a, comp) = (tau / NC, tau % NC), NC = 4 with potentials, else 3
            constexpr int NC = POT ? 4 : 3;
            T racc[NC] = {};
            __syncwarp();
            // binary64: the width from the lane-round model; double-float keeps the full width
            // (its pair terms cost several times the binary64 ones, which the model does not weigh)
            const int pcol = std::is_same<T, double>::value ? panel_cols<NC>(nA, nB, PCOL) : PCOL;
            for (int cb = 0; cb < nB; cb += pcol) {
                int ncol = min(pcol, nB - cb);
                int nint = nA * ncol;
                float rcol = 1.0f / (float)ncol;
                // pair terms of the panel: d = X_a - X_b (formed in the storage type), r^-1, d r^-3
                for (int t = lane; t < nint; t += 32) {
                    int a = __float2int_rz(((float)t + 0.5f) * rcol);  // t / ncol, exact for t < 2^12
                    int bl = t - a * ncol, b = cb + bl;
                    T fx = T(0), fy = T(0), fz = T(0), fr = T(0), fa = T(0);
                    if (!self || a < b) {
                        const PState<S>& pa = sA[w][a];
                        const PState<S>& pb = sB[w][b];
                        T dx = Prec<T>::sep(pa.x, pb.x), dy = Prec<T>::sep(pa.y, pb.y);
                        T dz = Prec<T>::sep(pa.z, pb.z);
                        T r2 = dx * dx + dy * dy + dz * dz;
                        if constexpr (FOLD) {
                            // the panel keeps d and m_b r^-3 (rows), WA m_a r^-3 (columns): two
                            // products per pair instead of the three of d r^-3
                            fx = dx;
                            fy = dy;
                            fz = dz;
                            if (!r2_zero(r2)) {
                                double w3, ir = 0.0;
                                rinv_f64<POT>(r2, w3, ir);
                                fr = pb.m * w3;
                                fa = pa.m * w3;
                                if (POT) IRR[a * PCOL + bl] = ir;
                            } else if (POT) {
                                IRR[a * PCOL + bl] = 0.0;
                            }
                        } else if (!r2_zero(r2)) {
                            T ir = rsqrt_t(r2);
                            T ir3 = ir * ir * ir;
                            fx = dx * ir3;
                            fy = dy * ir3;
                            fz = dz * ir3;
                            fr = ir;
                        }
                    } else if constexpr (FOLD && POT) {
                        IRR[a * PCOL + bl] = 0.0;
                    }
                    T* e = F + a * PROW + bl * 4;
                    e[0] = fx;
                    e[1] = fy;
                    e[2] = fz;
                    if (POT || FOLD) e[3] = fr;
                    if constexpr (FOLD) WA[a * PCOL + bl] = fa;
                }
                __syncwarp();
                // rows: sum_b m_b F[a][b], one lane per (a, component), NC nA tasks
#pragma unroll
                for (int q = 0; q < NC; q++) {
                    if (32 * q >= NC * nA) break;
                    int tau = lane + 32 * q, a = tau / NC, c = tau - a * NC;
                    if (a < nA) {
                        const T* row = F + a * PROW + c;
                        T sum = racc[q];
                        if constexpr (FOLD) {
                            // m_b r^-3 d_c, or m_b r^-1 for the potential (c = 3)
                            const T* wv = c < 3 ? F + a * PROW + 3 : &sB[w][cb].m;
                            const T* vv = c < 3 ? row : IRR + a * PCOL;
                            int vs = c < 3 ? 4 : 1;
                            for (int bl = 0; bl < ncol; bl++) sum = fma_t(wv[bl * 4], vv[bl * vs], sum);
                        } else {
                            for (int bl = 0; bl < ncol; bl++)
                                sum = fma_t(Prec<T>::mass(sB[w][cb + bl].m), row[bl * 4], sum);
                        }
                        racc[q] = sum;
                    }
                }
                // columns: sum_a m_a F[a][b], one lane per (b, component), NC ncol tasks
                for (int tau = lane; tau < NC * ncol; tau += 32) {
                    int bl = tau / NC, c = tau - bl * NC;
                    {
                        const T* col = F + bl * 4 + c;
                        T sum = cac[(cb + bl) * 4 + c];
                        if constexpr (FOLD) {
                            // m_a r^-3 d_c, or m_a r^-1 for the potential (c = 3)
                            const T* wv = c < 3 ? WA + bl : &sA[w][0].m;
                            const T* vv = c < 3 ? col : IRR + bl;
                            int ws = c < 3 ? PCOL : 4, vs = c < 3 ? PROW : PCOL;
                            for (int a = 0; a < nA; a++) sum = fma_t(wv[a * ws], vv[a * vs], sum);
                        } else {
                            for (int a = 0; a < nA; a++) sum = fma_t(Prec<T>::mass(sA[w][a].m), col[a * PROW], sum);
                        }
                        cac[(cb + bl) * 4 + c] = sum;
                    }
                }
                __syncwarp();
            }
            // write: rows are a_a = -sum (and phi_a = -sum); columns a_b = +sum, phi_b = -sum
            T* pd = reinterpret_cast<T*>(part);
#pragma unroll
            for (int q = 0; q < NC; q++) {
                int tau = lane + 32 * q, a = tau / NC, c = tau - a * NC;
                if (a < nA) {
                    T v = -racc[q];
                    if (self) v = v + ((c < 3) ? cac[a * 4 + c] : -cac[a * 4 + c]);
                    pd[(oA + a) * 4 + c] = Prec<T>::fin(v);
                    if (!POT && c == 2) pd[(oA + a) * 4 + 3] = T(0);
                }
            }
            if (!self) {
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    int tau = lane + 32 * q, b = tau >> 2, c = tau & 3;
                    if (b < nB) {
                        T v = cac[b * 4 + c];
                        pd[(oB + b) * 4 + c] = (c < 3) ? Prec<T>::fin(v) : (POT ? Prec<T>::fin(-v) : T(0));
                    }
                }
            }
            __syncwarp();
        } else {
            p2p_generic<T, POT>(lane, self, fA, nA, fB, nB, oA, oB, rx, ry, rz, pos, part);
        }
    }
}

// Ring classes.  A leaf pair with both leaves of at most 32 particles runs as a ring over
// its smaller leaf: w = min(nA, nB) slots (a self pair: w = nA), while the larger leaf
// passes through the ring in m = ceil(max(nA, nB) / w) chunks of at most w particles.  The
// pairs are ordered by the key (w - 1) * 32 + (m - 1) (pairs with a larger leaf take
// RING_BIG), stably, so the order is fixed by the list; a warp then carries 32 / w
// segments of one width with similar chunk counts.  A ring over the larger leaf would
// leave nA nB / max(nA, nB)^2 of its lane steps busy, about half for Plummer leaves.
constexpr int RING_BIG = 32 * 32;
constexpr int RING_KEY_BITS = 11;

struct RingTab {
    int start[34];  // first list index of width w = 1..32; [33]: pairs with a leaf above 32
    int count[34];  // pairs of width w
    int wpre[34];   // ring warps before width w; wpre[33]: all ring warps
};

__device__ __forceinline__ unsigned ring_key(int2 p, const int* __restrict__ ncount) {
    int nA = ncount[p.x], nB = ncount[p.y];
    if (nA > 32 || nB > 32) return RING_BIG;
    if (p.x == p.y) return (unsigned)(nA - 1) * 32u;
    int w = min(nA, nB), g = max(nA, nB);
    return (unsigned)(w - 1) * 32u + (unsigned)((g + w - 1) / w - 1);
}

// class of a key: the width w (1..32), or 33 for RING_BIG
__device__ __forceinline__ int ring_cls(uint64_t key) { return (int)(key >> 5) + 1; }

__global__ void p2p_ring_key_k(int64_t n, const int2* __restrict__ pairs, const int* __restrict__ ncount,
                               uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    int64_t k = (int64_t)blockIdx.x * PB + threadIdx.x;
    if (k >= n) return;
    keys[k] = ring_key(pairs[k], ncount);
    vals[k] = (uint32_t)k;
}

// first index and one-past-last index of every class present in the sorted keys (the
// table was set to -1 before)
__global__ void p2p_ring_bounds_k(int64_t n, const uint64_t* __restrict__ keys, RingTab* __restrict__ tab) {
    int64_t k = (int64_t)blockIdx.x * PB + threadIdx.x;
    if (k >= n) return;
    int c = ring_cls(keys[k]);
    if (k == 0 || ring_cls(keys[k - 1]) != c) tab->start[c] = (int)k;
    if (k == n - 1 || ring_cls(keys[k + 1]) != c) tab->count[c] = (int)(k + 1);
}

__global__ void p2p_ring_tab_k(RingTab* __restrict__ tab) {
    int wp = 0;
    for (int c = 1; c <= 33; c++) {
        int st = tab->start[c];
        int cnt = st < 0 ? 0 : tab->count[c] - st;
        tab->start[c] = st < 0 ? 0 : st;
        tab->count[c] = cnt;
        tab->wpre[c] = wp;
        if (c <= 32) {
            int per = 32 / c;
            wp += (cnt + per - 1) / per;
        }
    }
    tab->start[0] = tab->count[0] = tab->wpre[0] = 0;
}

// Everything the ring kernel needs of one leaf pair, in class order, as 64 aligned bytes:
// the lane leaf L (the larger one, A on a tie and for a self pair) and the ring leaf R,
// their first particles, L's count, both partial slots, and the centre separation
// Z_L - Z_R as double-float words.  A segment lane then waits for one load before it
// fetches particles, instead of the chain list -> pair -> leaf tables.
struct __align__(32) RingDesc {
    int fL, fR, nL, self;
    long long oL, oR;
    float rxh, rxl, ryh, ryl;
    float rzh, rzl, pad0, pad1;
};
static_assert(sizeof(RingDesc) == 64, "RingDesc: two 32-byte sectors");

// One thread per pair in class order: the ring descriptors, and the centre separation of
// the pairs with a leaf above 32 particles (class 33, read by p2p_big_k at 3k).  The
// separation is formed in binary64 and rounded to double-float words, as p2p_sep_k does;
// a lane leaf B takes Z_B - Z_A, the exact negation of Z_A - Z_B.
__global__ void p2p_ring_desc_k(int64_t n, const uint64_t* __restrict__ keys, const uint32_t* __restrict__ list,
                                const int2* __restrict__ pairs, const long long* __restrict__ pslot,
                                const int* __restrict__ nfirst, const int* __restrict__ ncount,
                                const double* __restrict__ Zx, const double* __restrict__ Zy,
                                const double* __restrict__ Zz, RingDesc* __restrict__ desc, df64* __restrict__ sep) {
    int64_t li = (int64_t)blockIdx.x * PB + threadIdx.x;
    if (li >= n) return;
    int k = (int)list[li];
    int2 p = pairs[k];
    double dx = Zx[p.x] - Zx[p.y], dy = Zy[p.x] - Zy[p.y], dz = Zz[p.x] - Zz[p.y];
    if (ring_cls(keys[li]) > 32) {
        sep[3 * k] = to_df(dx);
        sep[3 * k + 1] = to_df(dy);
        sep[3 * k + 2] = to_df(dz);
        return;
    }
    bool self = p.x == p.y;
    int nA = ncount[p.x], nB = ncount[p.y];
    bool laneA = nA >= nB;
    int L = laneA ? p.x : p.y, R = laneA ? p.y : p.x;
    long long oA = pslot[2 * k], oB = self ? 0 : pslot[2 * k + 1];
    if (!laneA) {
        dx = -dx;
        dy = -dy;
        dz = -dz;
    }
    df64 rx = to_df(dx), ry = to_df(dy), rz = to_df(dz);
    RingDesc d;
    d.fL = nfirst[L];
    d.fR = nfirst[R];
    d.nL = laneA ? nA : nB;
    d.self = self ? 1 : 0;
    d.oL = laneA ? oA : oB;
    d.oR = laneA ? oB : oA;
    d.rxh = rx.hi;
    d.rxl = rx.lo;
    d.ryh = ry.hi;
    d.ryl = ry.lo;
    d.rzh = rz.hi;
    d.rzl = rz.lo;
    d.pad0 = d.pad1 = 0.f;
    desc[li] = d;
}

// a ring descriptor in two 32-byte loads through the non-coherent path
__device__ __forceinline__ RingDesc load_desc(const RingDesc* __restrict__ p) {
    RingDesc d;
    int* w = reinterpret_cast<int*>(&d);
    const int* s = reinterpret_cast<const int*>(p);
#pragma unroll
    for (int h = 0; h < 2; h++)
        asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=r"(w[8 * h]), "=r"(w[8 * h + 1]), "=r"(w[8 * h + 2]), "=r"(w[8 * h + 3]), "=r"(w[8 * h + 4]),
              "=r"(w[8 * h + 5]), "=r"(w[8 * h + 6]), "=r"(w[8 * h + 7])
            : "l"(s + 8 * h));
    return d;
}

// one ring step of a lane particle a with ring particle b, positions as double-float words
// (hi, lo) in binary32 arithmetic: the pair force is formed once, -m_b d r^-3 goes to a's
// sum and +m_a d r^-3 to b's travelling sum (potentials -m r^-1); r = 0 adds nothing.
// The separation is (hi - hi) + (lo - lo), exact in its high difference for close pairs.
template <bool POT>
__device__ __forceinline__ void ring_pair(const float4& ah, const float4& al, float ma, const float4& bh,
                                          const float4& bl, float4& a, float& bx, float& by, float& bz, float& bp) {
    float dx = __fadd_rn(__fsub_rn(ah.x, bh.x), __fsub_rn(al.x, bl.x));
    float dy = __fadd_rn(__fsub_rn(ah.y, bh.y), __fsub_rn(al.y, bl.y));
    float dz = __fadd_rn(__fsub_rn(ah.z, bh.z), __fsub_rn(al.z, bl.z));
    float r2 = dx * dx + dy * dy + dz * dz;
    if (r2 != 0.f) {
        float ir = rsqrtf(r2);
        float ir3 = ir * ir * ir;
        float mb = bh.w;
        float sa = mb * ir3;
        a.x = fmaf(-sa, dx, a.x);
        a.y = fmaf(-sa, dy, a.y);
        a.z = fmaf(-sa, dz, a.z);
        if (POT) a.w = fmaf(-mb, ir, a.w);
        float sb = ma * ir3;
        bx = fmaf(sb, dx, bx);
        by = fmaf(sb, dy, by);
        bz = fmaf(sb, dz, bz);
        if (POT) bp = fmaf(-ma, ir, bp);
    }
}

// a double-float particle (32 bytes at a 16-byte aligned address in the packed array) in
// two 16-byte loads; the struct alone promises 4 bytes
__device__ __forceinline__ PState<df64> ld_pstate_g(const PState<df64>* __restrict__ p) {
    const float4* v = reinterpret_cast<const float4*>(p);
    float4 u = __ldg(v), t = __ldg(v + 1);
    return PState<df64>{df64(u.x, u.y), df64(u.z, u.w), df64(t.x, t.y), df64(t.z, t.w)};
}
// one binary32 partial (16 bytes, 16-byte aligned in the partial buffer) in one store
__device__ __forceinline__ void st_quad(Quad<float>* p, float x, float y, float z, float w) {
    *reinterpret_cast<float4*>(p) = make_float4(x, y, z, w);
}

// lane particles held at once by a ring lane (chunks of the lane leaf per pass)
constexpr int RING_CHUNKS = 2;

// The binary32 ring pair kernel for leaves of at most 32 particles.  A warp takes 32 / w
// segments of w lanes, one leaf pair each.  Lane i of a segment holds particle
// g = c w + i of the larger ("lane") leaf in chunk c, shifted by that leaf's side of
// R = Z_A - Z_B; the smaller ("ring") leaf sits in shared memory as two float4 arrays
// (high words and mass, low words), so that a quarter-warp's 16-byte reads are
// contiguous, each stored twice in a row so that the ring index never wraps.  A lane holds RING_CHUNKS chunks at a time: every ring particle read meets
// all of them.  In step k lane i meets ring particle j = (i + k) mod w: over w steps
// every (g, j) of the chunks meets exactly once.  The pair force is formed once and
// applied to both partners: g's sum stays in lane i and is stored after its chunk, j's
// sum travels with the ring (one shuffle from lane i + 1 per step), is back in lane j
// after every full turn and collects all chunks before it is stored.  A self pair runs
// one chunk over itself from both ends (each pair twice, 1/w of the work, no reduction)
// and drops the travelling sums.  Every sum runs in a fixed order.
// Eight blocks per SM (64 registers): 28 -> 32 warps per SM took 10% off the binary32
// P2P; 48 registers spilled into the ring loop and lost it again.
template <bool POT>
__global__ void __launch_bounds__(PB, 8) p2p_ring_k(const RingTab* __restrict__ tab, const RingDesc* __restrict__ desc,
                                                 const PState<df64>* __restrict__ pos, Quad<float>* __restrict__ part) {
    // the ring leaf twice in a row per segment (slots 0..w-1, 0..w-1): lane i reads slot
    // i + k without wrapping, at a fixed stride from one pointer
    __shared__ float4 sH[PW][64], sL[PW][64];
    __shared__ int ts[34], tc[34], tw[34];
    for (int t = threadIdx.x; t < 34; t += PB) {
        ts[t] = tab->start[t];
        tc[t] = tab->count[t];
        tw[t] = tab->wpre[t];
    }
    __syncthreads();
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t gw = (int64_t)blockIdx.x * PW + w, nw = (int64_t)gridDim.x * PW;
    int64_t total = tw[33];
    for (int64_t q = gw; q < total; q += nw) {
        // the width of this warp: the largest W with tw[W] <= q (tw is nondecreasing)
        int W = 1;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
            if (W + step <= 32 && tw[W + step] <= q) W += step;
        int per = 32 / W;
        int sg = lane / W;
        bool live = sg < per;
        // a lane past the last segment reads segment 0's rows (in bounds, unused)
        int i = live ? lane - sg * W : 0, base = live ? sg * W : 0;
        int64_t li = (q - tw[W]) * per + sg;
        bool ok = live && li < tc[W];
        // one descriptor load, then the particles (the chain list -> pair -> leaf tables
        // is resolved once per evaluation by p2p_ring_desc_k)
        RingDesc d{};
        if (ok) d = load_desc(desc + ts[W] + li);
        bool self = d.self != 0;
        int fL = d.fL, nL = d.nL;
        long long oL = d.oL, oR = d.oR;
        df64 rx(d.rxh, d.rxl), ry(d.ryh, d.ryl), rz(d.rzh, d.rzl);
        PState<df64> rb{};
        if (ok) rb = ld_pstate_g(pos + d.fR + i);  // i < W = the ring leaf's count
        __syncwarp();
        if (ok) {  // the segment's rows are [2 base, 2 base + 2 W)
            float4 h = make_float4(rb.x.hi, rb.y.hi, rb.z.hi, rb.m.hi), lo = make_float4(rb.x.lo, rb.y.lo, rb.z.lo, 0.f);
            sH[w][2 * base + i] = h;
            sH[w][2 * base + W + i] = h;
            sL[w][2 * base + i] = lo;
            sL[w][2 * base + W + i] = lo;
        }
        __syncwarp();
        int m = ok ? (self ? 1 : (nL + W - 1) / W) : 0;
        int mmax = __reduce_max_sync(FULL, m);
        int nxt = live ? base + (i + 1 < W ? i + 1 : 0) : lane;
        float bx = 0.f, by = 0.f, bz = 0.f, bp = 0.f;
        for (int ch = 0; ch < mmax; ch += RING_CHUNKS) {
            float4 ah[RING_CHUNKS], al[RING_CHUNKS], acc[RING_CHUNKS];
            float ma[RING_CHUNKS];
            bool mine[RING_CHUNKS];
#pragma unroll
            for (int r = 0; r < RING_CHUNKS; r++) {
                int g = (ch + r) * W + i;
                mine[r] = ok && ch + r < m && g < nL;
                ah[r] = al[r] = acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
                ma[r] = 0.f;
                if (mine[r]) {
                    PState<df64> qa = ld_pstate_g(pos + fL + g);
                    df64 x = rx + qa.x, y = ry + qa.y, z = rz + qa.z;
                    ah[r] = make_float4(x.hi, y.hi, z.hi, 0.f);
                    al[r] = make_float4(x.lo, y.lo, z.lo, 0.f);
                    ma[r] = qa.m.hi;
                }
            }
            const float4* rh = &sH[w][2 * base + i];  // slot i + kk for kk < W: row < 2 base + 2 W <= 64
            const float4* rl = &sL[w][2 * base + i];
            // one turn of the ring; a warp whose lanes hold no second chunk (equal leaves,
            // self pairs, the last pass of an odd chunk count) runs the one-chunk form
            auto turn = [&](auto both) {
#pragma unroll 4
                for (int kk = 0; kk < W; kk++) {
                    float4 bh = rh[kk], bl = rl[kk];
                    if (mine[0]) ring_pair<POT>(ah[0], al[0], ma[0], bh, bl, acc[0], bx, by, bz, bp);
                    if constexpr (decltype(both)::value)
                        if (mine[1]) ring_pair<POT>(ah[1], al[1], ma[1], bh, bl, acc[1], bx, by, bz, bp);
                    bx = __shfl_sync(FULL, bx, nxt);
                    by = __shfl_sync(FULL, by, nxt);
                    bz = __shfl_sync(FULL, bz, nxt);
                    if (POT) bp = __shfl_sync(FULL, bp, nxt);
                }
            };
            static_assert(RING_CHUNKS == 2, "the ring turn is written for two chunks");
            if (__any_sync(FULL, mine[1]))
                turn(std::true_type{});
            else
                turn(std::false_type{});
#pragma unroll
            for (int r = 0; r < RING_CHUNKS; r++)
                if (mine[r]) st_quad(part + oL + (ch + r) * W + i, acc[r].x, acc[r].y, acc[r].z, POT ? acc[r].w : 0.f);
        }
        if (ok && !self) st_quad(part + oR + i, bx, by, bz, POT ? bp : 0.f);
        __syncwarp();
    }
}

// pairs with a leaf above 32 particles (only at the deepest level), from the end of the
// sorted list
template <class T, bool POT>
__global__ void __launch_bounds__(PB) p2p_big_k(const RingTab* __restrict__ tab, const uint32_t* __restrict__ list,
                                                const int2* __restrict__ pairs, const long long* __restrict__ pslot,
                                                const int* __restrict__ nfirst, const int* __restrict__ ncount,
                                                const PState<typename Prec<T>::S>* __restrict__ pos,
                                                const typename Prec<T>::S* __restrict__ sep,
                                                Quad<T>* __restrict__ part) {
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t gw = (int64_t)blockIdx.x * PW + w, nw = (int64_t)gridDim.x * PW;
    int64_t first = tab->start[33], nlist = tab->count[33];
    for (int64_t li = gw; li < nlist; li += nw) {
        int k = (int)list[first + li];
        int2 pr = pairs[k];
        bool self = pr.x == pr.y;
        p2p_generic<T, POT>(lane, self, nfirst[pr.x], ncount[pr.x], nfirst[pr.y], ncount[pr.y], pslot[2 * k],
                            self ? 0 : pslot[2 * k + 1],
                            sep[3 * k], sep[3 * k + 1], sep[3 * k + 2], pos, part);
    }
}

// centre separation Z_A - Z_B of every P2P pair, formed in binary64 once per pair and
// stored in the storage type (one thread per pair: the pair kernel's lanes would all
// repeat this binary64 work)
template <class S>
__global__ void p2p_sep_k(int64_t npairs, const int2* __restrict__ pairs, const double* __restrict__ Zx,
                          const double* __restrict__ Zy, const double* __restrict__ Zz, S* __restrict__ sep) {
    int64_t k = (int64_t)blockIdx.x * PB + threadIdx.x;
    if (k >= npairs) return;
    int2 p = pairs[k];
    sep[3 * k] = to_storage(Zx[p.x] - Zx[p.y], S());
    sep[3 * k + 1] = to_storage(Zy[p.x] - Zy[p.y], S());
    sep[3 * k + 2] = to_storage(Zz[p.x] - Zz[p.y], S());
}

// packed (x - Z_leaf, y - Z_leaf, z - Z_leaf, m) of every sorted particle in the storage
// type S: offsets from the leaf centre keep double-float positions accurate to ~2^-48 of
// the leaf size rather than of the coordinate
template <class S>
__global__ void pack_pos_k(int n, const int* __restrict__ leaf_of, const double* __restrict__ xs,
                           const double* __restrict__ ys, const double* __restrict__ zs,
                           const double* __restrict__ ms, const double* __restrict__ Zx,
                           const double* __restrict__ Zy, const double* __restrict__ Zz, PState<S>* __restrict__ pos) {
    int i = blockIdx.x * PB + threadIdx.x;
    if (i < n) {
        int l = leaf_of[i];
        pos[i] = PState<S>{to_storage(xs[i] - Zx[l], S()), to_storage(ys[i] - Zy[l], S()),
                           to_storage(zs[i] - Zz[l], S()), to_storage(ms[i], S())};
    }
}

// which pair kernel each arithmetic runs (ring: binary32; panel: binary64 and double-float)
template <class T>
struct P2PRing {
    static constexpr bool value = std::is_same<T, float>::value;
};

// P2P set-up: packed positions, ring classes (binary32), the partial buffer (its size read
// once per walk) and the pairs' centre separations
template <class T>
static void p2p_prepare(fmm_ctx* c) {
    using S = typename Prec<T>::S;
    cudaStream_t s = c->stream;
    int n = (int)c->N;
    if (!c->pos_valid) {
        ensure(c->pos4, sizeof(PState<S>) * (size_t)n);
        pack_pos_k<S><<<grid_for(n, PB), PB, 0, s>>>(n, c->leaf_of.as<int>(), c->xs.as<double>(), c->ys.as<double>(),
                                                   c->zs.as<double>(), c->ms.as<double>(), c->nZx.as<double>(),
                                                   c->nZy.as<double>(), c->nZz.as<double>(), c->pos4.as<PState<S>>());
        GB_LAUNCH("pack_pos_k");
        c->pos_valid = true;
    }
    if constexpr (P2PRing<T>::value) {
        int64_t np = c->n_p2p;
        if (c->p2p_cls_gen != c->walk_gen && np > 0) {
            // ring classes of the leaf pairs: list bookkeeping, once per walk
            ensure(c->p2p_cls, sizeof(uint64_t) * (size_t)np);
            ensure(c->p2p_list, sizeof(uint32_t) * (size_t)np);
            ensure(c->p2p_tab, sizeof(RingTab));
            p2p_ring_key_k<<<grid_for(np, PB), PB, 0, s>>>(np, c->p2p_pairs.as<int2>(), c->ncount.as<int>(),
                                                          c->p2p_cls.as<uint64_t>(), c->p2p_list.as<uint32_t>());
            GB_LAUNCH("p2p_ring_key_k");
            radix_sort(c, c->p2p_cls, c->p2p_cls2, &c->p2p_list, &c->p2p_list2, np, RING_KEY_BITS);
            RingTab* tab = c->p2p_tab.as<RingTab>();
            GB_CUDA(cudaMemsetAsync(tab, 0xFF, sizeof(RingTab), s));
            p2p_ring_bounds_k<<<grid_for(np, PB), PB, 0, s>>>(np, c->p2p_cls.as<uint64_t>(), tab);
            GB_LAUNCH("p2p_ring_bounds_k");
            p2p_ring_tab_k<<<1, 1, 0, s>>>(tab);
            GB_LAUNCH("p2p_ring_tab_k");
            c->p2p_cls_gen = c->walk_gen;
        }
    }
    // partial slots of the walk's pairs: read once per walk (with the flag of the ring
    // class sort above), so that later evaluations on the same lists never wait on the host
    if (c->p2p_total_gen != c->walk_gen) {
        HostReads hr(c);
        const long long* total = hr.read<long long>(c->p2p_pbase.as<long long>() + c->n_nodes);
        const int* serr = hr.read<int>(sort_err(c));
        hr.wait();
        sort_err_throw(c, *serr);
        c->p2p_total = *total;
        c->p2p_total_gen = c->walk_gen;
    }
    long long total = c->p2p_total;
    ensure(c->p2p_part, sizeof(Quad<T>) * (size_t)(total > 0 ? total : 1));
    ensure(c->p2p_sep, sizeof(S) * 3 * (size_t)(c->n_p2p > 0 ? c->n_p2p : 1));
    if constexpr (P2PRing<T>::value) {
        // ring descriptors in class order (and the separations of the few large-leaf pairs)
        int64_t np = c->n_p2p;
        ensure(c->p2p_desc, sizeof(RingDesc) * (size_t)(np > 0 ? np : 1));
        if (np > 0) {
            p2p_ring_desc_k<<<grid_for(np, PB), PB, 0, s>>>(
                np, c->p2p_cls.as<uint64_t>(), c->p2p_list.as<uint32_t>(), c->p2p_pairs.as<int2>(),
                c->p2p_off.as<long long>(), c->nfirst.as<int>(), c->ncount.as<int>(), c->nZx.as<double>(),
                c->nZy.as<double>(), c->nZz.as<double>(), c->p2p_desc.as<RingDesc>(), c->p2p_sep.as<df64>());
            GB_LAUNCH("p2p_ring_desc_k");
        }
    } else {
        p2p_sep_k<S><<<grid_for(c->n_p2p, PB), PB, 0, s>>>(c->n_p2p, c->p2p_pairs.as<int2>(), c->nZx.as<double>(),
                                                         c->nZy.as<double>(), c->nZz.as<double>(), c->p2p_sep.as<S>());
        GB_LAUNCH("p2p_sep_k");
    }
}

// the pair kernels on the prepared lists (no host read, no allocation)
template <class T>
static void p2p_kernels(fmm_ctx* c, bool want_pot) {
    using S = typename Prec<T>::S;
    cudaStream_t s = c->stream;
    int dev_sms = 0;
    GB_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c->device));
    int64_t blocks = (c->n_p2p + PW - 1) / PW;
    int64_t cap = (int64_t)dev_sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    stage_begin(c, ST_P2P);
    if constexpr (P2PRing<T>::value) {
        int64_t np = c->n_p2p;
        if (np > 0) {
            const RingTab* tab = c->p2p_tab.as<RingTab>();
            const uint32_t* lst = c->p2p_list.as<uint32_t>();
            const RingDesc* dsc = c->p2p_desc.as<RingDesc>();
            auto ring = [&](auto kern, int64_t bl) {
                kern<<<(unsigned)bl, PB, 0, s>>>(tab, dsc, c->pos4.as<PState<S>>(), c->p2p_part.as<Quad<T>>());
            };
            auto big = [&](auto kern, int64_t bl) {
                kern<<<(unsigned)bl, PB, 0, s>>>(tab, lst, c->p2p_pairs.as<int2>(), c->p2p_off.as<long long>(),
                                                 c->nfirst.as<int>(), c->ncount.as<int>(), c->pos4.as<PState<S>>(),
                                                 c->p2p_sep.as<S>(), c->p2p_part.as<Quad<T>>());
            };
            // the warp counts live on the device: persistent grids, warps stride over the work
            int64_t ring_bl = (np + PW - 1) / PW;
            if (ring_bl > cap) ring_bl = cap;
            if (want_pot) {
                ring(p2p_ring_k<true>, ring_bl);
                GB_LAUNCH("p2p_ring_k");
                big(p2p_big_k<T, true>, dev_sms);
                GB_LAUNCH("p2p_big_k");
            } else {
                ring(p2p_ring_k<false>, ring_bl);
                GB_LAUNCH("p2p_ring_k");
                big(p2p_big_k<T, false>, dev_sms);
                GB_LAUNCH("p2p_big_k");
            }
        }
    } else {
        size_t shm = sizeof(T) * (size_t)(want_pot ? PanelRow<T, true>::WARP : PanelRow<T, false>::WARP) * PW;
        auto kern = want_pot ? p2p_k<T, true> : p2p_k<T, false>;
        GB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        kern<<<(unsigned)blocks, PB, shm, s>>>(c->n_p2p, c->p2p_pairs.as<int2>(), c->p2p_off.as<long long>(),
                                               c->nfirst.as<int>(), c->ncount.as<int>(), c->pos4.as<PState<S>>(),
                                               c->p2p_sep.as<S>(), c->p2p_part.as<Quad<T>>());
        GB_LAUNCH("p2p_k");
    }
    stage_end(c, ST_P2P);
}

void fused_p2p_launch(fmm_ctx* c, bool want_pot, double theta, Quad<double>* out);

// the fused schedule's near field (binary64): pack the leaf-relative positions, then one
// traversal per target leaf writes the leaf's per-particle P2P sums to p2p_direct
void run_p2p_fused(fmm_ctx* c, bool want_pot, double theta) {
    cudaStream_t s = c->stream;
    int n = (int)c->N;
    if (!c->pos_valid) {
        ensure(c->pos4, sizeof(PState<double>) * (size_t)n);
        pack_pos_k<double><<<grid_for(n, PB), PB, 0, s>>>(n, c->leaf_of.as<int>(), c->xs.as<double>(),
                                                        c->ys.as<double>(), c->zs.as<double>(), c->ms.as<double>(),
                                                        c->nZx.as<double>(), c->nZy.as<double>(), c->nZz.as<double>(),
                                                        c->pos4.as<PState<double>>());
        GB_LAUNCH("pack_pos_k");
        c->pos_valid = true;
    }
    ensure(c->p2p_direct, sizeof(Quad<double>) * (size_t)n);
    fused_p2p_launch(c, want_pot, theta, c->p2p_direct.as<Quad<double>>());
}

void run_p2p_prepare(fmm_ctx* c) {
    if (c->precision == FMM_FP64)
        p2p_prepare<double>(c);
    else if (c->precision == FMM_DF64)
        p2p_prepare<df64>(c);
    else
        p2p_prepare<float>(c);
}

void run_p2p_kernels(fmm_ctx* c, bool want_pot) {
    if (c->precision == FMM_FP64)
        p2p_kernels<double>(c, want_pot);
    else if (c->precision == FMM_DF64)
        p2p_kernels<df64>(c, want_pot);
    else
        p2p_kernels<float>(c, want_pot);
}

void run_p2p(fmm_ctx* c, bool want_pot) {
    run_p2p_prepare(c);
    run_p2p_kernels(c, want_pot);
}

// a12/a13 first level: one warp per P2P work item (up to P2P_CHUNK directed entries of
// one leaf).  Sums the per-pair partials of the item's entries into
// ipart[islot[item] + slot].  A leaf of cnt <= 32 particles uses 32 / cnt lane groups of
// cnt lanes (lane = particle slot): group g sums entries g, g + groups, ... in list order,
// and the group sums are added in group order, so the sum runs in one fixed order while
// most lanes work (leaves hold ~9 particles; one lane per slot left two thirds of the
// warp idle, and idle lanes cost full binary64 issue).  Larger leaves take one entry
// stream per slot.
//   part[] holds (ax, ay, az, phi) per (directed entry, slot), in target-segment order:
//   target t's entries own consecutive runs of count[t] slots from tbase[t] on, so an
//   item's partials are one contiguous run; the pair kernels write pair k's two sides at
//   pslot[2k], pslot[2k + 1].
// acc + v for the item sums: binary64 and double-float partials add as usual; a binary32
// partial is added to the double-float sum by TwoSum on the high word with the rounding
// error gathered in the low word (left unnormalised until the end: a few dozen terms keep
// it far inside the high word's last bits)
__device__ __forceinline__ double acc_add(double acc, double v) { return acc + v; }
__device__ __forceinline__ df64 acc_add(df64 acc, df64 v) { return acc + v; }
__device__ __forceinline__ df64 acc_add(df64 acc, float v) {
    df64 t = two_sum(acc.hi, v);
    return df64(t.hi, __fadd_rn(acc.lo, t.lo));
}
__device__ __forceinline__ double acc_fin(double a) { return a; }
__device__ __forceinline__ df64 acc_fin(df64 a) { return fast_two_sum(a.hi, a.lo); }

__device__ __forceinline__ double shfl_g(double v, int src) { return __shfl_sync(FULL, v, src); }
__device__ __forceinline__ df64 shfl_g(df64 v, int src) {
    return df64(__shfl_sync(FULL, v.hi, src), __shfl_sync(FULL, v.lo, src));
}

// sum of the partials of entries e0, e0 + step, ... < e1 for one slot, four in flight; the
// entries' slot runs are consecutive (cnt slots each), entry e0's starting at b0
// One partial in one load: the partial buffer holds 16-byte (binary32) or 32-byte
// (binary64, double-float) records from an aligned base, written by an earlier kernel.
// The records' own types promise only the alignment of their words, and four word
// loads per record cross each 32-byte sector four times.
__device__ __forceinline__ Quad<float> ld_part(const Quad<float>* __restrict__ p) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return Quad<float>{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Quad<double> ld_part(const Quad<double>* __restrict__ p) {
    Quad<double> q;
    asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(q.x), "=d"(q.y), "=d"(q.z), "=d"(q.w) : "l"(p));
    return q;
}
__device__ __forceinline__ Quad<df64> ld_part(const Quad<df64>* __restrict__ p) {
    float v[8];
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(p));
    return Quad<df64>{df64(v[0], v[1]), df64(v[2], v[3]), df64(v[4], v[5]), df64(v[6], v[7])};
}

template <class G, class PT>
__device__ __forceinline__ Quad<G> gather_run(int e0, int e1, int step, long long b0, int cnt, int slot,
                                              const Quad<PT>* __restrict__ part) {
    Quad<G> acc{G(0), G(0), G(0), G(0)};
    const Quad<PT>* p = part + b0 + slot;
    const long long stride = (long long)step * cnt;
    int e = e0;
    for (; e + 3 * step < e1; e += 4 * step, p += 4 * stride) {
        Quad<PT> q[4];
#pragma unroll
        for (int u = 0; u < 4; u++) q[u] = ld_part(p + u * stride);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            acc.x = acc_add(acc.x, q[u].x);
            acc.y = acc_add(acc.y, q[u].y);
            acc.z = acc_add(acc.z, q[u].z);
            acc.w = acc_add(acc.w, q[u].w);
        }
    }
    for (; e < e1; e += step, p += stride) {
        Quad<PT> q = ld_part(p);
        acc.x = acc_add(acc.x, q.x);
        acc.y = acc_add(acc.y, q.y);
        acc.z = acc_add(acc.z, q.z);
        acc.w = acc_add(acc.w, q.w);
    }
    return Quad<G>{acc_fin(acc.x), acc_fin(acc.y), acc_fin(acc.z), acc_fin(acc.w)};
}

template <class G, class PT>
__global__ void __launch_bounds__(PB) p2p_gather_k(int64_t nitems, const int4* __restrict__ items,
                                                   const int* __restrict__ ncount, const long long* __restrict__ seg,
                                                   const long long* __restrict__ tbase,
                                                   const Quad<PT>* __restrict__ part,
                                                   const long long* __restrict__ islot, Quad<G>* __restrict__ ipart) {
    int64_t it = ((int64_t)blockIdx.x * PB + threadIdx.x) >> 5;  // one item per warp
    int lane = threadIdx.x & 31;
    if (it >= nitems) return;
    int4 w = items[it];
    int cnt = ncount[w.x];
    long long b = tbase[w.x] + (w.y - seg[w.x]) * (long long)cnt;  // first slot of entry w.y
    if (cnt > 32) {
        for (int slot = lane; slot < cnt; slot += 32)
            ipart[islot[it] + slot] = gather_run<G, PT>(w.y, w.z, 1, b, cnt, slot, part);
        return;
    }
    int groups = 32 / cnt, grp = lane / cnt, slot = lane - grp * cnt;
    Quad<G> own{G(0), G(0), G(0), G(0)};
    if (grp < groups) own = gather_run<G, PT>(w.y + grp, w.z, groups, b + (long long)grp * cnt, cnt, slot, part);
    // group 0's lanes add the other groups' sums (read from the unchanged own values) in
    // group order
    Quad<G> acc = own;
    for (int g = 1; g < groups; g++) {
        int src = lane + g * cnt;  // < 32 for group 0's lanes
        Quad<G> o{shfl_g(own.x, src), shfl_g(own.y, src), shfl_g(own.z, src), shfl_g(own.w, src)};
        acc = Quad<G>{acc.x + o.x, acc.y + o.y, acc.z + o.z, acc.w + o.w};
    }
    if (grp == 0) ipart[islot[it] + slot] = acc;
}

// slot offsets of the P2P items: islot[i] = sum of the leaf sizes of items before i
__global__ void item_slots_k(int64_t nitems, const int4* __restrict__ items, const int* __restrict__ ncount,
                             long long* __restrict__ sizes) {
    int64_t i = (int64_t)blockIdx.x * PB + threadIdx.x;
    if (i < nitems) sizes[i] = ncount[items[i].x];
}

// item slots depend only on the lists: formed once per walk (the targets' partial bases,
// p2p_pbase, come with the lists)
static void gather_setup(fmm_ctx* c) {
    if (c->gather_gen == c->walk_gen) return;
    cudaStream_t s = c->stream;
    const ItemSet& it = c->p2p_items;
    int64_t ni = it.n_items;
    ensure(c->p2p_islot, sizeof(long long) * (size_t)(ni + 1));
    ensure(c->flags, sizeof(long long) * (size_t)(ni + 1));
    item_slots_k<<<grid_for(ni, PB), PB, 0, s>>>(ni, it.items.as<int4>(), c->ncount.as<int>(), c->flags.as<long long>());
    GB_LAUNCH("item_slots_k");
    scan_i64_from_i64(c, c->flags.as<long long>(), ni, c->p2p_islot.as<long long>());
    HostReads hr(c);
    const long long* nslots = hr.read<long long>(c->p2p_islot.as<long long>() + ni);
    const int* serr = hr.read<int>(sort_err(c));  // the ring class sort of the pair kernels' set-up
    hr.wait();
    sort_err_throw(c, *serr);
    c->p2p_nslots = *nslots;
    c->gather_gen = c->walk_gen;
}

template <class G, class PT>
static void gather_launch(fmm_ctx* c) {
    cudaStream_t s = c->stream;
    gather_setup(c);
    const ItemSet& it = c->p2p_items;
    int64_t ni = it.n_items;
    long long nslots = c->p2p_nslots;
    ensure(c->p2p_ipart, sizeof(Quad<G>) * (size_t)(nslots > 0 ? nslots : 1));
    if (ni > 0) {
        p2p_gather_k<G, PT><<<grid_for(ni * 32, PB), PB, 0, s>>>(ni, it.items.as<int4>(), c->ncount.as<int>(),
                                                                  c->p2p_seg.as<long long>(),
                                                                  c->p2p_pbase.as<long long>(),
                                                                  c->p2p_part.as<Quad<PT>>(),
                                                                  c->p2p_islot.as<long long>(),
                                                                  c->p2p_ipart.as<Quad<G>>());
        GB_LAUNCH("p2p_gather_k");
    }
}

void run_p2p_gather(fmm_ctx* c) {
    if (c->precision == FMM_FP64)
        gather_launch<double, double>(c);
    else if (c->precision == FMM_DF64)
        gather_launch<df64, df64>(c);
    else
        gather_launch<df64, float>(c);
}

// ------------------------------------------------------------------ diagnostics

constexpr int DB = 256;

__device__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = DB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// fixed-order sums of m a and m X x a over sorted particles: per-block tree, then one block
__global__ void diag_partial_k(int n, const double* __restrict__ xs, const double* __restrict__ ys,
                               const double* __restrict__ zs, const double* __restrict__ ms,
                               const double* __restrict__ acc, double* __restrict__ part) {
    __shared__ double sh[DB];
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int i = blockIdx.x * DB + threadIdx.x; i < n; i += gridDim.x * DB) {
        double m = ms[i], ax = acc[i], ay = acc[n + i], az = acc[2 * (int64_t)n + i];
        double x = xs[i], y = ys[i], z = zs[i];
        v[0] += m * ax;
        v[1] += m * ay;
        v[2] += m * az;
        v[3] += m * (y * az - z * ay);
        v[4] += m * (z * ax - x * az);
        v[5] += m * (x * ay - y * ax);
    }
    for (int d = 0; d < 6; d++) {
        double r = block_sum(v[d], sh);
        if (threadIdx.x == 0) part[6 * blockIdx.x + d] = r;
    }
}

__global__ void diag_final_k(int nb, const double* __restrict__ part, double* __restrict__ out) {
    __shared__ double sh[DB];
    for (int d = 0; d < 6; d++) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nb; b += DB) v += part[6 * b + d];
        double r = block_sum(v, sh);
        if (threadIdx.x == 0) out[d] = r;
    }
}

// per-system sums (batch): one block per system over its sorted particle range
__global__ void diag_sys_k(const long long* __restrict__ off, int n, const double* __restrict__ xs,
                           const double* __restrict__ ys, const double* __restrict__ zs, const double* __restrict__ ms,
                           const double* __restrict__ acc, double* __restrict__ out) {
    __shared__ double sh[DB];
    int sys = blockIdx.x;
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (long long i = off[sys] + threadIdx.x; i < off[sys + 1]; i += DB) {
        double m = ms[i], ax = acc[i], ay = acc[n + i], az = acc[2 * (int64_t)n + i];
        double x = xs[i], y = ys[i], z = zs[i];
        v[0] += m * ax;
        v[1] += m * ay;
        v[2] += m * az;
        v[3] += m * (y * az - z * ay);
        v[4] += m * (z * ax - x * az);
        v[5] += m * (x * ay - y * ax);
    }
    for (int d = 0; d < 6; d++) {
        double r = block_sum(v[d], sh);
        if (threadIdx.x == 0) out[6 * sys + d] = r;
    }
}

void run_diagnostics_sys(fmm_ctx* c, double* out) {
    cudaStream_t s = c->stream;
    diag_sys_k<<<c->n_sys, DB, 0, s>>>(c->sys_off.as<long long>(), (int)c->N, c->xs.as<double>(), c->ys.as<double>(),
                                       c->zs.as<double>(), c->ms.as<double>(), c->acc_s.as<double>(), out);
    GB_LAUNCH("diag_sys_k");
}

void run_diagnostics(fmm_ctx* c, double* out6) {
    cudaStream_t s = c->stream;
    int n = (int)c->N;
    int nb = (n + DB - 1) / DB;
    if (nb > 592) nb = 592;
    ensure(c->diag_tmp, sizeof(double) * (size_t)(6 * nb + 6));
    double* part = c->diag_tmp.as<double>();
    diag_partial_k<<<nb, DB, 0, s>>>(n, c->xs.as<double>(), c->ys.as<double>(), c->zs.as<double>(),
                                     c->ms.as<double>(), c->acc_s.as<double>(), part);
    GB_LAUNCH("diag_partial_k");
    diag_final_k<<<1, DB, 0, s>>>(nb, part, part + 6 * nb);
    GB_LAUNCH("diag_final_k");
    GB_CUDA(cudaMemcpyAsync(out6, part + 6 * nb, sizeof(double) * 6, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
}

// ================================================================ fused schedule
// Near field of the fused schedule (fused_traverse.cuh): P2P evaluated from every target
// leaf's own traversal, with no P2P list, partial buffer or gather (binary64).

// ---------------------------------------------------------------- near field

template <bool POT>
struct NearVisitor {
    const NodeView* nv;
    const PState<double>* pos;
    int T, fT, nT, a, grp, ngrp;
    bool live;
    double ax, ay, az, ph;

    __device__ void m2l(int) {}
    __device__ void p2p(int Y) {
        if (!live) return;
        bool self = Y == T;
        int fY = nv->first[Y], nY = nv->count[Y];
        // T's particle with its side of R = Z_T - Z_Y, as the list schedule's panel forms it
        double rx = nv->Zx[T] - nv->Zx[Y], ry = nv->Zy[T] - nv->Zy[Y], rz = nv->Zz[T] - nv->Zz[Y];
        PState<double> pa = pos[fT + a];
        double xa = rx + pa.x, ya = ry + pa.y, za = rz + pa.z;
        for (int b = grp; b < nY; b += ngrp) {
            if (self && b == a) continue;
            PState<double> pb = pos[fY + b];
            double dx = xa - pb.x, dy = ya - pb.y, dz = za - pb.z;
            double r2 = dx * dx + dy * dy + dz * dz;
            if (__double_as_longlong(r2) != 0ll) {
                double w3, ir = 0.0;
                rinv_f64<POT>(r2, w3, ir);  // r^-3 (and r^-1) as the list schedule's panel forms them
                double mir3 = pb.m * w3;
                ax = fma(-mir3, dx, ax);
                ay = fma(-mir3, dy, ay);
                az = fma(-mir3, dz, az);
                if (POT) ph = fma(-pb.m, ir, ph);
            }
        }
    }
};

// a12 without lists: one warp per target leaf of at most 32 particles.  Lane l takes
// particle a = l mod nT and group g = l / nT of G = floor(32 / nT) groups; group g meets the
// partner's particles g, g + G, ...; at the end lane a adds its groups' sums in group
// order.  Leaves above 32 particles (only at the deepest level, from coincident keys) run
// in fused_p2p_big_k.
template <bool POT>
__global__ void __launch_bounds__(FB) fused_p2p_k(int nn, NodeView nv, double theta, float th2,
                                                  const PState<double>* __restrict__ pos,
                                                  Quad<double>* __restrict__ out, int* __restrict__ err) {
    __shared__ int2 stk[FW][FQCAP];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int T = blockIdx.x * FW + w; T < nn; T += gridDim.x * FW) {
        if (nv.nchild[T] != 0) continue;  // warp-uniform
        int nT = nv.count[T];
        if (nT > 32) continue;
        NearVisitor<POT> vis;
        vis.nv = &nv;
        vis.pos = pos;
        vis.T = T;
        vis.fT = nv.first[T];
        vis.nT = nT;
        vis.ngrp = 32 / nT;
        vis.a = lane % nT;
        vis.grp = lane / nT;
        vis.live = vis.grp < vis.ngrp;
        vis.ax = vis.ay = vis.az = vis.ph = 0.0;
        traverse(nv, T, theta, th2, stk[w], err, vis);
        double s[4] = {vis.ax, vis.ay, vis.az, vis.ph};
        double tot[4] = {0.0, 0.0, 0.0, 0.0};
        for (int g = 0; g < vis.ngrp; g++) {
#pragma unroll
            for (int cc = 0; cc < 4; cc++) tot[cc] += __shfl_sync(FULL, s[cc], (g * nT + vis.a) & 31);
        }
        if (lane < nT) out[vis.fT + lane] = Quad<double>{tot[0], tot[1], tot[2], POT ? tot[3] : 0.0};
        __syncwarp();
    }
}

// leaves above 32 particles: one warp per leaf, 32 particles per pass, partners in the
// traversal's order (these leaves are rare: coincident particles at the deepest level)
template <bool POT>
struct BigVisitor {
    const NodeView* nv;
    const PState<double>* pos;
    int T, fT, a;
    double ax, ay, az, ph;
    __device__ void m2l(int) {}
    __device__ void p2p(int Y) {
        bool self = Y == T;
        int fY = nv->first[Y], nY = nv->count[Y];
        double rx = nv->Zx[T] - nv->Zx[Y], ry = nv->Zy[T] - nv->Zy[Y], rz = nv->Zz[T] - nv->Zz[Y];
        PState<double> pa = pos[fT + a];
        double xa = rx + pa.x, ya = ry + pa.y, za = rz + pa.z;
        for (int b = 0; b < nY; b++) {
            if (self && b == a) continue;
            PState<double> pb = pos[fY + b];
            double dx = xa - pb.x, dy = ya - pb.y, dz = za - pb.z;
            double r2 = dx * dx + dy * dy + dz * dz;
            if (__double_as_longlong(r2) != 0ll) {
                double w3, ir = 0.0;
                rinv_f64<POT>(r2, w3, ir);  // r^-3 (and r^-1) as the list schedule's panel forms them
                double mir3 = pb.m * w3;
                ax = fma(-mir3, dx, ax);
                ay = fma(-mir3, dy, ay);
                az = fma(-mir3, dz, az);
                if (POT) ph = fma(-pb.m, ir, ph);
            }
        }
    }
};

template <bool POT>
__global__ void __launch_bounds__(FB) fused_p2p_big_k(int nn, NodeView nv, double theta, float th2,
                                                      const PState<double>* __restrict__ pos,
                                                      Quad<double>* __restrict__ out, int* __restrict__ err) {
    __shared__ int2 stk[FW][FQCAP];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int T = blockIdx.x * FW + w; T < nn; T += gridDim.x * FW) {
        if (nv.nchild[T] != 0 || nv.count[T] <= 32) continue;  // warp-uniform
        int nT = nv.count[T], fT = nv.first[T];
        for (int a0 = 0; a0 < nT; a0 += 32) {
            BigVisitor<POT> vis;
            vis.nv = &nv;
            vis.pos = pos;
            vis.T = T;
            vis.fT = fT;
            vis.a = min(a0 + lane, nT - 1);  // lanes past the end repeat the last particle (not stored)
            vis.ax = vis.ay = vis.az = vis.ph = 0.0;
            traverse(nv, T, theta, th2, stk[w], err, vis);
            if (a0 + lane < nT) out[fT + a0 + lane] = Quad<double>{vis.ax, vis.ay, vis.az, POT ? vis.ph : 0.0};
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------- host side

void fused_p2p_launch(fmm_ctx* c, bool want_pot, double theta, Quad<double>* out) {
    NodeView nv = node_view(c);
    float th2 = (float)theta * (float)theta;
    int nn = (int)c->n_nodes;
    int* err = c->errflag.as<int>() + 2;
    const PState<double>* pos = c->pos4.as<PState<double>>();
    int sms = 0;
    GB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    int g = sms * 16;
    if (want_pot) {
        fused_p2p_k<true><<<g, FB, 0, c->stream>>>(nn, nv, theta, th2, pos, out, err);
        GB_LAUNCH("fused_p2p_k");
        fused_p2p_big_k<true><<<g, FB, 0, c->stream>>>(nn, nv, theta, th2, pos, out, err);
    } else {
        fused_p2p_k<false><<<g, FB, 0, c->stream>>>(nn, nv, theta, th2, pos, out, err);
        GB_LAUNCH("fused_p2p_k");
        fused_p2p_big_k<false><<<g, FB, 0, c->stream>>>(nn, nv, theta, th2, pos, out, err);
    }
    GB_LAUNCH("fused_p2p_big_k");
}

}  // namespace gbfmm
