/*
 * fmm_oracle.c -- plain, slow, single-threaded FP64 reference of the symmetric
 * Cartesian fast multipole method (FMM) for Newtonian gravity (G = 1), in the
 * standard form and in the angular-momentum-conserving (realigned) form of
 * Korobkin et al., "Conservation of Angular Momentum in the Fast Multipole
 * Method" (arXiv:2107.07166).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle for the CUDA
 * path.  Only the test-suite, the package smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, table or header with the
 * CUDA library and must never be used as a fallback for it.
 *
 * Every floating-point step is written out in the order stated below and is
 * compiled with -ffp-contract=off, so that geometry (bounding cube, Morton
 * keys, centres of mass, r_max, the multipole acceptance test) is reproducible
 * bit for bit by any IEEE double implementation that uses the same order.
 *
 * Conventions (order p = multipole/potential order of Sec. 2.1, "expansion up
 * to 4-th order"; the paper's "zeroth order FMM" of Sec. 3.1 is p = 1):
 *   multi-index alpha = (ax, ay, az), |alpha| = ax + ay + az, ordered by
 *   degree, then ax descending, then ay descending.
 *   raw moments     M_alpha = sum_b m_b (-y_b)^alpha / alpha!      (Sec. 2.1, eq. jiaB)
 *   field tensors   D_alpha = d^alpha (-1/r) at R                  (eqs. D .. Dijkl)
 *   locals          L_gamma = sum_{|b|+|g|<=p} M_beta D_{beta+gamma}(R)   (eq. taylor)
 *   potential       phi(x)  = sum_gamma L_gamma x^gamma / gamma!   (eq. potential)
 *   acceleration    a_i(x)  = -sum_{|g|<=p-1} L_{gamma+e_i} x^gamma/gamma!  (eq. g_acc_BtoA)
 * Conserving form (realignment of Sec. 3.2, eq. realign, carried to any p):
 *   the pair force m_b g(d+R) with g(r) = -r/|r|^3 is projected on the line
 *   X_a - Y_b = R + d; the projected scalar is h(R + d) with h(r) = -|r|^-3,
 *   expanded to degree p-1 in d = x_a - y_b:
 *       a_{a<-b} = m_b T_{p-1}[h](d) (R + d),
 *   summed over b through the same raw moments:
 *       S_gamma   = sum_{|b|+|g|<=p-1} M_beta h_{beta+gamma}(R)
 *       W_{i,g}   = sum_{|b|+|g|<=p-1} (beta_i + 1) M_{beta+e_i} h_{beta+gamma}(R)
 *       U_gamma   = R S_gamma + W_gamma
 *       a(x)      = x S(x) + U(x).
 * Literal order-0 realigned form (Sec. 3.2, eqs. realign2, nab-expansion, aaB0;
 * variant 2, API order p = 1): every pair force is -m_b/R^2 times the expanded
 * unit vector (n + delta)(1 - n.delta), delta = (x_a - y_b)/R, n = R/|R|; summed
 * over b with sum m_b y_b = 0 this is
 *       a(x) = -(M/R^2) [n + x_perp/R - (n.x) x/R^2] + Qbar n / R^4,
 *       Qbar = sum_b m_b y_b y_b^T (raw second moment, trace included),
 * a polynomial of degree 1 in x written as x S(x) + U(x).  It needs moments up to
 * order 2, so the run carries order-2 moments (and, for the potential, the
 * standard order-2 locals) and degree-1 conserving locals.
 */
#define _POSIX_C_SOURCE 199309L
#include <math.h>
#include <stdint.h>
#include <time.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PMAX 8
#define ORC_NMI_MAX 165 /* (8+1)(8+2)(8+3)/6 */
#define ORC_MAXLEVEL 21

/* ------------------------------------------------------------------ */
/* multi-index tables                                                 */
/* ------------------------------------------------------------------ */

static int g_tables_ready = 0;
static int g_mi[ORC_NMI_MAX][3];                            /* index -> alpha */
static int g_idx[ORC_PMAX + 2][ORC_PMAX + 2][ORC_PMAX + 2]; /* alpha -> index */
static double g_fact[ORC_PMAX + 2];

static void orc_tables(void) {
    if (g_tables_ready) return;
    int k = 0;
    for (int n = 0; n <= ORC_PMAX; n++)
        for (int ax = n; ax >= 0; ax--)
            for (int ay = n - ax; ay >= 0; ay--) {
                int az = n - ax - ay;
                g_mi[k][0] = ax;
                g_mi[k][1] = ay;
                g_mi[k][2] = az;
                g_idx[ax][ay][az] = k;
                k++;
            }
    g_fact[0] = 1.0;
    for (int i = 1; i < ORC_PMAX + 2; i++) g_fact[i] = g_fact[i - 1] * (double)i;
    g_tables_ready = 1;
}

/* number of multi-indices with |alpha| <= p */
int orc_nmi(int p) {
    if (p < 0) return 0;
    return (p + 1) * (p + 2) * (p + 3) / 6;
}

/* alpha of index k (for tests) */
void orc_multi_index(int k, int *alpha) {
    orc_tables();
    alpha[0] = g_mi[k][0];
    alpha[1] = g_mi[k][1];
    alpha[2] = g_mi[k][2];
}

static double mi_fact(int k) { return g_fact[g_mi[k][0]] * g_fact[g_mi[k][1]] * g_fact[g_mi[k][2]]; }

static int mi_deg(int k) { return g_mi[k][0] + g_mi[k][1] + g_mi[k][2]; }

/* index of alpha + beta */
static int mi_add(int a, int b) {
    return g_idx[g_mi[a][0] + g_mi[b][0]][g_mi[a][1] + g_mi[b][1]][g_mi[a][2] + g_mi[b][2]];
}

/* v^alpha / alpha! for all |alpha| <= p */
static void mono_over_fact(int p, const double v[3], double *out) {
    int n = orc_nmi(p);
    for (int k = 0; k < n; k++) {
        double t = 1.0;
        for (int d = 0; d < 3; d++)
            for (int e = 0; e < g_mi[k][d]; e++) t = t * v[d];
        out[k] = t / mi_fact(k);
    }
}

/* ------------------------------------------------------------------ */
/* derivative tensors of radial kernels                               */
/* ------------------------------------------------------------------ */

/*
 * Taylor coefficients c_alpha = d^alpha f(R) / alpha! of f(r) = (r.r)^(-s),
 * |alpha| <= p, from the identity (u + 2R.t + t.t) sum_i t_i d_i g = -2s (R.t + t.t) g,
 * g(t) = f(R + t), u = R.R, which gives for |alpha| >= 1
 *   u |alpha| c_alpha = -(2|alpha| - 2 + 2s) sum_i R_i c_{alpha-e_i}
 *                       -( |alpha| - 2 + 2s) sum_i c_{alpha-2e_i}.
 */
static void radial_taylor(int p, double s, const double R[3], double *c) {
    double u = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
    int n = orc_nmi(p);
    c[0] = pow(u, -s);
    for (int k = 1; k < n; k++) {
        int na = mi_deg(k);
        double t1 = 0.0, t2 = 0.0;
        for (int d = 0; d < 3; d++) {
            int a[3] = {g_mi[k][0], g_mi[k][1], g_mi[k][2]};
            if (a[d] >= 1) {
                a[d] -= 1;
                t1 += R[d] * c[g_idx[a[0]][a[1]][a[2]]];
                if (a[d] >= 1) {
                    a[d] -= 1;
                    t2 += c[g_idx[a[0]][a[1]][a[2]]];
                }
            }
        }
        c[k] = -((2.0 * na - 2.0 + 2.0 * s) * t1 + (na - 2.0 + 2.0 * s) * t2) / (u * na);
    }
}

/* D_alpha = d^alpha (-1/r) at R, |alpha| <= p  (eqs. D, Di, Dij, Dijk, Dijkl) */
void orc_dtensor(int p, const double *R, double *D) {
    orc_tables();
    radial_taylor(p, 0.5, R, D);
    int n = orc_nmi(p);
    for (int k = 0; k < n; k++) D[k] = -D[k] * mi_fact(k);
}

/* h_alpha = d^alpha (-|r|^-3) at R, |alpha| <= p  (kernel of the realigned force) */
void orc_htensor(int p, const double *R, double *H) {
    orc_tables();
    radial_taylor(p, 1.5, R, H);
    int n = orc_nmi(p);
    for (int k = 0; k < n; k++) H[k] = -H[k] * mi_fact(k);
}

/* ------------------------------------------------------------------ */
/* bounding cube, Morton keys, stable sort                            */
/* ------------------------------------------------------------------ */

/* lo = per-axis minimum, side = largest extent (1 if all points coincide). */
void orc_bbox(const double *x, int64_t N, double *lo, double *side) {
    double mn[3], mx[3];
    for (int d = 0; d < 3; d++) mn[d] = mx[d] = x[d];
    for (int64_t i = 1; i < N; i++)
        for (int d = 0; d < 3; d++) {
            double v = x[3 * i + d];
            if (v < mn[d]) mn[d] = v;
            if (v > mx[d]) mx[d] = v;
        }
    double s = 0.0;
    for (int d = 0; d < 3; d++) {
        lo[d] = mn[d];
        double e = mx[d] - mn[d];
        if (e > s) s = e;
    }
    if (s == 0.0) s = 1.0;
    *side = s;
}

static uint64_t spread3(uint64_t q) {
    uint64_t r = 0;
    for (int b = 0; b < ORC_MAXLEVEL; b++) r |= ((q >> b) & 1ull) << (3 * b);
    return r;
}

/* 63-bit Morton key: bit 3b+2 = x bit b, 3b+1 = y bit b, 3b = z bit b.
 * q = min(floor((x - lo) * (2^21 / side)), 2^21 - 1). */
void orc_keys(const double *x, int64_t N, const double *lo, double side, uint64_t *keys) {
    double scale = 2097152.0 / side;
    for (int64_t i = 0; i < N; i++) {
        uint64_t q[3];
        for (int d = 0; d < 3; d++) {
            double t = (x[3 * i + d] - lo[d]) * scale;
            double f = floor(t);
            uint64_t v = (f <= 0.0) ? 0 : (uint64_t)f;
            if (v > 2097151ull) v = 2097151ull;
            q[d] = v;
        }
        keys[i] = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    }
}

typedef struct {
    uint64_t key;
    int64_t idx;
} kv_t;

static int kv_cmp(const void *a, const void *b) {
    const kv_t *x = (const kv_t *)a, *y = (const kv_t *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

/* stable sort by key: ties keep input order (sort by (key, index)) */
void orc_sort(const uint64_t *keys, int64_t N, uint64_t *sorted, int64_t *perm) {
    kv_t *t = (kv_t *)malloc(sizeof(kv_t) * (size_t)N);
    for (int64_t i = 0; i < N; i++) {
        t[i].key = keys[i];
        t[i].idx = i;
    }
    qsort(t, (size_t)N, sizeof(kv_t), kv_cmp);
    for (int64_t i = 0; i < N; i++) {
        sorted[i] = t[i].key;
        perm[i] = t[i].idx;
    }
    free(t);
}

/* ------------------------------------------------------------------ */
/* the oracle run                                                     */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t N;
    int leaf_size, p, variant, want_pot;
    double theta;
    double lo[3], side;
    uint64_t *keys; /* sorted */
    int64_t *perm;  /* sorted position -> input index */
    double *X;      /* sorted positions, N x 3 */
    double *m;      /* sorted masses */
    /* tree (breadth-first order) */
    int64_t n_nodes, cap_nodes;
    int32_t *first, *count, *level, *parent, *child_first, *nchild;
    double *M, *S, *Z, *rmax; /* mass, sum m X (x3), COM (x3), max radius */
    int32_t *leaf_of;         /* sorted particle -> leaf node */
    /* expansions */
    int nmom, nloc;
    double *mom;            /* n_nodes x nmi(p) */
    double *L;              /* standard locals, n_nodes x nmi(p) */
    double *SU;             /* conserving locals, n_nodes x 4*nmi(p-1): S, Ux, Uy, Uz */
    /* interaction lists (canonical: (min id, max id) lexicographic) */
    int64_t n_m2l, cap_m2l, n_p2p, cap_p2p;
    int32_t *m2l, *p2p;
    /* optional record of the walk: every visited pair (A, B) with its decision */
    int64_t n_trace, cap_trace;
    int32_t *trace; /* triples (A, B, decision), see WALK_* */
    /* seconds spent in [tree and geometry, P2M/M2M, walk, M2L, L2L + L2P, P2P] */
    double stage_s[6];
    /* results (input order) */
    double *acc, *pot;
    double *acc_s, *pot_s; /* sorted order */
} orc_t;

static void push_pair(int32_t **buf, int64_t *n, int64_t *cap, int32_t a, int32_t b) {
    if (*n == *cap) {
        *cap = *cap ? 2 * *cap : 1024;
        *buf = (int32_t *)realloc(*buf, sizeof(int32_t) * 2 * (size_t)*cap);
    }
    (*buf)[2 * *n] = a < b ? a : b;
    (*buf)[2 * *n + 1] = a < b ? b : a;
    (*n)++;
}

static int pair_cmp(const void *a, const void *b) {
    const int32_t *x = (const int32_t *)a, *y = (const int32_t *)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1;
    return 0;
}

static void grow_nodes(orc_t *o) {
    if (o->n_nodes < o->cap_nodes) return;
    o->cap_nodes = o->cap_nodes ? 2 * o->cap_nodes : 1024;
    size_t c = (size_t)o->cap_nodes;
    o->first = (int32_t *)realloc(o->first, 4 * c);
    o->count = (int32_t *)realloc(o->count, 4 * c);
    o->level = (int32_t *)realloc(o->level, 4 * c);
    o->parent = (int32_t *)realloc(o->parent, 4 * c);
    o->child_first = (int32_t *)realloc(o->child_first, 4 * c);
    o->nchild = (int32_t *)realloc(o->nchild, 4 * c);
}

/* Octree from sorted keys: a node is split while it holds more than leaf_size
 * particles and its level is below 21; children are the non-empty octants in
 * Morton order; node ids are breadth-first. */
static void build_tree(orc_t *o) {
    o->n_nodes = 0;
    grow_nodes(o);
    o->first[0] = 0;
    o->count[0] = (int32_t)o->N;
    o->level[0] = 0;
    o->parent[0] = -1;
    o->child_first[0] = -1;
    o->nchild[0] = 0;
    o->n_nodes = 1;
    for (int64_t n = 0; n < o->n_nodes; n++) {
        int lev = o->level[n];
        if (o->count[n] <= o->leaf_size || lev >= ORC_MAXLEVEL) continue;
        int shift = 60 - 3 * lev;
        int64_t beg = o->first[n], end = beg + o->count[n];
        int64_t i = beg;
        o->child_first[n] = (int32_t)o->n_nodes;
        while (i < end) {
            uint64_t oct = (o->keys[i] >> shift) & 7ull;
            int64_t j = i + 1;
            while (j < end && ((o->keys[j] >> shift) & 7ull) == oct) j++;
            grow_nodes(o);
            int64_t c = o->n_nodes++;
            o->first[c] = (int32_t)i;
            o->count[c] = (int32_t)(j - i);
            o->level[c] = lev + 1;
            o->parent[c] = (int32_t)n;
            o->child_first[c] = -1;
            o->nchild[c] = 0;
            o->nchild[n]++;
            i = j;
        }
    }
}

static int is_leaf(const orc_t *o, int64_t n) { return o->nchild[n] == 0; }

/* Centres of mass: leaves sum m and m*X sequentially in sorted order,
 * parents sum their children's sums in child order; Z = (sum m X) / M.
 * r_max = sqrt(max over the node's particles of |X - Z|^2). */
static void node_geometry(orc_t *o) {
    int64_t nn = o->n_nodes;
    o->M = (double *)malloc(8 * (size_t)nn);
    o->S = (double *)malloc(24 * (size_t)nn);
    o->Z = (double *)malloc(24 * (size_t)nn);
    o->rmax = (double *)malloc(8 * (size_t)nn);
    for (int64_t n = nn - 1; n >= 0; n--) {
        double M = 0.0, S[3] = {0.0, 0.0, 0.0};
        if (is_leaf(o, n)) {
            for (int64_t i = o->first[n]; i < o->first[n] + o->count[n]; i++) {
                M = M + o->m[i];
                for (int d = 0; d < 3; d++) S[d] = S[d] + o->m[i] * o->X[3 * i + d];
            }
        } else {
            for (int64_t c = o->child_first[n]; c < o->child_first[n] + o->nchild[n]; c++) {
                M = M + o->M[c];
                for (int d = 0; d < 3; d++) S[d] = S[d] + o->S[3 * c + d];
            }
        }
        o->M[n] = M;
        for (int d = 0; d < 3; d++) {
            o->S[3 * n + d] = S[d];
            /* a node without mass is centred on its first particle */
            o->Z[3 * n + d] = (M > 0.0) ? S[d] / M : o->X[3 * (int64_t)o->first[n] + d];
        }
        double r2 = 0.0;
        for (int64_t i = o->first[n]; i < o->first[n] + o->count[n]; i++) {
            double dx = o->X[3 * i] - o->Z[3 * n];
            double dy = o->X[3 * i + 1] - o->Z[3 * n + 1];
            double dz = o->X[3 * i + 2] - o->Z[3 * n + 2];
            double q = (dx * dx + dy * dy) + dz * dz;
            if (q > r2) r2 = q;
        }
        o->rmax[n] = sqrt(r2);
    }
    o->leaf_of = (int32_t *)malloc(4 * (size_t)o->N);
    for (int64_t n = 0; n < nn; n++)
        if (is_leaf(o, n))
            for (int64_t i = o->first[n]; i < o->first[n] + o->count[n]; i++) o->leaf_of[i] = (int32_t)n;
}

/* ---------------- dual-tree walk (mutual) ---------------- */

/* decisions recorded by the walk trace (a debug export for the tests) */
enum { WALK_SELF_SPLIT = 0, WALK_M2L = 1, WALK_P2P = 2, WALK_SPLIT_A = 3, WALK_SPLIT_B = 4 };
static int g_trace_on = 0;

/* switch the walk trace of later orc_run calls on (1) or off (0) */
void orc_set_trace(int on) { g_trace_on = on; }

static void trace(orc_t *o, int32_t A, int32_t B, int32_t decision) {
    if (!g_trace_on) return;
    if (o->n_trace == o->cap_trace) {
        o->cap_trace = o->cap_trace ? 2 * o->cap_trace : 1024;
        o->trace = (int32_t *)realloc(o->trace, sizeof(int32_t) * 3 * (size_t)o->cap_trace);
    }
    o->trace[3 * o->n_trace] = A;
    o->trace[3 * o->n_trace + 1] = B;
    o->trace[3 * o->n_trace + 2] = decision;
    o->n_trace++;
}

static void walk_pair(orc_t *o, int32_t A, int32_t B);

static void walk_self(orc_t *o, int32_t A) {
    if (is_leaf(o, A)) {
        trace(o, A, A, WALK_P2P);
        push_pair(&o->p2p, &o->n_p2p, &o->cap_p2p, A, A);
        return;
    }
    trace(o, A, A, WALK_SELF_SPLIT);
    int32_t c0 = o->child_first[A], nc = o->nchild[A];
    for (int32_t i = 0; i < nc; i++)
        for (int32_t j = i; j < nc; j++) {
            if (i == j)
                walk_self(o, c0 + i);
            else
                walk_pair(o, c0 + i, c0 + j);
        }
}

/* MAC (eq. mac_criterion): accept when R > 0 and r_A + r_B <= theta * R. */
static int mac_accept(const orc_t *o, int32_t A, int32_t B) {
    double dx = o->Z[3 * A] - o->Z[3 * B];
    double dy = o->Z[3 * A + 1] - o->Z[3 * B + 1];
    double dz = o->Z[3 * A + 2] - o->Z[3 * B + 2];
    double R = sqrt((dx * dx + dy * dy) + dz * dz);
    return R > 0.0 && (o->rmax[A] + o->rmax[B]) <= o->theta * R;
}

/* split A (rather than B): the larger r_max, ties -> larger count, then lower id */
static int split_first(const orc_t *o, int32_t A, int32_t B) {
    if (o->rmax[A] != o->rmax[B]) return o->rmax[A] > o->rmax[B];
    if (o->count[A] != o->count[B]) return o->count[A] > o->count[B];
    return A < B;
}

static void walk_pair(orc_t *o, int32_t A, int32_t B) {
    if (mac_accept(o, A, B)) {
        trace(o, A, B, WALK_M2L);
        push_pair(&o->m2l, &o->n_m2l, &o->cap_m2l, A, B);
        return;
    }
    int la = is_leaf(o, A), lb = is_leaf(o, B);
    if (la && lb) {
        trace(o, A, B, WALK_P2P);
        push_pair(&o->p2p, &o->n_p2p, &o->cap_p2p, A, B);
        return;
    }
    int splitA = lb ? 1 : (la ? 0 : split_first(o, A, B));
    trace(o, A, B, splitA ? WALK_SPLIT_A : WALK_SPLIT_B);
    if (splitA) {
        for (int32_t c = o->child_first[A]; c < o->child_first[A] + o->nchild[A]; c++) walk_pair(o, c, B);
    } else {
        for (int32_t c = o->child_first[B]; c < o->child_first[B] + o->nchild[B]; c++) walk_pair(o, A, c);
    }
}

/* ---------------- expansions ---------------- */

/* P2M: M_alpha = sum_b m_b (-y_b)^alpha / alpha!, y_b = Y_b - Z */
static void p2m(orc_t *o, int64_t n, double *mom) {
    double w[ORC_NMI_MAX];
    int nm = o->nmom;
    for (int k = 0; k < nm; k++) mom[k] = 0.0;
    for (int64_t i = o->first[n]; i < o->first[n] + o->count[n]; i++) {
        double y[3];
        for (int d = 0; d < 3; d++) y[d] = -(o->X[3 * i + d] - o->Z[3 * n + d]);
        mono_over_fact(o->p, y, w);
        for (int k = 0; k < nm; k++) mom[k] += o->m[i] * w[k];
    }
}

/* M2M: M^P_alpha += sum_{beta <= alpha} M^c_{alpha-beta} (-c)^beta / beta!, c = Z_c - Z_P */
static void m2m(orc_t *o, int64_t child, int64_t par) {
    double w[ORC_NMI_MAX], c[3];
    for (int d = 0; d < 3; d++) c[d] = -(o->Z[3 * child + d] - o->Z[3 * par + d]);
    mono_over_fact(o->p, c, w);
    const double *Mc = o->mom + child * o->nmom;
    double *Mp = o->mom + par * o->nmom;
    for (int a = 0; a < o->nmom; a++)
        for (int b = 0; b < o->nmom; b++) {
            int ok = 1;
            int r[3];
            for (int d = 0; d < 3; d++) {
                r[d] = g_mi[a][d] - g_mi[b][d];
                if (r[d] < 0) ok = 0;
            }
            if (ok) Mp[a] += Mc[g_idx[r[0]][r[1]][r[2]]] * w[b];
        }
}

/* standard M2L: L_gamma += sum_{|beta| <= p-|gamma|} M_beta D_{beta+gamma}(R), R = Z_tgt - Z_src */
static void m2l_standard(orc_t *o, int64_t tgt, int64_t src) {
    double R[3], D[ORC_NMI_MAX];
    for (int d = 0; d < 3; d++) R[d] = o->Z[3 * tgt + d] - o->Z[3 * src + d];
    orc_dtensor(o->p, R, D);
    const double *Ms = o->mom + src * o->nmom;
    double *L = o->L + tgt * o->nmom;
    for (int g = 0; g < o->nmom; g++)
        for (int b = 0; b < o->nmom; b++)
            if (mi_deg(g) + mi_deg(b) <= o->p) L[g] += Ms[b] * D[mi_add(b, g)];
}

/* conserving M2L: S and U = R S + W of the realigned pair force summed over the source */
static void m2l_conserving(orc_t *o, int64_t tgt, int64_t src) {
    double R[3], H[ORC_NMI_MAX];
    int q = o->p - 1, nq = orc_nmi(q);
    for (int d = 0; d < 3; d++) R[d] = o->Z[3 * tgt + d] - o->Z[3 * src + d];
    orc_htensor(q, R, H);
    const double *Ms = o->mom + src * o->nmom;
    double *S = o->SU + tgt * o->nloc;
    double *U = S + nq;
    for (int g = 0; g < nq; g++) {
        double s = 0.0, w[3] = {0.0, 0.0, 0.0};
        for (int b = 0; b < nq; b++) {
            if (mi_deg(g) + mi_deg(b) > q) continue;
            double hv = H[mi_add(b, g)];
            s += Ms[b] * hv;
            for (int d = 0; d < 3; d++) {
                int e[3] = {g_mi[b][0], g_mi[b][1], g_mi[b][2]};
                e[d] += 1;
                w[d] += (double)(g_mi[b][d] + 1) * Ms[g_idx[e[0]][e[1]][e[2]]] * hv;
            }
        }
        S[g] += s;
        for (int d = 0; d < 3; d++) U[d * nq + g] += R[d] * s + w[d];
    }
}

/* literal order-0 realigned M2L (eq. aaB0): the terms of
 *   a(x) = -(M/R^2) [n + x/R - (n.x) n/R - (n.x) x/R^2] + Qbar n / R^4
 * sorted into x S(x) + U(x) with S, U of degree 1:
 *   S_0 = -M/R^3            S_{e_j} = M n_j / R^4
 *   U_{i,0} = -M n_i/R^2 + (Qbar n)_i / R^4      U_{i,e_j} = M n_i n_j / R^3
 * with M = M_0 and Qbar_ij = sum m y_i y_j read from the raw moments
 * (Qbar_ii = 2 M_{2e_i}, Qbar_ij = M_{e_i+e_j} for i != j). */
static void m2l_paper0(orc_t *o, int64_t tgt, int64_t src) {
    double R[3];
    for (int d = 0; d < 3; d++) R[d] = o->Z[3 * tgt + d] - o->Z[3 * src + d];
    double r = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
    double n[3] = {R[0] / r, R[1] / r, R[2] / r};
    const double *Ms = o->mom + src * o->nmom;
    double M = Ms[0];
    double Q[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            int e[3] = {0, 0, 0};
            e[i] += 1;
            e[j] += 1;
            double v = Ms[g_idx[e[0]][e[1]][e[2]]];
            Q[i][j] = (i == j) ? 2.0 * v : v;
        }
    double r2 = r * r, r3 = r2 * r, r4 = r2 * r2;
    int nq = orc_nmi(1); /* 1, x, y, z */
    double *S = o->SU + tgt * o->nloc;
    double *U = S + nq;
    S[0] += -M / r3;
    for (int j = 0; j < 3; j++) S[1 + j] += M * n[j] / r4;
    for (int i = 0; i < 3; i++) {
        double Qn = Q[i][0] * n[0] + Q[i][1] * n[1] + Q[i][2] * n[2];
        U[i * nq] += -M * n[i] / r2 + Qn / r4;
        for (int j = 0; j < 3; j++) U[i * nq + 1 + j] += M * n[i] * n[j] / r3;
    }
}

/* L2L (polynomial shift): L'_gamma += sum_{|gamma+beta|<=p} L_{gamma+beta} s^beta/beta!, s = Z_c - Z_P */
static void l2l_poly(int p, const double *Lp, double *Lc, const double *w) {
    int n = orc_nmi(p);
    for (int g = 0; g < n; g++)
        for (int b = 0; b < n; b++)
            if (mi_deg(g) + mi_deg(b) <= p) Lc[g] += Lp[mi_add(g, b)] * w[b];
}

/* evaluate sum_gamma C_gamma x^gamma/gamma! over |gamma| <= p */
static double poly_eval(int p, const double *C, const double *w) {
    double s = 0.0;
    for (int g = 0; g < orc_nmi(p); g++) s += C[g] * w[g];
    return s;
}

/* L2P at offset x from the centre of node n.  Standard: a_i = -sum_{|g|<=p-1}
 * L_{g+e_i} x^g/g!.  Conserving: a = x S(x) + U(x).  Potential: sum_g L_g x^g/g!. */
static void l2p_one(const orc_t *o, int64_t n, const double *xv, double *acc, double *pot) {
    double w[ORC_NMI_MAX];
    int p = o->p;
    mono_over_fact(p, xv, w);
    if (o->variant == 0) {
        const double *L = o->L + n * o->nmom;
        for (int d = 0; d < 3; d++) {
            double a = 0.0;
            for (int g = 0; g < orc_nmi(p - 1); g++) {
                int e[3] = {g_mi[g][0], g_mi[g][1], g_mi[g][2]};
                e[d] += 1;
                a += L[g_idx[e[0]][e[1]][e[2]]] * w[g];
            }
            acc[d] = -a;
        }
    } else {
        int q = p - 1, nq = orc_nmi(q);
        const double *Sc = o->SU + n * o->nloc;
        double sv = poly_eval(q, Sc, w);
        for (int d = 0; d < 3; d++) acc[d] = xv[d] * sv + poly_eval(q, Sc + (d + 1) * nq, w);
    }
    if (pot) *pot = poly_eval(p, o->L + n * o->nmom, w);
}

/* ---------------- particle-particle ---------------- */

static void p2p_pair(orc_t *o, int64_t a, int64_t b, double *acc, double *pot) {
    double d[3];
    for (int k = 0; k < 3; k++) d[k] = o->X[3 * a + k] - o->X[3 * b + k];
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 == 0.0) return; /* coincident particles do not interact */
    double r = sqrt(r2);
    double ir3 = 1.0 / (r2 * r);
    for (int k = 0; k < 3; k++) {
        acc[3 * a + k] -= o->m[b] * d[k] * ir3;
        acc[3 * b + k] += o->m[a] * d[k] * ir3;
    }
    if (pot) {
        pot[a] -= o->m[b] / r;
        pot[b] -= o->m[a] / r;
    }
}

/* ---------------- driver ---------------- */

static double now_s(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

void orc_free(orc_t *o);

/* Full evaluation.  x: N x 3 input order, m: N.  variant 0 standard, 1 conserving,
 * 2 literal order-0 realigned (p must be 1; carried internally at expansion order 2:
 * order-2 moments, degree-1 conserving locals, standard order-2 potential). */
orc_t *orc_run(const double *x, const double *m, int64_t N, int leaf_size, int p, double theta, int variant,
               int want_pot) {
    orc_tables();
    if (N < 1 || leaf_size < 1 || p < 1 || p > ORC_PMAX || variant < 0 || variant > 2) return NULL;
    if (variant == 2) {
        if (p != 1) return NULL;
        p = 2;
    }
    orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
    o->N = N;
    o->leaf_size = leaf_size;
    o->p = p;
    o->theta = theta;
    o->variant = variant;
    o->want_pot = want_pot;
    double t0 = now_s();
    /* a1 bounding cube, a2 keys, a3 sort */
    uint64_t *k0 = (uint64_t *)malloc(8 * (size_t)N);
    orc_bbox(x, N, o->lo, &o->side);
    orc_keys(x, N, o->lo, o->side, k0);
    o->keys = (uint64_t *)malloc(8 * (size_t)N);
    o->perm = (int64_t *)malloc(8 * (size_t)N);
    orc_sort(k0, N, o->keys, o->perm);
    free(k0);
    o->X = (double *)malloc(24 * (size_t)N);
    o->m = (double *)malloc(8 * (size_t)N);
    for (int64_t i = 0; i < N; i++) {
        for (int d = 0; d < 3; d++) o->X[3 * i + d] = x[3 * o->perm[i] + d];
        o->m[i] = m[o->perm[i]];
    }
    /* a4 tree, node geometry */
    build_tree(o);
    node_geometry(o);
    int64_t nn = o->n_nodes;
    double t1 = now_s();
    o->stage_s[0] = t1 - t0;
    /* a5 P2M, a6 M2M (children before parents: reverse breadth-first order) */
    o->nmom = orc_nmi(p);
    o->nloc = 4 * orc_nmi(p - 1);
    o->mom = (double *)calloc((size_t)nn * o->nmom, 8);
    for (int64_t n = nn - 1; n >= 0; n--) {
        if (is_leaf(o, n))
            p2m(o, n, o->mom + n * o->nmom);
        else
            for (int64_t c = o->child_first[n]; c < o->child_first[n] + o->nchild[n]; c++) m2m(o, c, n);
    }
    double t2 = now_s();
    o->stage_s[1] = t2 - t1;
    /* a7 walk, canonical order */
    walk_self(o, 0);
    if (o->n_m2l) qsort(o->m2l, (size_t)o->n_m2l, 8, pair_cmp);
    if (o->n_p2p) qsort(o->p2p, (size_t)o->n_p2p, 8, pair_cmp);
    double t3 = now_s();
    o->stage_s[2] = t3 - t2;
    /* a8 M2L (both partners of each mutual pair), a9 accumulation in list order */
    int need_L = (variant == 0) || want_pot;
    if (need_L) o->L = (double *)calloc((size_t)nn * o->nmom, 8);
    if (variant >= 1) o->SU = (double *)calloc((size_t)nn * o->nloc, 8);
    for (int64_t k = 0; k < o->n_m2l; k++) {
        int32_t A = o->m2l[2 * k], B = o->m2l[2 * k + 1];
        if (need_L) {
            m2l_standard(o, A, B);
            m2l_standard(o, B, A);
        }
        if (variant == 1) {
            m2l_conserving(o, A, B);
            m2l_conserving(o, B, A);
        }
        if (variant == 2) {
            m2l_paper0(o, A, B);
            m2l_paper0(o, B, A);
        }
    }
    double t4 = now_s();
    o->stage_s[3] = t4 - t3;
    /* a10 L2L, parents before children (breadth-first order) */
    double w[ORC_NMI_MAX];
    for (int64_t n = 1; n < nn; n++) {
        int64_t P = o->parent[n];
        double s[3];
        for (int d = 0; d < 3; d++) s[d] = o->Z[3 * n + d] - o->Z[3 * P + d];
        mono_over_fact(p, s, w);
        if (need_L) l2l_poly(p, o->L + P * o->nmom, o->L + n * o->nmom, w);
        if (variant >= 1) {
            int q = p - 1, nq = orc_nmi(q);
            double *Sc = o->SU + n * o->nloc;
            const double *Sp = o->SU + P * o->nloc;
            double shS[ORC_NMI_MAX];
            for (int g = 0; g < nq; g++) shS[g] = 0.0;
            l2l_poly(q, Sp, shS, w);
            for (int g = 0; g < nq; g++) Sc[g] += shS[g];
            for (int d = 0; d < 3; d++) {
                l2l_poly(q, Sp + (d + 1) * nq, Sc + (d + 1) * nq, w);
                for (int g = 0; g < nq; g++) Sc[(d + 1) * nq + g] += s[d] * shS[g];
            }
        }
    }
    /* a11 L2P */
    o->acc_s = (double *)calloc(3 * (size_t)N, 8);
    o->pot_s = want_pot ? (double *)calloc((size_t)N, 8) : NULL;
    for (int64_t i = 0; i < N; i++) {
        int32_t n = o->leaf_of[i];
        double xv[3];
        for (int d = 0; d < 3; d++) xv[d] = o->X[3 * i + d] - o->Z[3 * n + d];
        l2p_one(o, n, xv, o->acc_s + 3 * i, want_pot ? o->pot_s + i : NULL);
    }
    double t5 = now_s();
    o->stage_s[4] = t5 - t4;
    /* a12 P2P (mutual, list order) */
    double *acc_pp = (double *)calloc(3 * (size_t)N, 8);
    double *pot_pp = want_pot ? (double *)calloc((size_t)N, 8) : NULL;
    for (int64_t k = 0; k < o->n_p2p; k++) {
        int32_t A = o->p2p[2 * k], B = o->p2p[2 * k + 1];
        if (A == B) {
            for (int64_t a = o->first[A]; a < o->first[A] + o->count[A]; a++)
                for (int64_t b = a + 1; b < o->first[A] + o->count[A]; b++) p2p_pair(o, a, b, acc_pp, pot_pp);
        } else {
            for (int64_t a = o->first[A]; a < o->first[A] + o->count[A]; a++)
                for (int64_t b = o->first[B]; b < o->first[B] + o->count[B]; b++) p2p_pair(o, a, b, acc_pp, pot_pp);
        }
    }
    o->stage_s[5] = now_s() - t5;
    /* a13 sum and return to input order */
    o->acc = (double *)malloc(24 * (size_t)N);
    o->pot = want_pot ? (double *)malloc(8 * (size_t)N) : NULL;
    for (int64_t i = 0; i < N; i++) {
        int64_t j = o->perm[i];
        for (int d = 0; d < 3; d++) {
            o->acc_s[3 * i + d] += acc_pp[3 * i + d];
            o->acc[3 * j + d] = o->acc_s[3 * i + d];
        }
        if (want_pot) {
            o->pot_s[i] += pot_pp[i];
            o->pot[j] = o->pot_s[i];
        }
    }
    free(acc_pp);
    free(pot_pp);
    return o;
}

/* Interaction counts of the walk alone (steps a1..a4 and a7, no expansions), for the
 * timing model of the oracle at sizes it is not run at: nodes, mutual M2L pairs, P2P
 * pairs, and unordered particle pairs evaluated directly. */
void orc_counts(const double *x, const double *m, int64_t N, int leaf_size, double theta, int64_t *out4) {
    orc_tables();
    orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
    o->N = N;
    o->leaf_size = leaf_size;
    o->theta = theta;
    uint64_t *k0 = (uint64_t *)malloc(8 * (size_t)N);
    orc_bbox(x, N, o->lo, &o->side);
    orc_keys(x, N, o->lo, o->side, k0);
    o->keys = (uint64_t *)malloc(8 * (size_t)N);
    o->perm = (int64_t *)malloc(8 * (size_t)N);
    orc_sort(k0, N, o->keys, o->perm);
    free(k0);
    o->X = (double *)malloc(24 * (size_t)N);
    o->m = (double *)malloc(8 * (size_t)N);
    for (int64_t i = 0; i < N; i++) {
        for (int d = 0; d < 3; d++) o->X[3 * i + d] = x[3 * o->perm[i] + d];
        o->m[i] = m[o->perm[i]];
    }
    build_tree(o);
    node_geometry(o);
    walk_self(o, 0);
    int64_t npp = 0;
    for (int64_t k = 0; k < o->n_p2p; k++) {
        int64_t a = o->count[o->p2p[2 * k]], b = o->count[o->p2p[2 * k + 1]];
        npp += o->p2p[2 * k] == o->p2p[2 * k + 1] ? a * (a - 1) / 2 : a * b;
    }
    out4[0] = o->n_nodes;
    out4[1] = o->n_m2l;
    out4[2] = o->n_p2p;
    out4[3] = npp;
    orc_free(o);
}

void orc_free(orc_t *o) {
    if (!o) return;
    void *ptrs[] = {o->keys, o->perm, o->X, o->m, o->first, o->count, o->level, o->parent, o->child_first,
                    o->nchild, o->M, o->S, o->Z, o->rmax, o->leaf_of, o->mom, o->L, o->SU, o->m2l, o->p2p,
                    o->acc, o->pot, o->acc_s, o->pot_s, o->trace};
    for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); i++) free(ptrs[i]);
    free(o);
}

/* ---------------- accessors ---------------- */

int64_t orc_n_nodes(const orc_t *o) { return o->n_nodes; }
int64_t orc_n_trace(const orc_t *o) { return o->n_trace; }
/* seconds of [tree and geometry, P2M/M2M, walk, M2L, L2L + L2P, P2P] of the run */
void orc_stage_seconds(const orc_t *o, double *out6) { memcpy(out6, o->stage_s, sizeof(o->stage_s)); }
/* the walk trace (orc_set_trace): n_trace x 3 int32, in visiting order */
void orc_get_trace(const orc_t *o, int32_t *out) {
    if (o->n_trace) memcpy(out, o->trace, sizeof(int32_t) * 3 * (size_t)o->n_trace);
}
int64_t orc_n_m2l(const orc_t *o) { return o->n_m2l; }
int64_t orc_n_p2p(const orc_t *o) { return o->n_p2p; }

void orc_get_keys(const orc_t *o, uint64_t *keys, int64_t *perm, double *lo, double *side) {
    memcpy(keys, o->keys, 8 * (size_t)o->N);
    memcpy(perm, o->perm, 8 * (size_t)o->N);
    memcpy(lo, o->lo, 24);
    *side = o->side;
}

void orc_get_tree(const orc_t *o, int32_t *first, int32_t *count, int32_t *level, int32_t *parent,
                  int32_t *child_first, int32_t *nchild) {
    size_t b = 4 * (size_t)o->n_nodes;
    memcpy(first, o->first, b);
    memcpy(count, o->count, b);
    memcpy(level, o->level, b);
    memcpy(parent, o->parent, b);
    memcpy(child_first, o->child_first, b);
    memcpy(nchild, o->nchild, b);
}

void orc_get_geometry(const orc_t *o, double *M, double *Z, double *rmax) {
    memcpy(M, o->M, 8 * (size_t)o->n_nodes);
    memcpy(Z, o->Z, 24 * (size_t)o->n_nodes);
    memcpy(rmax, o->rmax, 8 * (size_t)o->n_nodes);
}

void orc_get_moments(const orc_t *o, double *mom) { memcpy(mom, o->mom, 8 * (size_t)o->n_nodes * o->nmom); }

/* standard locals (n_nodes x nmi(p)) if computed; conserving (n_nodes x 4 nmi(p-1)) if computed */
int orc_get_locals(const orc_t *o, double *L, double *SU) {
    int r = 0;
    if (L && o->L) {
        memcpy(L, o->L, 8 * (size_t)o->n_nodes * o->nmom);
        r |= 1;
    }
    if (SU && o->SU) {
        memcpy(SU, o->SU, 8 * (size_t)o->n_nodes * o->nloc);
        r |= 2;
    }
    return r;
}

void orc_get_lists(const orc_t *o, int32_t *m2l, int32_t *p2p) {
    if (o->n_m2l) memcpy(m2l, o->m2l, 8 * (size_t)o->n_m2l);
    if (o->n_p2p) memcpy(p2p, o->p2p, 8 * (size_t)o->n_p2p);
}

void orc_get_result(const orc_t *o, double *acc, double *pot) {
    memcpy(acc, o->acc, 24 * (size_t)o->N);
    if (pot && o->pot) memcpy(pot, o->pot, 8 * (size_t)o->N);
}

/* ------------------------------------------------------------------ */
/* references used by the pins                                        */
/* ------------------------------------------------------------------ */

/* O(N^2) direct sum (eq. jia and its gradient), pairs with r = 0 skipped. */
void orc_direct(const double *x, const double *m, int64_t N, double *acc, double *pot) {
    for (int64_t i = 0; i < 3 * N; i++) acc[i] = 0.0;
    if (pot)
        for (int64_t i = 0; i < N; i++) pot[i] = 0.0;
    for (int64_t a = 0; a < N; a++)
        for (int64_t b = a + 1; b < N; b++) {
            double d[3];
            for (int k = 0; k < 3; k++) d[k] = x[3 * a + k] - x[3 * b + k];
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 == 0.0) continue;
            double r = sqrt(r2);
            double ir3 = 1.0 / (r2 * r);
            for (int k = 0; k < 3; k++) {
                acc[3 * a + k] -= m[b] * d[k] * ir3;
                acc[3 * b + k] += m[a] * d[k] * ir3;
            }
            if (pot) {
                pot[a] -= m[b] / r;
                pot[b] -= m[a] / r;
            }
        }
}

/* Direct sum for a subset of targets (indices tgt[0..nt)) over all sources. */
void orc_direct_targets(const double *x, const double *m, int64_t N, const int64_t *tgt, int64_t nt, double *acc,
                        double *pot) {
    for (int64_t t = 0; t < nt; t++) {
        int64_t a = tgt[t];
        double ax = 0.0, ay = 0.0, az = 0.0, ph = 0.0;
        for (int64_t b = 0; b < N; b++) {
            double d[3];
            for (int k = 0; k < 3; k++) d[k] = x[3 * a + k] - x[3 * b + k];
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 == 0.0) continue;
            double r = sqrt(r2);
            double ir3 = 1.0 / (r2 * r);
            ax -= m[b] * d[0] * ir3;
            ay -= m[b] * d[1] * ir3;
            az -= m[b] * d[2] * ir3;
            ph -= m[b] / r;
        }
        acc[3 * t] = ax;
        acc[3 * t + 1] = ay;
        acc[3 * t + 2] = az;
        if (pot) pot[t] = ph;
    }
}

/*
 * Per-pair truncated Taylor forces between two clusters, without moments:
 * for every a in A (positions XA, nA) and every b in B (YB, mB, nB), with
 * R = ZA - ZB, d = (XA_a - ZA) - (YB_b - ZB):
 *   standard   : a_a += m_b T_{p-1}[g](d) with g = -grad(-1/r) = -r/|r|^3, i.e.
 *                a_i += -m_b sum_{|alpha| <= p-1} d^alpha/alpha! D_{alpha+e_i}(R)
 *   conserving : a_a += m_b T_{p-1}[h](d) (R + d)
 *   potential  : phi_a += m_b T_p[-1/r](d)
 * This is the quantity the multipole route must reproduce exactly (up to rounding).
 */
void orc_pair_taylor(int p, int variant, const double *ZA, const double *XA, int64_t nA, const double *ZB,
                     const double *YB, const double *mB, int64_t nB, double *acc, double *pot) {
    orc_tables();
    double R[3], D[ORC_NMI_MAX], H[ORC_NMI_MAX], w[ORC_NMI_MAX];
    for (int k = 0; k < 3; k++) R[k] = ZA[k] - ZB[k];
    orc_dtensor(p, R, D);
    orc_htensor(p - 1, R, H);
    for (int64_t a = 0; a < nA; a++) {
        double av[3] = {0.0, 0.0, 0.0}, ph = 0.0;
        for (int64_t b = 0; b < nB; b++) {
            double d[3];
            for (int k = 0; k < 3; k++) d[k] = (XA[3 * a + k] - ZA[k]) - (YB[3 * b + k] - ZB[k]);
            mono_over_fact(p, d, w);
            ph += mB[b] * poly_eval(p, D, w);
            if (variant == 0) {
                for (int k = 0; k < 3; k++) {
                    double s = 0.0;
                    for (int g = 0; g < orc_nmi(p - 1); g++) {
                        int e[3] = {g_mi[g][0], g_mi[g][1], g_mi[g][2]};
                        e[k] += 1;
                        s += D[g_idx[e[0]][e[1]][e[2]]] * w[g];
                    }
                    av[k] += -mB[b] * s;
                }
            } else {
                double s = poly_eval(p - 1, H, w);
                for (int k = 0; k < 3; k++) av[k] += mB[b] * s * (R[k] + d[k]);
            }
        }
        for (int k = 0; k < 3; k++) acc[3 * a + k] = av[k];
        if (pot) pot[a] = ph;
    }
}

/* Moments of a particle set about Z (P2M alone), and one M2M shift. */
void orc_p2m(int p, const double *Z, const double *Y, const double *m, int64_t n, double *mom) {
    orc_tables();
    double w[ORC_NMI_MAX];
    int nm = orc_nmi(p);
    for (int k = 0; k < nm; k++) mom[k] = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double y[3];
        for (int d = 0; d < 3; d++) y[d] = -(Y[3 * i + d] - Z[d]);
        mono_over_fact(p, y, w);
        for (int k = 0; k < nm; k++) mom[k] += m[i] * w[k];
    }
}

/* shift moments from centre Zc to centre Zp */
void orc_m2m(int p, const double *Zc, const double *Zp, const double *Mc, double *Mp) {
    orc_tables();
    orc_t o;
    memset(&o, 0, sizeof(o));
    double Z[6] = {Zc[0], Zc[1], Zc[2], Zp[0], Zp[1], Zp[2]};
    int nm = orc_nmi(p);
    double *mom = (double *)calloc(2 * (size_t)nm, 8);
    memcpy(mom, Mc, 8 * (size_t)nm);
    o.p = p;
    o.nmom = nm;
    o.Z = Z;
    o.mom = mom;
    m2m(&o, 0, 1);
    memcpy(Mp, mom + nm, 8 * (size_t)nm);
    free(mom);
}

/* shift a local polynomial of degree p by s (L2L) */
void orc_l2l(int p, const double *s, const double *Lp, double *Lc) {
    orc_tables();
    double w[ORC_NMI_MAX];
    mono_over_fact(p, s, w);
    for (int g = 0; g < orc_nmi(p); g++) Lc[g] = 0.0;
    l2l_poly(p, Lp, Lc, w);
}

/* One mutual cell interaction through the multipole route, target A <- source B:
 * P2M of B about ZB, M2L into a local about ZA, L2P at every XA.  The pins compare
 * it with orc_pair_taylor, which sums the same truncated series particle by particle. */
void orc_cell_pair(int p, int variant, const double *ZA, const double *XA, int64_t nA, const double *ZB,
                   const double *YB, const double *mB, int64_t nB, double *acc, double *pot) {
    orc_tables();
    if (variant == 2) p = 2; /* literal order-0 form: order-2 moments, degree-1 locals */
    orc_t o;
    memset(&o, 0, sizeof(o));
    double Z[6] = {ZA[0], ZA[1], ZA[2], ZB[0], ZB[1], ZB[2]};
    o.p = p;
    o.variant = variant;
    o.nmom = orc_nmi(p);
    o.nloc = 4 * orc_nmi(p - 1);
    o.Z = Z;
    o.mom = (double *)calloc(2 * (size_t)o.nmom, 8);
    o.L = (double *)calloc(2 * (size_t)o.nmom, 8);
    o.SU = (double *)calloc(2 * (size_t)o.nloc, 8);
    orc_p2m(p, ZB, YB, mB, nB, o.mom + o.nmom);
    m2l_standard(&o, 0, 1);
    if (variant == 1) m2l_conserving(&o, 0, 1);
    if (variant == 2) m2l_paper0(&o, 0, 1);
    for (int64_t a = 0; a < nA; a++) {
        double xv[3];
        for (int d = 0; d < 3; d++) xv[d] = XA[3 * a + d] - ZA[d];
        l2p_one(&o, 0, xv, acc + 3 * a, pot ? pot + a : NULL);
    }
    free(o.mom);
    free(o.L);
    free(o.SU);
}
