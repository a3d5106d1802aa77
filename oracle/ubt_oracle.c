/*
 * ubt_oracle.c -- plain, slow, single-threaded CPU oracle for uncertain
 * balanced / unbalanced triangle counting and enumeration.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  It shares no code, header, table or helper
 * with the CUDA library, and the CUDA library never calls it.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg load it.
 *
 * What it computes, and the passage each part follows (paper: "Counting
 * Balanced Triangles on Social Networks With Uncertain Edge Signs"):
 *
 *  - Uncertain signed graph G = (V, E, P+), each edge present with certainty,
 *    its sign positive with probability P+(e)                 (Def. 1, Sec. 3)
 *  - Triangle listing by forward edge iteration under Node Order: for u, for
 *    v in N>(u), w in N>(u) n N>(v), lists sorted by id, merged  (Def. Node
 *    Order and Alg. 1, Sec. 4)
 *  - P_bal as the four-term sum over the classes T3 and T1 of products of
 *    independent P+ / P- values                          (equation in Sec. 3)
 *  - balanced iff P_bal >= t, unbalanced iff P_unbal = 1 - P_bal > t
 *                                         (Defs. 4 and 5; Alg. 1, Sec. 3-4)
 *  - expected counts  E_bal = sum_t P_bal(t), E_unbal = sum_t P_unbal(t), and
 *    dE_bal/dp_e from the term-wise derivative of the four-term sum
 *    (derived from the same equation; not in the paper)
 *  - local counts |B_t(e)|, |B_t(v)|: classified triangles through an edge
 *    or a vertex, the per-sample quantities of the samplers (Sec. 6)
 *  - Monte-Carlo sign worlds: a world is one draw of every edge sign; a
 *    triangle is balanced in a world iff it holds an odd number of positive
 *    edges (Def. 3, Sec. 3).  The draws come from Philox4x64-10 (Salmon,
 *    Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 *    SC'11), written here from that paper's description.
 *
 * Fixed point.  P+(e) = k_e / 65536 with integer k_e in [0, 65536].  The
 * four-term sum is then an exact integer N_bal = P_bal * 2^48 (each product
 * of three factors in [0, 65536] is <= 2^48 and the four products sum to at
 * most 2^48), so every threshold test below is exact.  With t a double in
 * [0.5, 1], t * 2^48 is exact, and
 *     P_bal  >= t  <=>  N_bal            >= ceil (t * 2^48)
 *     P_unbal > t  <=>  2^48 - N_bal     >  floor(t * 2^48).
 * The enumeration record's P_bal = N_bal / 2^48 is exact in double.
 *
 * Floating-point inputs (p as float32) are handled in double with Neumaier
 * compensated summation of the per-triangle terms.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ONE16 65536ULL          /* fixed-point denominator of one probability */
#define ONE48 (1ULL << 48)      /* denominator of a product of three */

/* status codes of this oracle (independent of the CUDA library's) */
#define OR_OK 0
#define OR_BAD_VERTEX (-1)
#define OR_SELF_LOOP (-2)
#define OR_DUPLICATE (-3)
#define OR_BAD_PROB (-4)
#define OR_BAD_TAU (-5)
#define OR_NOMEM (-6)

/* ------------------------------------------------------------------------ */
/* Graph in forward form: N>(u) for every u, sorted by neighbour id.         */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n, m;
    int64_t* deg;     /* undirected degree */
    int64_t* off;     /* n+1 offsets into nbr/eix */
    uint32_t* nbr;    /* forward neighbours (later in Node Order) */
    uint32_t* eix;    /* input edge index of each forward entry */
} fgraph;

/* Node Order (Def. Node Order, Sec. 4): a before b iff deg(a) < deg(b), or
 * equal degrees and id(a) < id(b). */
static int node_before(const fgraph* g, uint32_t a, uint32_t b) {
    if (g->deg[a] != g->deg[b]) return g->deg[a] < g->deg[b];
    return a < b;
}

typedef struct { uint32_t nb, ex; } pair32;

static int cmp_pair(const void* x, const void* y) {
    const pair32* a = (const pair32*)x;
    const pair32* b = (const pair32*)y;
    if (a->nb != b->nb) return a->nb < b->nb ? -1 : 1;
    return 0;
}

static void fgraph_free(fgraph* g) {
    free(g->deg); free(g->off); free(g->nbr); free(g->eix);
    memset(g, 0, sizeof(*g));
}

/* Validates the edge list (ids < n, no self-loops, no repeated pair) and
 * builds N>(u) under Node Order. */
static int fgraph_build(fgraph* g, int64_t n, int64_t m, const uint32_t* src, const uint32_t* dst) {
    memset(g, 0, sizeof(*g));
    g->n = n; g->m = m;
    g->deg = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    g->off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    g->nbr = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
    g->eix = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
    if (!g->deg || !g->off || !g->nbr || !g->eix) { fgraph_free(g); return OR_NOMEM; }
    for (int64_t i = 0; i < m; i++) {
        if ((int64_t)src[i] >= n || (int64_t)dst[i] >= n) { fgraph_free(g); return OR_BAD_VERTEX; }
        if (src[i] == dst[i]) { fgraph_free(g); return OR_SELF_LOOP; }
        g->deg[src[i]]++;
        g->deg[dst[i]]++;
    }
    /* each edge goes into the list of its earlier endpoint */
    for (int64_t i = 0; i < m; i++) {
        uint32_t a = src[i], b = dst[i];
        uint32_t lo = node_before(g, a, b) ? a : b;
        g->off[lo + 1]++;
    }
    for (int64_t u = 0; u < n; u++) g->off[u + 1] += g->off[u];
    int64_t* fill = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    pair32* tmp = (pair32*)malloc(sizeof(pair32) * (size_t)(m > 0 ? m : 1));
    if (!fill || !tmp) { free(fill); free(tmp); fgraph_free(g); return OR_NOMEM; }
    for (int64_t i = 0; i < m; i++) {
        uint32_t a = src[i], b = dst[i];
        uint32_t lo = node_before(g, a, b) ? a : b;
        uint32_t hi = (lo == a) ? b : a;
        int64_t at = g->off[lo] + fill[lo]++;
        tmp[at].nb = hi;
        tmp[at].ex = (uint32_t)i;
    }
    int rc = OR_OK;
    for (int64_t u = 0; u < n && rc == OR_OK; u++) {
        int64_t s = g->off[u], e = g->off[u + 1];
        qsort(tmp + s, (size_t)(e - s), sizeof(pair32), cmp_pair);
        for (int64_t j = s + 1; j < e; j++)
            if (tmp[j].nb == tmp[j - 1].nb) { rc = OR_DUPLICATE; break; }
    }
    for (int64_t j = 0; j < m; j++) { g->nbr[j] = tmp[j].nb; g->eix[j] = tmp[j].ex; }
    free(fill); free(tmp);
    if (rc != OR_OK) fgraph_free(g);
    return rc;
}

/* A listed triangle, vertices sorted by id a < b < c, with the input edge
 * index of each of its three edges. */
typedef struct { uint32_t a, b, c, e_ab, e_ac, e_bc; } tri_t;
typedef void (*tri_visit)(void* ctx, const tri_t* t);

/* Alg. 1's inner loops for one u: for v in N>(u), for w in N>(u) n N>(v)
 * (merge of the two id-sorted lists).  Returns the number of triangles. */
static int64_t triangles_from(const fgraph* g, int64_t u, tri_visit fn, void* ctx) {
    int64_t count = 0;
    int64_t us = g->off[u], ue = g->off[u + 1];
    for (int64_t iv = us; iv < ue; iv++) {
        uint32_t v = g->nbr[iv];
        uint32_t e_uv = g->eix[iv];
        int64_t i = us, j = g->off[v], je = g->off[v + 1];
        while (i < ue && j < je) {
            if (g->nbr[i] < g->nbr[j]) i++;
            else if (g->nbr[i] > g->nbr[j]) j++;
            else {
                uint32_t w = g->nbr[i];
                uint32_t e_uw = g->eix[i], e_vw = g->eix[j];
                if (fn) {
                    /* sort (u, v, w) by id, carrying the opposite-edge labels */
                    uint32_t x[3] = {(uint32_t)u, v, w};
                    /* edge between x[p] and x[q] for p<q */
                    uint32_t e01 = e_uv, e02 = e_uw, e12 = e_vw;
                    /* bubble sort of three with edge relabelling */
                    if (x[0] > x[1]) { uint32_t t = x[0]; x[0] = x[1]; x[1] = t; t = e02; e02 = e12; e12 = t; }
                    if (x[1] > x[2]) { uint32_t t = x[1]; x[1] = x[2]; x[2] = t; t = e01; e01 = e02; e02 = t; }
                    if (x[0] > x[1]) { uint32_t t = x[0]; x[0] = x[1]; x[1] = t; t = e02; e02 = e12; e12 = t; }
                    tri_t tr = {x[0], x[1], x[2], e01, e02, e12};
                    fn(ctx, &tr);
                }
                count++;
                i++; j++;
            }
        }
    }
    return count;
}

/* Alg. 1 framework: for u (every vertex), the loops above.  Returns the
 * number of triangles. */
static int64_t for_each_triangle(const fgraph* g, tri_visit fn, void* ctx) {
    int64_t count = 0;
    for (int64_t u = 0; u < g->n; u++) count += triangles_from(g, u, fn, ctx);
    return count;
}

/* ------------------------------------------------------------------------ */
/* Balance probability, fixed point (equation in Sec. 3)                     */
/* ------------------------------------------------------------------------ */

/* N_bal = 2^48 * P_bal = sum over T3 and T1 of products of P+ / P-:
 *   P+P+P+  +  P+P-P-  +  P-P+P-  +  P-P-P+   (each factor scaled by 65536) */
static uint64_t nbal_fixed(uint32_t k1, uint32_t k2, uint32_t k3) {
    uint64_t p1 = k1, p2 = k2, p3 = k3;
    uint64_t n1 = ONE16 - p1, n2 = ONE16 - p2, n3 = ONE16 - p3;
    return p1 * p2 * p3 + p1 * n2 * n3 + n1 * p2 * n3 + n1 * n2 * p3;
}

/* thresholds for one t: balanced iff N_bal >= tb; unbalanced iff 2^48 - N_bal > tu */
static int tau_levels(double t, uint64_t* tb, uint64_t* tu) {
    if (!(t >= 0.5 && t <= 1.0)) return OR_BAD_TAU;   /* Sec. 3 assumes t >= 0.5 */
    double x = ldexp(t, 48);                           /* exact */
    *tb = (uint64_t)ceil(x);
    *tu = (uint64_t)floor(x);
    return OR_OK;
}

static int check_k(int64_t m, const uint32_t* k) {
    for (int64_t i = 0; i < m; i++) if (k[i] > ONE16) return OR_BAD_PROB;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Exported entry points                                                     */
/* ------------------------------------------------------------------------ */

/* Number of triangles (-status on invalid input). */
int64_t ubto_num_triangles(int64_t n, int64_t m, const uint32_t* src, const uint32_t* dst) {
    fgraph g;
    int rc = fgraph_build(&g, n, m, src, dst);
    if (rc != OR_OK) return rc;
    int64_t t = for_each_triangle(&g, NULL, NULL);
    fgraph_free(&g);
    return t;
}

typedef struct { int64_t cap, n; uint32_t* vtx; uint32_t* eid; } list_ctx;
static void visit_list(void* c, const tri_t* t) {
    list_ctx* x = (list_ctx*)c;
    if (x->n < x->cap) {
        int64_t i = x->n;
        x->vtx[3 * i] = t->a; x->vtx[3 * i + 1] = t->b; x->vtx[3 * i + 2] = t->c;
        x->eid[3 * i] = t->e_ab; x->eid[3 * i + 1] = t->e_ac; x->eid[3 * i + 2] = t->e_bc;
    }
    x->n++;
}

/* Lists triangles: vtx[3i..3i+2] = (a<b<c), eid[3i..] = (e_ab, e_ac, e_bc).
 * Writes at most cap triangles; returns the total number (or -status). */
int64_t ubto_list(int64_t n, int64_t m, const uint32_t* src, const uint32_t* dst,
                  int64_t cap, uint32_t* vtx, uint32_t* eid) {
    fgraph g;
    int rc = fgraph_build(&g, n, m, src, dst);
    if (rc != OR_OK) return rc;
    list_ctx c = {cap, 0, vtx, eid};
    for_each_triangle(&g, visit_list, &c);
    fgraph_free(&g);
    return c.n;
}

typedef struct {
    const uint32_t* k;
    int n_tau;
    const uint64_t* tb;
    const uint64_t* tu;
    int64_t* bal;
    int64_t* unbal;
} count_ctx;
static void visit_count(void* c, const tri_t* t) {
    count_ctx* x = (count_ctx*)c;
    uint64_t nb = nbal_fixed(x->k[t->e_ab], x->k[t->e_ac], x->k[t->e_bc]);
    uint64_t nu = ONE48 - nb;          /* 2^48 * P_unbal */
    for (int i = 0; i < x->n_tau; i++) {
        if (nb >= x->tb[i]) x->bal[i]++;    /* P_bal >= t   (Def. 4; Alg. 1) */
        if (nu > x->tu[i]) x->unbal[i]++;   /* P_unbal > t  (Def. 5; Alg. 1) */
    }
}

/* Counting problem (Def. UBTC): counts of t-balanced and t-unbalanced
 * triangles for each of n_tau thresholds. */
int ubto_count_threshold(int64_t n, int64_t m, const uint32_t* src, const uint32_t* dst,
                         const uint32_t* k, int n_tau, const double* tau,
                         int64_t* bal, int64_t* unbal) {
    int rc = check_k(m, k);
    if (rc != OR_OK) return rc;
    if (n_tau < 0) return OR_BAD_TAU;
    uint64_t* tb = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n_tau + 1));
    uint64_t* tu = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n_tau + 1));
    if (!tb || !tu) { free(tb); free(tu); return OR_NOMEM; }
    for (int i = 0; i < n_tau; i++) {
        rc = tau_levels(tau[i], &tb[i], &tu[i]);
        if (rc != OR_OK) { free(tb); free(tu); return rc; }
        bal[i] = 0; unbal[i] = 0;
    }
    fgraph g;
    rc = fgraph_build(&g, n, m, src, dst);
    if (rc == OR_OK) {
        count_ctx c = {k, n_tau, tb, tu, bal, unbal};
        for_each_triangle(&g, visit_count, &c);
        fgraph_free(&g);
    }
    free(tb); free(tu);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* A built graph kept between queries, counted by several threads            */
/* ------------------------------------------------------------------------ */

/* The benchmark's CPU arm times queries on a graph already built, as the GPU
 * arm does: ubto_graph_new builds the forward lists once (validating the
 * edge list as fgraph_build does) and ubto_graph_count answers the counting
 * problem (Def. UBTC) on it.  The outer loop of Alg. 1 (over u) is split
 * among OpenMP threads; each thread counts into its own arrays, which are
 * added at the end, so the counts do not depend on the thread count.  With
 * sample_mod > 1 only the u with h(u) % sample_mod == sample_rem are visited,
 * h(u) = bits 40..63 of u * 0x9E3779B97F4A7C15 (a multiplicative hash, so that
 * a sample is spread over the id range): exactly the triangles whose earliest
 * vertex in Node Order is such a u (the samples rem = 0 .. mod-1 partition
 * the triangles). */
#ifdef _OPENMP
#include <omp.h>
#endif

int64_t ubto_sample_class(int64_t u, int64_t sample_mod) {
    return (int64_t)((((uint64_t)u * 0x9E3779B97F4A7C15ULL) >> 40) % (uint64_t)sample_mod);
}

int ubto_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void* ubto_graph_new(int64_t n, int64_t m, const uint32_t* src, const uint32_t* dst, int* status) {
    fgraph* g = (fgraph*)malloc(sizeof(fgraph));
    if (!g) { *status = OR_NOMEM; return NULL; }
    *status = fgraph_build(g, n, m, src, dst);
    if (*status != OR_OK) { free(g); return NULL; }
    return g;
}

void ubto_graph_free(void* g) {
    if (!g) return;
    fgraph_free((fgraph*)g);
    free(g);
}

/* Returns the number of triangles visited (or -status); bal / unbal as in
 * ubto_count_threshold, over the sampled u only. */
int64_t ubto_graph_count(void* gp, const uint32_t* k, int n_tau, const double* tau, int64_t sample_mod,
                         int64_t sample_rem, int threads, int64_t* bal, int64_t* unbal) {
    const fgraph* g = (const fgraph*)gp;
    int rc = check_k(g->m, k);
    if (rc != OR_OK) return rc;
    if (n_tau < 1 || sample_mod < 1 || sample_rem < 0 || sample_rem >= sample_mod) return OR_BAD_TAU;
    uint64_t* tb = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n_tau);
    uint64_t* tu = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n_tau);
    if (!tb || !tu) { free(tb); free(tu); return OR_NOMEM; }
    for (int i = 0; i < n_tau && rc == OR_OK; i++) rc = tau_levels(tau[i], &tb[i], &tu[i]);
    if (rc != OR_OK) { free(tb); free(tu); return rc; }
    for (int i = 0; i < n_tau; i++) { bal[i] = 0; unbal[i] = 0; }
    int64_t total = 0;
    if (threads < 1) threads = 1;
#pragma omp parallel num_threads(threads) reduction(+ : total)
    {
        int64_t* b = (int64_t*)calloc((size_t)n_tau, sizeof(int64_t));
        int64_t* u = (int64_t*)calloc((size_t)n_tau, sizeof(int64_t));
        count_ctx c = {k, n_tau, tb, tu, b, u};
        if (b && u) {
#pragma omp for schedule(dynamic, 64)
            for (int64_t x = 0; x < g->n; x++)
                if (ubto_sample_class(x, sample_mod) == sample_rem) total += triangles_from(g, x, visit_count, &c);
#pragma omp critical
            for (int i = 0; i < n_tau; i++) { bal[i] += b[i]; unbal[i] += u[i]; }
        } else {
#pragma omp critical
            rc = OR_NOMEM;
        }
        free(b); free(u);
    }
    free(tb); free(tu);
    return rc != OR_OK ? rc : total;
}

typedef struct {
    const uint32_t* k;
    uint64_t tb, tu;
    int which;
    int64_t cap, n;
    uint32_t* uvw;
    uint32_t* cls;
    double* pbal;
} enum_ctx;
static void visit_enum(void* c, const tri_t* t) {
    enum_ctx* x = (enum_ctx*)c;
    uint64_t nb = nbal_fixed(x->k[t->e_ab], x->k[t->e_ac], x->k[t->e_bc]);
    uint64_t nu = ONE48 - nb;
    uint32_t cl = 0;
    if ((x->which & 1) && nb >= x->tb) cl = 1;
    if ((x->which & 2) && nu > x->tu) cl = 2;
    if (!cl) return;
    if (x->n < x->cap) {
        int64_t i = x->n;
        x->uvw[3 * i] = t->a; x->uvw[3 * i + 1] = t->b; x->uvw[3 * i + 2] = t->c;
        x->cls[i] = cl;
        x->pbal[i] = ldexp((double)nb, -48);
    }
    x->n++;
}

/* Enumeration problem (Def. UBTE): which = 1 balanced, 2 unbalanced, 3 both.
 * Record i: uvw[3i..] = (a<b<c), cls[i] = 1 (balanced) or 2 (unbalanced),
 * pbal[i] = P_bal exactly.  Records come in listing order (callers sort).
 * Returns the total number of records (or -status); writes at most cap. */
int64_t ubto_enumerate(int64_t n, int64_t m, const uint32_t* src, const uint32_t* dst,
                       const uint32_t* k, double tau, int which, int64_t cap,
                       uint32_t* uvw, uint32_t* cls, double* pbal) {
    int rc = check_k(m, k);
    if (rc != OR_OK) return rc;
    uint64_t tb, tu;
    rc = tau_levels(tau, &tb, &tu);
    if (rc != OR_OK) return rc;
    fgraph g;
    rc = fgraph_build(&g, n, m, src, dst);
    if (rc != OR_OK) return rc;
    enum_ctx c = {k, tb, tu, which, cap, 0, uvw, cls, pbal};
    for_each_triangle(&g, visit_enum, &c);
    fgraph_free(&g);
    return c.n;
}

typedef struct { const uint32_t* k; int64_t t; unsigned __int128 s; } efix_ctx;
static void visit_efix(void* c, const tri_t* t) {
    efix_ctx* x = (efix_ctx*)c;
    x->s += nbal_fixed(x->k[t->e_ab], x->k[t->e_ac], x->k[t->e_bc]);
    x->t++;
}

/* Expected counts, fixed-point input, exactly:
 *   E_bal = (sum_t N_bal(t)) / 2^48,  E_unbal = T - E_bal.
 * Outputs T and the 128-bit sum of N_bal as (lo, hi) 64-bit words. */
int ubto_expected_fixed(int64_t n, int64_t m, const uint32_t* src, const uint32_t* dst,
                        const uint32_t* k, int64_t* tri, uint64_t* sum_lo, uint64_t* sum_hi) {
    int rc = check_k(m, k);
    if (rc != OR_OK) return rc;
    fgraph g;
    rc = fgraph_build(&g, n, m, src, dst);
    if (rc != OR_OK) return rc;
    efix_ctx c = {k, 0, 0};
    for_each_triangle(&g, visit_efix, &c);
    fgraph_free(&g);
    *tri = c.t;
    *sum_lo = (uint64_t)c.s;
    *sum_hi = (uint64_t)(c.s >> 64);
    return OR_OK;
}

/* P_bal of three real probabilities, four-term sum (equation in Sec. 3). */
static double pbal_real(double p1, double p2, double p3) {
    double n1 = 1.0 - p1, n2 = 1.0 - p2, n3 = 1.0 - p3;
    return p1 * p2 * p3 + p1 * n2 * n3 + n1 * p2 * n3 + n1 * n2 * p3;
}

/* Neumaier compensated sum */
typedef struct { double s, c; } csum;
static void csum_add(csum* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

typedef struct { const float* p; int64_t t; csum bal; } ereal_ctx;
static void visit_ereal(void* c, const tri_t* t) {
    ereal_ctx* x = (ereal_ctx*)c;
    csum_add(&x->bal, pbal_real(x->p[t->e_ab], x->p[t->e_ac], x->p[t->e_bc]));
    x->t++;
}

/* Expected counts for float32 probabilities, accumulated in double:
 * out[0] = E_bal, out[1] = E_unbal = T - E_bal, out[2] = T. */
int ubto_expected_real(int64_t n, int64_t m, const uint32_t* src, const uint32_t* dst,
                       const float* p, double* out) {
    for (int64_t i = 0; i < m; i++) if (!(p[i] >= 0.0f && p[i] <= 1.0f)) return OR_BAD_PROB;
    fgraph g;
    int rc = fgraph_build(&g, n, m, src, dst);
    if (rc != OR_OK) return rc;
    ereal_ctx c = {p, 0, {0.0, 0.0}};
    for_each_triangle(&g, visit_ereal, &c);
    fgraph_free(&g);
    double eb = c.bal.s + c.bal.c;
    out[0] = eb;
    out[1] = (double)c.t - eb;
    out[2] = (double)c.t;
    return OR_OK;
}

/* dP_bal/dp1 of the four-term sum, term by term:
 *   d/dp1 [p1 p2 p3 + p1 n2 n3 + n1 p2 n3 + n1 n2 p3]
 *     = p2 p3 + n2 n3 - p2 n3 - n2 p3                                        */
static double dpbal_dp1(double p2, double p3) {
    double n2 = 1.0 - p2, n3 = 1.0 - p3;
    return p2 * p3 + n2 * n3 - p2 * n3 - n2 * p3;
}

typedef struct { const float* p; double* g; double* gabs; } grad_ctx;
static void visit_grad(void* c, const tri_t* t) {
    grad_ctx* x = (grad_ctx*)c;
    double pab = x->p[t->e_ab], pac = x->p[t->e_ac], pbc = x->p[t->e_bc];
    double dab = dpbal_dp1(pac, pbc);
    double dac = dpbal_dp1(pab, pbc);
    double dbc = dpbal_dp1(pab, pac);
    x->g[t->e_ab] += dab; x->g[t->e_ac] += dac; x->g[t->e_bc] += dbc;
    if (x->gabs) {
        x->gabs[t->e_ab] += fabs(dab); x->gabs[t->e_ac] += fabs(dac); x->gabs[t->e_bc] += fabs(dbc);
    }
}

/* Analytic gradient of E_bal with respect to every p_e (input edge order):
 * grad[e] = sum over triangles through e of dP_bal/dp_e; dE_unbal/dp_e is
 * its negation.  gabs (optional) receives sum of |dP_bal/dp_e|. */
int ubto_grad_real(int64_t n, int64_t m, const uint32_t* src, const uint32_t* dst,
                   const float* p, double* grad, double* gabs) {
    for (int64_t i = 0; i < m; i++) {
        grad[i] = 0.0;
        if (gabs) gabs[i] = 0.0;
    }
    fgraph g;
    int rc = fgraph_build(&g, n, m, src, dst);
    if (rc != OR_OK) return rc;
    grad_ctx c = {p, grad, gabs};
    for_each_triangle(&g, visit_grad, &c);
    fgraph_free(&g);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Local counts (the quantities the samplers of Sec. 6 estimate from)        */
/* ------------------------------------------------------------------------ */

typedef struct {
    const uint32_t* k;
    int n_tau;
    const uint64_t* tb;
    const uint64_t* tu;
    int64_t* ebal;
    int64_t* eunb;
    int64_t* vbal;
    int64_t* vunb;
} local_ctx;
static void visit_local(void* c, const tri_t* t) {
    local_ctx* x = (local_ctx*)c;
    uint64_t nb = nbal_fixed(x->k[t->e_ab], x->k[t->e_ac], x->k[t->e_bc]);
    uint64_t nu = ONE48 - nb;
    const uint32_t es[3] = {t->e_ab, t->e_ac, t->e_bc};
    const uint32_t vs[3] = {t->a, t->b, t->c};
    for (int i = 0; i < x->n_tau; i++) {
        int b = nb >= x->tb[i], u = nu > x->tu[i];
        for (int j = 0; j < 3; j++) {
            if (x->ebal && b) x->ebal[(int64_t)es[j] * x->n_tau + i]++;
            if (x->eunb && u) x->eunb[(int64_t)es[j] * x->n_tau + i]++;
            if (x->vbal && b) x->vbal[(int64_t)vs[j] * x->n_tau + i]++;
            if (x->vunb && u) x->vunb[(int64_t)vs[j] * x->n_tau + i]++;
        }
    }
}

/* Local counts for every edge and every vertex: the number of t-balanced /
 * t-unbalanced triangles that contain it (|B_t(e)|, |B_t(v)| of Sec. 6),
 * for each of n_tau thresholds.  Every triangle is listed once (Alg. 1) and
 * credited to its three edges and three vertices.  Arrays are [item][tau]
 * (edges in input order); any of them may be NULL. */
int ubto_local_counts(int64_t n, int64_t m, const uint32_t* src, const uint32_t* dst,
                      const uint32_t* k, int n_tau, const double* tau, int64_t* edge_bal,
                      int64_t* edge_unbal, int64_t* vtx_bal, int64_t* vtx_unbal) {
    int rc = check_k(m, k);
    if (rc != OR_OK) return rc;
    if (n_tau < 1) return OR_BAD_TAU;
    uint64_t* tb = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n_tau);
    uint64_t* tu = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n_tau);
    if (!tb || !tu) { free(tb); free(tu); return OR_NOMEM; }
    for (int i = 0; i < n_tau && rc == OR_OK; i++) rc = tau_levels(tau[i], &tb[i], &tu[i]);
    if (rc == OR_OK) {
        if (edge_bal) memset(edge_bal, 0, sizeof(int64_t) * (size_t)(m * n_tau));
        if (edge_unbal) memset(edge_unbal, 0, sizeof(int64_t) * (size_t)(m * n_tau));
        if (vtx_bal) memset(vtx_bal, 0, sizeof(int64_t) * (size_t)(n * n_tau));
        if (vtx_unbal) memset(vtx_unbal, 0, sizeof(int64_t) * (size_t)(n * n_tau));
        fgraph g;
        rc = fgraph_build(&g, n, m, src, dst);
        if (rc == OR_OK) {
            local_ctx c = {k, n_tau, tb, tu, edge_bal, edge_unbal, vtx_bal, vtx_unbal};
            for_each_triangle(&g, visit_local, &c);
            fgraph_free(&g);
        }
    }
    free(tb); free(tu);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon et al., SC'11)                                      */
/* ------------------------------------------------------------------------ */

/* Round multipliers and Weyl key increments published with Philox4x64. */
#define PHILOX_M0 0xD2E7470EE14C6C93ULL
#define PHILOX_M1 0xCA5A826395121157ULL
#define PHILOX_W0 0x9E3779B97F4A7C15ULL
#define PHILOX_W1 0xBB67AE8584CAA73BULL

static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
    unsigned __int128 r = (unsigned __int128)a * b;
    *lo = (uint64_t)r;
    *hi = (uint64_t)(r >> 64);
}

/* One Philox4x64 bijection with 10 rounds: each round multiplies words 0 and
 * 2 by the two constants, and the new state is (hi(M1*x2) ^ x1 ^ k0,
 * lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0)); the key is bumped by the Weyl
 * increments between rounds. */
void ubto_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(PHILOX_M0, x0, &hi0, &lo0);
        mulhilo64(PHILOX_M1, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y1 = lo1;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        uint64_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Sign draws of one edge in 64 consecutive worlds.
 *
 * World j of word w (global world index 64 w + j), edge with key `ekey`:
 * sixteen 64-bit words r_0..r_15 come from four Philox4x64-10 calls with key
 * (seed, 0) and counters (ekey, w, c, 0), c = 0..3, call c giving r_{4c..4c+3}.
 * The world's 16-bit uniform is u_j = sum_b ((r_b >> j) & 1) << b, and the
 * edge is positive in that world iff u_j < k (so P(+) = k / 65536 exactly).
 * Bit j of the result is 1 iff the edge is positive in world 64 w + j. */
uint64_t ubto_world_word(uint64_t seed, uint32_t ekey, uint32_t w, uint32_t k) {
    uint64_t r[16];
    uint64_t key[2] = {seed, 0};
    for (uint32_t c = 0; c < 4; c++) {
        uint64_t ctr[4] = {ekey, w, c, 0};
        ubto_philox4x64_10(ctr, key, r + 4 * c);
    }
    uint64_t word = 0;
    for (int j = 0; j < 64; j++) {
        uint32_t u = 0;
        for (int b = 0; b < 16; b++) u |= (uint32_t)((r[b] >> j) & 1u) << b;
        if (u < k) word |= 1ULL << j;
    }
    return word;
}

typedef struct {
    const uint64_t* signs;   /* m x n_words table of world words */
    int n_words;
    int64_t* counts;         /* n_words * 64 */
} world_ctx;
static void visit_world(void* c, const tri_t* t) {
    world_ctx* x = (world_ctx*)c;
    const uint64_t* a = x->signs + (size_t)t->e_ab * x->n_words;
    const uint64_t* b = x->signs + (size_t)t->e_ac * x->n_words;
    const uint64_t* d = x->signs + (size_t)t->e_bc * x->n_words;
    for (int w = 0; w < x->n_words; w++) {
        for (int j = 0; j < 64; j++) {
            int pos = (int)((a[w] >> j) & 1u) + (int)((b[w] >> j) & 1u) + (int)((d[w] >> j) & 1u);
            if (pos & 1) x->counts[(size_t)w * 64 + j]++;   /* odd # of '+' = balanced (Def. 3) */
        }
    }
}

/* Per-world balanced-triangle counts for the worlds of the listed words:
 * counts[i*64 + j] = number of triangles balanced in world 64*words[i] + j.
 * ekey (optional) gives the Philox key of each edge (default: edge index). */
int ubto_world_counts(int64_t n, int64_t m, const uint32_t* src, const uint32_t* dst,
                      const uint32_t* k, const uint32_t* ekey, uint64_t seed,
                      int n_words, const uint32_t* words, int64_t* counts) {
    int rc = check_k(m, k);
    if (rc != OR_OK) return rc;
    uint64_t* signs = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1) * (size_t)(n_words > 0 ? n_words : 1));
    if (!signs) return OR_NOMEM;
    for (int64_t e = 0; e < m; e++)
        for (int i = 0; i < n_words; i++)
            signs[(size_t)e * n_words + i] = ubto_world_word(seed, ekey ? ekey[e] : (uint32_t)e, words[i], k[e]);
    for (int64_t i = 0; i < (int64_t)n_words * 64; i++) counts[i] = 0;
    fgraph g;
    rc = fgraph_build(&g, n, m, src, dst);
    if (rc == OR_OK) {
        world_ctx c = {signs, n_words, counts};
        for_each_triangle(&g, visit_world, &c);
        fgraph_free(&g);
    }
    free(signs);
    return rc;
}
