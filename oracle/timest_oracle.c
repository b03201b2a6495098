/*
 * TIMEST CPU oracle (arXiv 2507.20441) -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the package smoke check and the benchmark's CPU
 * baseline / reference arm may load this file.  The product path (the CUDA
 * library) never calls it, shares no code, header, table or helper with it,
 * and fails loudly when its own extension is missing.
 *
 * This is a plain, slow, obviously-correct restatement of the paper:
 *
 *   O1  or_brute_count      exact count C of M-matches by chronological
 *                           backtracking over the definition (Def. 1.2).
 *   O2  or_partial_count    brute-force count of delta-partial matches of the
 *                           spanning tree inside one 2*delta window
 *                           (Def. of delta-partial match, Sec. 3; Constraint 3).
 *   O3  or_weights/or_sample  TIMEST itself: the weight DP (Claims 3.2-3.4,
 *                           Alg. 1-2), the sampler (Alg. 3, Sec. 3.2), the
 *                           validator and DeriveCnt (Alg. 4-5) and the
 *                           estimate (Alg. 6).
 *   O4  or_exact_by_trees   exact C as the sum over every partial match of
 *                           cnt(phi)/N_phi (proof of Lemma 3.6).
 *
 * Readings of the paper where it is silent, garbled or inconsistent (each one
 * is listed in the design notes as well):
 *   R1  t' = t - t_min (Sec. 3 preamble).  Windows are half-open
 *       [i*delta, (i+2)*delta) in t', i = 0..floor(T/delta), T = max t'.
 *   R2  Constraint 1 is strict on the order side and inclusive on delta: a
 *       child that comes later in pi lies in (t, t+delta], an earlier child
 *       in [t-delta, t).
 *   R3  Parent/child ("dependent") edges are defined by rooting the tree at
 *       the root edge c; both endpoints of c are lower endpoints.  The
 *       candidate list of child s' meeting s at motif vertex z is the z-side
 *       out-list (s' leaves z) or in-list (s' enters z) minus the multi-edge
 *       list between phi(z) and the image of the other endpoint of s, in the
 *       direction of s' (Claim 3.1).  Claim 3.2 reads L_{e,s,s_i} in factor i.
 *   R4  N_phi = number of windows that contain every tree edge of phi.
 *   R5  Draw protocol: Philox4x32-10 with key (seed_lo, seed_hi) and counter
 *       (j_lo, j_hi, d, 0), j the global sample index and d the per-sample
 *       attempt counter.  U[0,n): n<=1 -> 0 without a draw; otherwise mask
 *       the low bitlen(n-1) bits of the block's low 64 (or all 128) bits and
 *       accept if < n.  Draw order: the root (window then edge over the
 *       (layer, window, GLOBAL order) concatenation), then the tree edges in
 *       breadth-first order from c (children of c at its source endpoint, then
 *       at its destination endpoint; increasing motif-edge index within a
 *       vertex).  Candidate lists are in (t', other endpoint) order.
 *   R6  contribution = cnt * (2 / N_phi); hits2 = sum of contributions;
 *       estimate = W * hits2 / (2k).  Reject priority vertex > delta > order
 *       (Alg. 4).
 *   R7  Weights are exact unsigned 64-bit integers; any candidate-list sum,
 *       product or per-window root total >= 2^64 is reported as overflow.
 *   R8  Constraint toggles of the ablation (Table of constraints):
 *       Constraint 1 always holds; without Constraint 2 the candidate list
 *       keeps the multi-edges to the parent's other endpoint; without
 *       Constraint 3 a single window [0, 2^34) holds every edge (window unit
 *       2^33 > any t' span), so every N_phi is 1.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

enum {
    OR_OK = 0, OR_E_ARG = 1, OR_E_DUP = 2, OR_E_SELFLOOP = 3, OR_E_MOTIF = 4,
    OR_E_NOMEM = 5, OR_E_OVERFLOW = 6, OR_E_STATE = 7, OR_E_LIMIT = 8
};
enum { OR_DEDUP = 1, OR_DROP_SELF = 2 };
enum { OR_MAXV = 8, OR_MAXE = 16 };
#define OR_WD_OFF ((int64_t)1 << 33)   /* window unit without Constraint 3: above any t' span */
#define OR_NO_VERTEX 0xFFFFFFFFu        /* never a vertex id (n < 2^32 - 1)             */
enum { RS_VALID = 0, RS_VERTEX = 1, RS_DELTA = 2, RS_ORDER = 3 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, restated from Salmon, Moraes, Dror and Shaw, "Parallel     */
/* Random Numbers: As Easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64  */
/* multiplications whose high halves are xored with the other counter words  */
/* and the round key; the key is bumped by the two Weyl constants between    */
/* rounds.                                                                   */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

typedef struct { uint64_t seed, j; uint32_t d; } draw_state;

static void next_block(draw_state *s, uint32_t out[4])
{
    uint32_t ctr[4] = { (uint32_t)s->j, (uint32_t)(s->j >> 32), s->d, 0u };
    uint32_t key[2] = { (uint32_t)s->seed, (uint32_t)(s->seed >> 32) };
    s->d += 1;
    or_philox4x32_10(ctr, key, out);
}

static int bitlen64(uint64_t x) { int b = 0; while (x) { ++b; x >>= 1; } return b; }
static int bitlen128(u128 x) { int b = 0; while (x) { ++b; x >>= 1; } return b; }

/* Uniform integer in [0, n) by masked rejection (R5). */
static uint64_t uniform_u64(draw_state *s, uint64_t n)
{
    if (n <= 1) return 0;
    int b = bitlen64(n - 1);
    uint64_t mask = (b >= 64) ? ~(uint64_t)0 : (((uint64_t)1 << b) - 1);
    for (;;) {
        uint32_t blk[4];
        next_block(s, blk);
        uint64_t x = ((uint64_t)blk[0] | ((uint64_t)blk[1] << 32)) & mask;
        if (x < n) return x;
    }
}

static u128 uniform_u128(draw_state *s, u128 n)
{
    if (n <= 1) return 0;
    int b = bitlen128(n - 1);
    u128 mask = (b >= 128) ? ~(u128)0 : ((((u128)1) << b) - 1);
    for (;;) {
        uint32_t blk[4];
        next_block(s, blk);
        u128 x = (u128)blk[0] | ((u128)blk[1] << 32) | ((u128)blk[2] << 64) | ((u128)blk[3] << 96);
        x &= mask;
        if (x < n) return x;
    }
}

/* Exposed for the generator pins: the k-th value of U[0,n) for sample j. */
uint64_t or_uniform_u64(uint64_t seed, uint64_t j, uint32_t d0, uint64_t n, uint32_t *d_after)
{
    draw_state s = { seed, j, d0 };
    uint64_t x = uniform_u64(&s, n);
    if (d_after) *d_after = s.d;
    return x;
}

/* ------------------------------------------------------------------------ */
/* Graph: the edge set sorted four ways (Sec. 3 preamble; Defs. 3.1-3.3).   */
/* GLOBAL order (t', src, dst) defines the edge id "gid" used everywhere.   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n, m;
    int64_t tmin, T;               /* T = max t' */
    uint32_t *src, *dst;           /* by gid */
    int64_t *t;                    /* t' by gid */
    int64_t *out_beg; uint32_t *out_gid;   /* per vertex, (t', dst) order  */
    int64_t *in_beg;  uint32_t *in_gid;    /* per vertex, (t', src) order  */
    int64_t npairs;
    uint32_t *pair_src, *pair_dst;         /* pairs sorted by (src, dst)    */
    int64_t *pair_beg; uint32_t *pair_gid; /* multi-edge list, t' order     */
} or_graph;

typedef struct {
    int nv, ne;
    int a[OR_MAXE], b[OR_MAXE], rank[OR_MAXE];
    int pos_edge[OR_MAXE];
    int64_t delta;
    int64_t wd;                    /* window unit: delta, or OR_WD_OFF without Constraint 3 */
    int c2;                        /* 1: Constraint 2 (distinct far endpoints) enforced     */
    int is_tree[OR_MAXE];
    int root, ntree;
    int order[OR_MAXV];            /* tree edges, breadth-first from root  */
    int parent[OR_MAXE];           /* parent tree edge (-1 for the root)   */
    int meet[OR_MAXE];             /* motif vertex shared with the parent  */
    int nchild[OR_MAXE];
    int child[OR_MAXE][OR_MAXE];
    int height[OR_MAXE];
} or_plan;

typedef struct {
    or_graph g;
    or_plan P;
    int have_plan, have_weights;
    uint64_t *w[OR_MAXE][2];       /* w[s][layer][gid]; NULL for leaves   */
    int64_t nwin;                  /* floor(T/delta)+1 windows            */
    uint64_t *Wi;                  /* per window i                        */
    uint64_t *rootcum[2];          /* running sum of w_c inside each window */
    u128 W;
} or_ctx;

typedef struct {
    uint64_t W_lo, W_hi, hits2_lo, hits2_hi;
    uint64_t k, valid, rej_vertex, rej_delta, rej_order;
    double estimate;
} or_result;

/* sort helpers (qsort over gid with a file-scope view of the arrays) */
static const uint32_t *cmp_src, *cmp_dst;
static const int64_t *cmp_t;
static int cmp_global(const void *x, const void *y)
{
    uint32_t i = *(const uint32_t *)x, j = *(const uint32_t *)y;
    if (cmp_t[i] != cmp_t[j]) return cmp_t[i] < cmp_t[j] ? -1 : 1;
    if (cmp_src[i] != cmp_src[j]) return cmp_src[i] < cmp_src[j] ? -1 : 1;
    if (cmp_dst[i] != cmp_dst[j]) return cmp_dst[i] < cmp_dst[j] ? -1 : 1;
    return 0;
}
static int cmp_out(const void *x, const void *y)
{
    uint32_t i = *(const uint32_t *)x, j = *(const uint32_t *)y;
    if (cmp_src[i] != cmp_src[j]) return cmp_src[i] < cmp_src[j] ? -1 : 1;
    if (cmp_t[i] != cmp_t[j]) return cmp_t[i] < cmp_t[j] ? -1 : 1;
    if (cmp_dst[i] != cmp_dst[j]) return cmp_dst[i] < cmp_dst[j] ? -1 : 1;
    return 0;
}
static int cmp_in(const void *x, const void *y)
{
    uint32_t i = *(const uint32_t *)x, j = *(const uint32_t *)y;
    if (cmp_dst[i] != cmp_dst[j]) return cmp_dst[i] < cmp_dst[j] ? -1 : 1;
    if (cmp_t[i] != cmp_t[j]) return cmp_t[i] < cmp_t[j] ? -1 : 1;
    if (cmp_src[i] != cmp_src[j]) return cmp_src[i] < cmp_src[j] ? -1 : 1;
    return 0;
}
static int cmp_multi(const void *x, const void *y)
{
    uint32_t i = *(const uint32_t *)x, j = *(const uint32_t *)y;
    if (cmp_src[i] != cmp_src[j]) return cmp_src[i] < cmp_src[j] ? -1 : 1;
    if (cmp_dst[i] != cmp_dst[j]) return cmp_dst[i] < cmp_dst[j] ? -1 : 1;
    if (cmp_t[i] != cmp_t[j]) return cmp_t[i] < cmp_t[j] ? -1 : 1;
    return 0;
}

static void free_weights(or_ctx *C)
{
    for (int s = 0; s < OR_MAXE; ++s)
        for (int p = 0; p < 2; ++p) { free(C->w[s][p]); C->w[s][p] = NULL; }
    free(C->Wi); C->Wi = NULL;
    free(C->rootcum[0]); free(C->rootcum[1]); C->rootcum[0] = C->rootcum[1] = NULL;
    C->have_weights = 0;
}

void or_free(or_ctx *C)
{
    if (!C) return;
    free_weights(C);
    or_graph *g = &C->g;
    free(g->src); free(g->dst); free(g->t);
    free(g->out_beg); free(g->out_gid); free(g->in_beg); free(g->in_gid);
    free(g->pair_src); free(g->pair_dst); free(g->pair_beg); free(g->pair_gid);
    free(C);
}

/* Build the oracle graph from raw tuples (u, v, t); Sec. 1.1 input contract. */
int or_create(int64_t n, int64_t m, const uint32_t *src, const uint32_t *dst,
              const int64_t *t, int flags, or_ctx **out)
{
    *out = NULL;
    if (n <= 0 || m < 0 || n > 0xFFFFFFF0LL || m > 0xFFFFFFF0LL) return OR_E_ARG;
    or_ctx *C = (or_ctx *)calloc(1, sizeof(or_ctx));
    if (!C) return OR_E_NOMEM;
    or_graph *g = &C->g;
    g->n = n;
    /* drop or reject self loops */
    uint32_t *s0 = malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t *d0 = malloc(sizeof(uint32_t) * (m ? m : 1));
    int64_t *t0 = malloc(sizeof(int64_t) * (m ? m : 1));
    int64_t mm = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (src[i] >= (uint64_t)n || dst[i] >= (uint64_t)n) { free(s0); free(d0); free(t0); free(C); return OR_E_ARG; }
        if (src[i] == dst[i]) {
            if (flags & OR_DROP_SELF) continue;
            free(s0); free(d0); free(t0); free(C); return OR_E_SELFLOOP;
        }
        s0[mm] = src[i]; d0[mm] = dst[i]; t0[mm] = t[i]; ++mm;
    }
    int64_t tmin = 0, tmax = 0;
    for (int64_t i = 0; i < mm; ++i) {
        if (i == 0 || t0[i] < tmin) tmin = t0[i];
        if (i == 0 || t0[i] > tmax) tmax = t0[i];
    }
    if (mm > 0 && (tmax - tmin) >= 0xFFFFFFFFLL) { free(s0); free(d0); free(t0); free(C); return OR_E_ARG; }
    for (int64_t i = 0; i < mm; ++i) t0[i] -= tmin;
    /* GLOBAL order and duplicate handling */
    uint32_t *idx = malloc(sizeof(uint32_t) * (mm ? mm : 1));
    for (int64_t i = 0; i < mm; ++i) idx[i] = (uint32_t)i;
    cmp_src = s0; cmp_dst = d0; cmp_t = t0;
    qsort(idx, (size_t)mm, sizeof(uint32_t), cmp_global);
    int64_t mu = 0;
    for (int64_t i = 0; i < mm; ++i) {
        if (i > 0 && cmp_global(&idx[i], &idx[i - 1]) == 0) {
            if (flags & OR_DEDUP) continue;
            free(idx); free(s0); free(d0); free(t0); free(C); return OR_E_DUP;
        }
        idx[mu++] = idx[i];
    }
    g->m = mu;
    g->tmin = mm ? tmin : 0;
    size_t M1 = (size_t)(mu ? mu : 1);
    g->src = malloc(sizeof(uint32_t) * M1);
    g->dst = malloc(sizeof(uint32_t) * M1);
    g->t = malloc(sizeof(int64_t) * M1);
    g->T = 0;
    for (int64_t i = 0; i < mu; ++i) {
        g->src[i] = s0[idx[i]]; g->dst[i] = d0[idx[i]]; g->t[i] = t0[idx[i]];
        if (g->t[i] > g->T) g->T = g->t[i];
    }
    free(idx); free(s0); free(d0); free(t0);
    /* out-lists, in-lists, multi-edge lists */
    cmp_src = g->src; cmp_dst = g->dst; cmp_t = g->t;
    g->out_gid = malloc(sizeof(uint32_t) * M1);
    g->in_gid = malloc(sizeof(uint32_t) * M1);
    g->pair_gid = malloc(sizeof(uint32_t) * M1);
    for (int64_t i = 0; i < mu; ++i) g->out_gid[i] = g->in_gid[i] = g->pair_gid[i] = (uint32_t)i;
    qsort(g->out_gid, (size_t)mu, sizeof(uint32_t), cmp_out);
    qsort(g->in_gid, (size_t)mu, sizeof(uint32_t), cmp_in);
    qsort(g->pair_gid, (size_t)mu, sizeof(uint32_t), cmp_multi);
    g->out_beg = calloc((size_t)n + 1, sizeof(int64_t));
    g->in_beg = calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t i = 0; i < mu; ++i) { g->out_beg[g->src[i] + 1]++; g->in_beg[g->dst[i] + 1]++; }
    for (int64_t v = 0; v < n; ++v) { g->out_beg[v + 1] += g->out_beg[v]; g->in_beg[v + 1] += g->in_beg[v]; }
    int64_t np = 0;
    for (int64_t i = 0; i < mu; ++i) {
        uint32_t e = g->pair_gid[i], f = i ? g->pair_gid[i - 1] : 0;
        if (i == 0 || g->src[e] != g->src[f] || g->dst[e] != g->dst[f]) ++np;
    }
    g->npairs = np;
    g->pair_src = malloc(sizeof(uint32_t) * (np ? np : 1));
    g->pair_dst = malloc(sizeof(uint32_t) * (np ? np : 1));
    g->pair_beg = malloc(sizeof(int64_t) * (np + 1));
    np = 0;
    for (int64_t i = 0; i < mu; ++i) {
        uint32_t e = g->pair_gid[i], f = i ? g->pair_gid[i - 1] : 0;
        if (i == 0 || g->src[e] != g->src[f] || g->dst[e] != g->dst[f]) {
            g->pair_src[np] = g->src[e]; g->pair_dst[np] = g->dst[e]; g->pair_beg[np] = i; ++np;
        }
    }
    g->pair_beg[np] = mu;
    *out = C;
    return OR_OK;
}

int64_t or_num_edges(const or_ctx *C) { return C->g.m; }
int64_t or_time_min(const or_ctx *C) { return C->g.tmin; }
int64_t or_time_span(const or_ctx *C) { return C->g.T; }

/* Export the GLOBAL order (t', src, dst) so tests can index by gid. */
void or_export_edges(const or_ctx *C, uint32_t *src, uint32_t *dst, int64_t *tprime)
{
    for (int64_t i = 0; i < C->g.m; ++i) { src[i] = C->g.src[i]; dst[i] = C->g.dst[i]; tprime[i] = C->g.t[i]; }
}

/* Multi-edge list El_{u,v} (Def. 3.2): returns [beg, end) in pair_gid, or an empty range. */
static void pair_range(const or_graph *g, uint32_t u, uint32_t v, int64_t *beg, int64_t *end)
{
    int64_t lo = 0, hi = g->npairs;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (g->pair_src[mid] < u || (g->pair_src[mid] == u && g->pair_dst[mid] < v)) lo = mid + 1;
        else hi = mid;
    }
    if (lo < g->npairs && g->pair_src[lo] == u && g->pair_dst[lo] == v) { *beg = g->pair_beg[lo]; *end = g->pair_beg[lo + 1]; }
    else { *beg = 0; *end = 0; }
}

/* First position in list[beg,end) (time-sorted gids) with t' >= x. */
static int64_t lower_time(const or_graph *g, const uint32_t *list, int64_t beg, int64_t end, int64_t x)
{
    int64_t lo = beg, hi = end;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->t[list[mid]] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* ------------------------------------------------------------------------ */
/* Motif and spanning tree (Defs. 1.1, 3.4-3.5)                              */
/* ------------------------------------------------------------------------ */
static int other_end(const or_plan *P, int e, int z) { return P->a[e] == z ? P->b[e] : P->a[e]; }

int or_set_motif(or_ctx *C, int nv, int ne, const int32_t *ea, const int32_t *eb,
                 const int32_t *rank, int64_t delta, const int32_t *tree_edges, int root)
{
    free_weights(C);
    C->have_plan = 0;
    or_plan *P = &C->P;
    memset(P, 0, sizeof(*P));
    if (nv < 2 || nv > OR_MAXV || ne < nv - 1 || ne > OR_MAXE || delta <= 0) return OR_E_MOTIF;
    P->nv = nv; P->ne = ne; P->delta = delta;
    P->wd = delta; P->c2 = 1;
    int seen_rank[OR_MAXE] = {0};
    for (int i = 0; i < ne; ++i) {
        if (ea[i] < 0 || ea[i] >= nv || eb[i] < 0 || eb[i] >= nv || ea[i] == eb[i]) return OR_E_MOTIF;
        if (rank[i] < 0 || rank[i] >= ne || seen_rank[rank[i]]) return OR_E_MOTIF;
        seen_rank[rank[i]] = 1;
        P->a[i] = ea[i]; P->b[i] = eb[i]; P->rank[i] = rank[i];
        P->pos_edge[rank[i]] = i;
    }
    /* tree: nv-1 distinct edges, connected and acyclic on the undirected graph */
    P->ntree = nv - 1;
    int comp[OR_MAXV];
    for (int v = 0; v < nv; ++v) comp[v] = v;
    for (int k = 0; k < nv - 1; ++k) {
        int e = tree_edges[k];
        if (e < 0 || e >= ne || P->is_tree[e]) return OR_E_MOTIF;
        P->is_tree[e] = 1;
        int ca = comp[P->a[e]], cb = comp[P->b[e]];
        if (ca == cb) return OR_E_MOTIF;
        for (int v = 0; v < nv; ++v) if (comp[v] == cb) comp[v] = ca;
    }
    if (root < 0 || root >= ne || !P->is_tree[root]) return OR_E_MOTIF;
    P->root = root;
    /* root the tree at edge c: breadth-first, children of c at its source
     * endpoint then at its destination endpoint, increasing edge index. */
    for (int e = 0; e < ne; ++e) { P->parent[e] = -1; P->meet[e] = -1; P->nchild[e] = 0; }
    int head = 0, tail = 0;
    int placed[OR_MAXE] = {0};
    P->order[tail++] = root; placed[root] = 1;
    while (head < tail) {
        int s = P->order[head++];
        int zs[2]; int nz;
        if (s == root) { zs[0] = P->a[s]; zs[1] = P->b[s]; nz = 2; }
        else { zs[0] = other_end(P, s, P->meet[s]); nz = 1; }
        for (int q = 0; q < nz; ++q) {
            int z = zs[q];
            for (int e = 0; e < ne; ++e) {
                if (!P->is_tree[e] || placed[e]) continue;
                if (P->a[e] != z && P->b[e] != z) continue;
                placed[e] = 1;
                P->parent[e] = s; P->meet[e] = z;
                P->child[s][P->nchild[s]++] = e;
                P->order[tail++] = e;
            }
        }
    }
    if (tail != nv - 1) return OR_E_MOTIF;
    for (int q = nv - 2; q >= 0; --q) {
        int s = P->order[q], h = 0;
        for (int c = 0; c < P->nchild[s]; ++c) { int hc = P->height[P->child[s][c]] + 1; if (hc > h) h = hc; }
        P->height[s] = h;
    }
    C->nwin = C->g.T / delta + 1;
    C->have_plan = 1;
    return OR_OK;
}

/* Constraint toggles for the ablation (R8): c2 = 0 drops Constraint 2 (a
 * child's candidate list keeps the multi-edges to the parent's other
 * endpoint); c3 = 0 drops Constraint 3 (one window holds every edge, so
 * N_phi = 1).  Constraint 1 always holds.  Weights must be recomputed. */
int or_set_constraints(or_ctx *C, int c2, int c3)
{
    if (!C->have_plan) return OR_E_STATE;
    free_weights(C);
    C->P.c2 = c2 ? 1 : 0;
    C->P.wd = c3 ? C->P.delta : OR_WD_OFF;
    C->nwin = C->g.T / C->P.wd + 1;
    return OR_OK;
}

/* sampling order and parents, for tests that read the plan */
void or_plan_info(const or_ctx *C, int32_t *order, int32_t *parent, int32_t *meet, int32_t *height)
{
    const or_plan *P = &C->P;
    for (int q = 0; q < P->ntree; ++q) order[q] = P->order[q];
    for (int e = 0; e < P->ne; ++e) { parent[e] = P->parent[e]; meet[e] = P->meet[e]; height[e] = P->height[e]; }
}

/* ------------------------------------------------------------------------ */
/* Candidate list L_{e,s,s'} (Claim 3.1 with R2/R3), restricted to window i  */
/* ------------------------------------------------------------------------ */
typedef struct {
    const uint32_t *list; int64_t beg, end;   /* time-sorted gids of phi(z)'s list */
    uint32_t excl;                            /* image of the parent's other endpoint */
    int use_src_as_nbr;                       /* in-list: neighbour is the source   */
} cand_range;

/* Given tree edge s matched to graph edge e (gid ge) in window i, describe the
 * candidate range of child c.  Returns 0 if the time interval is empty. */
static int child_candidates(const or_ctx *C, int s, uint32_t ge, int c, int64_t wi, cand_range *R)
{
    const or_graph *g = &C->g; const or_plan *P = &C->P;
    int64_t d = P->delta, te = g->t[ge];
    int z = P->meet[c];
    int o = other_end(P, s, z);                 /* the other endpoint of s */
    uint32_t zg = (P->a[s] == z) ? g->src[ge] : g->dst[ge];
    uint32_t og = (P->a[s] == o) ? g->src[ge] : g->dst[ge];
    int64_t lo, hi;                              /* inclusive t' range */
    if (P->rank[c] > P->rank[s]) { lo = te + 1; hi = te + d; }
    else { lo = te - d; hi = te - 1; }
    int64_t wlo = wi * P->wd, whi = (wi + 2) * P->wd - 1;
    if (lo < wlo) lo = wlo;
    if (hi > whi) hi = whi;
    if (lo > hi) return 0;
    int out_dir = (P->a[c] == z);               /* s' leaves phi(z) */
    const uint32_t *list = out_dir ? g->out_gid : g->in_gid;
    const int64_t *beg = out_dir ? g->out_beg : g->in_beg;
    R->list = list;
    R->beg = lower_time(g, list, beg[zg], beg[zg + 1], lo);
    R->end = lower_time(g, list, R->beg, beg[zg + 1], hi + 1);
    R->excl = P->c2 ? og : OR_NO_VERTEX;       /* without C2 nothing is excluded */
    R->use_src_as_nbr = !out_dir;
    return R->beg < R->end;
}

static uint32_t cand_nbr(const or_graph *g, const cand_range *R, int64_t pos)
{
    uint32_t x = R->list[pos];
    return R->use_src_as_nbr ? g->src[x] : g->dst[x];
}

static int64_t window_of(int64_t tp, int p, int64_t d)
{
    /* window of layer p holding t', or -1 (R1) */
    if (tp < p * d) return -1;
    return p + 2 * ((tp - p * d) / (2 * d));
}

static uint64_t child_weight(const or_ctx *C, int c, int p, uint32_t gid)
{
    return C->w[c][p] ? C->w[c][p][gid] : 1;
}

/* ------------------------------------------------------------------------ */
/* O3 weights: Claim 3.2 evaluated per edge, height by height (Alg. 2),      */
/* for every window (Alg. 1) -- windows of one parity are disjoint, so one   */
/* value per (tree edge, parity, edge) holds all of them.                    */
/* ------------------------------------------------------------------------ */
int or_weights(or_ctx *C, uint64_t *W_lo, uint64_t *W_hi)
{
    if (!C->have_plan) return OR_E_STATE;
    free_weights(C);
    const or_graph *g = &C->g; const or_plan *P = &C->P;
    int64_t m = g->m;
    int overflow = 0;
    int maxh = 0;
    for (int q = 0; q < P->ntree; ++q) if (P->height[P->order[q]] > maxh) maxh = P->height[P->order[q]];
    for (int p = 0; p < 2; ++p) {
        for (int h = 1; h <= maxh; ++h) {
            for (int q = 0; q < P->ntree; ++q) {
                int s = P->order[q];
                if (P->height[s] != h) continue;
                uint64_t *w = malloc(sizeof(uint64_t) * (size_t)(m ? m : 1));
                if (!w) return OR_E_NOMEM;
                C->w[s][p] = w;
                for (int64_t e = 0; e < m; ++e) {
                    int64_t wi = window_of(g->t[e], p, P->wd);
                    if (wi < 0) { w[e] = 0; continue; }
                    /* factor i = sum of w_{s_i} over L_{e,s,s_i}; R7: a factor
                     * >= 2^64 or an exact product >= 2^64 is an overflow. */
                    u128 fac[OR_MAXE];
                    int zero = 0;
                    for (int ci = 0; ci < P->nchild[s]; ++ci) {
                        int c = P->child[s][ci];
                        cand_range R;
                        u128 sum = 0;
                        if (child_candidates(C, s, (uint32_t)e, c, wi, &R))
                            for (int64_t x = R.beg; x < R.end; ++x)
                                if (cand_nbr(g, &R, x) != R.excl)
                                    sum += child_weight(C, c, p, R.list[x]);
                        if (sum >> 64) overflow = 1;
                        if (sum == 0) zero = 1;
                        fac[ci] = sum;
                    }
                    u128 prod = zero ? 0 : 1;
                    for (int ci = 0; ci < P->nchild[s] && prod; ++ci) {
                        prod *= (fac[ci] >> 64) ? 1 : fac[ci];
                        if (prod >> 64) { overflow = 1; prod = 1; }
                    }
                    w[e] = (uint64_t)prod;
                }
            }
        }
    }
    /* per-window totals W_i and W (Claim 3.4 summed over Alg. 1's windows) */
    C->Wi = calloc((size_t)C->nwin, sizeof(uint64_t));
    u128 *acc = calloc((size_t)C->nwin, sizeof(u128));
    int c = P->root;
    for (int p = 0; p < 2; ++p) {
        C->rootcum[p] = malloc(sizeof(uint64_t) * (size_t)(m ? m : 1));
        for (int64_t e = 0; e < m; ++e) {
            int64_t wi = window_of(g->t[e], p, P->wd);
            if (wi < 0) { C->rootcum[p][e] = 0; continue; }
            acc[wi] += child_weight(C, c, p, (uint32_t)e);
            C->rootcum[p][e] = (uint64_t)acc[wi];
        }
    }
    C->W = 0;
    for (int64_t i = 0; i < C->nwin; ++i) {
        if (acc[i] >> 64) overflow = 1;
        C->Wi[i] = (uint64_t)acc[i];
        C->W += acc[i];
    }
    free(acc);
    C->have_weights = 1;
    *W_lo = (uint64_t)C->W; *W_hi = (uint64_t)(C->W >> 64);
    return overflow ? OR_E_OVERFLOW : OR_OK;
}

/* w_{s,e} of tree edge s in layer p for every gid (1/0 for leaves). */
int or_export_weights(const or_ctx *C, int s, int p, uint64_t *out)
{
    if (!C->have_weights || s < 0 || s >= C->P.ne || !C->P.is_tree[s] || p < 0 || p > 1) return OR_E_ARG;
    for (int64_t e = 0; e < C->g.m; ++e) {
        if (C->w[s][p]) out[e] = C->w[s][p][e];
        else out[e] = window_of(C->g.t[e], p, C->P.wd) >= 0 ? 1 : 0;
    }
    return OR_OK;
}

int64_t or_num_windows(const or_ctx *C) { return C->nwin; }
int or_window_totals(const or_ctx *C, uint64_t *out)
{
    if (!C->have_weights) return OR_E_STATE;
    for (int64_t i = 0; i < C->nwin; ++i) out[i] = C->Wi[i];
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Validation and DeriveCnt (Alg. 4-5)                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    const or_ctx *C;
    uint32_t phiV[OR_MAXV];
    int64_t tau[OR_MAXE];                  /* times of tree edges */
    int64_t lb, ub;                        /* every time lies in [lb, ub] */
    int64_t lbeg[OR_MAXE], lend[OR_MAXE];  /* multi-edge lists of non-tree edges */
    int overflow;
} derive_state;

/* Enumerate the non-tree edges position by position in pi order: every chain
 * of strictly increasing times whose total span is at most delta (Def. 1.2). */
static uint64_t derive_rec(derive_state *S, int pos, int64_t prev, int64_t first)
{
    const or_plan *P = &S->C->P; const or_graph *g = &S->C->g;
    if (pos == P->ne) return 1;
    int e = P->pos_edge[pos];
    if (P->is_tree[e]) {
        int64_t t = S->tau[e];
        if (pos > 0 && (t <= prev || t - first > P->delta)) return 0;
        return derive_rec(S, pos + 1, t, pos == 0 ? t : first);
    }
    uint64_t total = 0;
    int64_t x = lower_time(g, g->pair_gid, S->lbeg[e], S->lend[e], S->lb);
    for (; x < S->lend[e]; ++x) {
        int64_t t = g->t[g->pair_gid[x]];
        if (t > S->ub) break;
        if (pos > 0 && t <= prev) continue;
        if (pos > 0 && t - first > P->delta) break;
        uint64_t r = derive_rec(S, pos + 1, t, pos == 0 ? t : first);
        if (total + r < total) S->overflow = 1;
        total += r;
    }
    return total;
}

/* Validate a tree match; returns the reject reason and sets *contrib to
 * cnt * 2 / N_phi on success (R4, R6). */
static int validate_and_count(const or_ctx *C, const uint32_t *treegid, uint64_t *contrib, int *ovf)
{
    const or_plan *P = &C->P; const or_graph *g = &C->g;
    derive_state S; memset(&S, 0, sizeof(S)); S.C = C;
    uint32_t phiV[OR_MAXV];
    for (int q = 0; q < P->ntree; ++q) {
        int s = P->order[q]; uint32_t e = treegid[q];
        phiV[P->a[s]] = g->src[e];
        phiV[P->b[s]] = g->dst[e];
        S.tau[s] = g->t[e];
    }
    *contrib = 0;
    for (int x = 0; x < P->nv; ++x)
        for (int y = x + 1; y < P->nv; ++y)
            if (phiV[x] == phiV[y]) return RS_VERTEX;
    int64_t a = -1, b = -1;
    for (int q = 0; q < P->ntree; ++q) {
        int64_t t = S.tau[P->order[q]];
        if (a < 0 || t < a) a = t;
        if (b < 0 || t > b) b = t;
    }
    if (b - a > P->delta) return RS_DELTA;
    int64_t prev = -1; int have = 0;
    for (int pos = 0; pos < P->ne; ++pos) {
        int e = P->pos_edge[pos];
        if (!P->is_tree[e]) continue;
        if (have && S.tau[e] <= prev) return RS_ORDER;
        prev = S.tau[e]; have = 1;
    }
    for (int v = 0; v < P->nv; ++v) S.phiV[v] = phiV[v];
    for (int e = 0; e < P->ne; ++e)
        if (!P->is_tree[e]) pair_range(g, phiV[P->a[e]], phiV[P->b[e]], &S.lbeg[e], &S.lend[e]);
    S.lb = b - P->delta; S.ub = a + P->delta;
    uint64_t cnt = derive_rec(&S, 0, -1, -1);
    int64_t wd = P->wd;                         /* N_phi counts windows (R4) */
    int N = 1 + ((a >= wd && (b / wd) == (a / wd)) ? 1 : 0);
    uint64_t c2 = (N == 1) ? cnt * 2 : cnt;
    if (N == 1 && cnt > (UINT64_MAX >> 1)) S.overflow = 1;
    if (S.overflow) *ovf = 1;
    *contrib = c2;
    return RS_VALID;
}

/* ------------------------------------------------------------------------ */
/* O3 sampler (Alg. 3 and Alg. 6 with the draw protocol R5)                  */
/* ------------------------------------------------------------------------ */
static int sample_one(const or_ctx *C, uint64_t seed, uint64_t j, uint32_t *treegid)
{
    const or_graph *g = &C->g; const or_plan *P = &C->P;
    int64_t m = g->m;
    draw_state st = { seed, j, 0 };
    u128 r = uniform_u128(&st, C->W);
    /* window: windows ordered by (layer, index) */
    int64_t wi = -1;
    for (int p = 0; p < 2 && wi < 0; ++p)
        for (int64_t i = p; i < C->nwin; i += 2) {
            if (r < (u128)C->Wi[i]) { wi = i; break; }
            r -= C->Wi[i];
        }
    if (wi < 0) return -1;
    int p = (int)(wi & 1);
    /* root edge: first edge of the window (GLOBAL order) whose running sum
     * of w_c exceeds r, i.e. probability w_{c,e} / W_i (Alg. 3). */
    uint64_t rr = (uint64_t)r;
    int64_t lo = 0, hi = m;                       /* first gid with t' >= wi*d */
    while (lo < hi) { int64_t mid = lo + (hi - lo) / 2; if (g->t[mid] < wi * P->wd) lo = mid + 1; else hi = mid; }
    int64_t wbeg = lo;
    hi = m;                                       /* first gid with t' >= (wi+2)*d */
    while (lo < hi) { int64_t mid = lo + (hi - lo) / 2; if (g->t[mid] < (wi + 2) * P->wd) lo = mid + 1; else hi = mid; }
    int64_t wend = lo;
    lo = wbeg; hi = wend;
    while (lo < hi) { int64_t mid = lo + (hi - lo) / 2; if (C->rootcum[p][mid] <= rr) lo = mid + 1; else hi = mid; }
    int64_t root = (lo < wend) ? lo : -1;
    if (root < 0) return -1;
    uint32_t match[OR_MAXE];
    match[P->root] = (uint32_t)root;
    treegid[0] = (uint32_t)root;
    for (int q = 1; q < P->ntree; ++q) {
        int c = P->order[q], s = P->parent[c];
        cand_range R;
        if (!child_candidates(C, s, match[s], c, wi, &R)) return -1;
        u128 total = 0;
        for (int64_t x = R.beg; x < R.end; ++x)
            if (cand_nbr(g, &R, x) != R.excl) total += child_weight(C, c, p, R.list[x]);
        if (total == 0 || (total >> 64)) return -1;
        uint64_t rc = uniform_u64(&st, (uint64_t)total);
        uint64_t run = 0; int64_t pick = -1;
        for (int64_t x = R.beg; x < R.end; ++x) {
            if (cand_nbr(g, &R, x) == R.excl) continue;
            run += child_weight(C, c, p, R.list[x]);
            if (run > rc) { pick = x; break; }
        }
        if (pick < 0) return -1;
        match[c] = R.list[pick];
        treegid[q] = R.list[pick];
    }
    return 0;
}

int or_sample(const or_ctx *C, uint64_t k, uint64_t seed, uint64_t first, int nthreads,
              or_result *res, uint32_t *trace_gid, uint64_t *trace_contrib, int32_t *trace_reason)
{
    memset(res, 0, sizeof(*res));
    if (!C->have_weights) return OR_E_STATE;
    res->k = k;
    res->W_lo = (uint64_t)C->W; res->W_hi = (uint64_t)(C->W >> 64);
    if (C->W == 0 || k == 0) return OR_OK;
    int nt = C->P.ntree;
    int err = 0, ovf = 0;
    u128 hits = 0;
    uint64_t valid = 0, rv = 0, rd = 0, ro = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        u128 h_loc = 0; uint64_t v_loc = 0, rv_loc = 0, rd_loc = 0, ro_loc = 0;
        int err_loc = 0, ovf_loc = 0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4096)
#endif
        for (int64_t i = 0; i < (int64_t)k; ++i) {
            uint32_t tg[OR_MAXV];
            uint64_t contrib = 0; int reason = -1;
            if (sample_one(C, seed, first + (uint64_t)i, tg) != 0) { err_loc = 1; }
            else {
                reason = validate_and_count(C, tg, &contrib, &ovf_loc);
                if (reason == RS_VALID) { ++v_loc; h_loc += contrib; }
                else if (reason == RS_VERTEX) ++rv_loc;
                else if (reason == RS_DELTA) ++rd_loc;
                else ++ro_loc;
            }
            if (trace_gid) for (int q = 0; q < nt; ++q) trace_gid[(size_t)i * nt + q] = tg[q];
            if (trace_contrib) trace_contrib[i] = contrib;
            if (trace_reason) trace_reason[i] = reason;
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        {
            hits += h_loc; valid += v_loc; rv += rv_loc; rd += rd_loc; ro += ro_loc;
            err |= err_loc; ovf |= ovf_loc;
        }
    }
    res->hits2_lo = (uint64_t)hits; res->hits2_hi = (uint64_t)(hits >> 64);
    res->valid = valid; res->rej_vertex = rv; res->rej_delta = rd; res->rej_order = ro;
    res->estimate = (double)C->W * (double)hits / (2.0 * (double)k);
    if (err) return OR_E_STATE;
    return ovf ? OR_E_OVERFLOW : OR_OK;
}

/* ------------------------------------------------------------------------ */
/* O2 / O4: brute force over every delta-partial match inside window i      */
/* (Def. of delta-partial match: homomorphism, Constraint 1 on every        */
/* parent/child pair, Constraint 2 on the far endpoints, Constraint 3).     */
/* Each candidate for a child is tested against every condition directly;   */
/* the weights are not used.                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    const or_ctx *C;
    int64_t wi;
    uint32_t match[OR_MAXE];
    uint32_t tree_by_order[OR_MAXV];
    uint64_t count;          /* O2: number of partial matches */
    u128 sum2;               /* O4: sum of cnt * 2 / N_phi    */
    int do_count_motifs;
    int overflow;
    uint32_t *list_out; int64_t list_cap, list_len;
} enum_state;

static int in_window(int64_t t, int64_t wi, int64_t d) { return t >= wi * d && t < (wi + 2) * d; }

static void enum_rec(enum_state *E, int q)
{
    const or_ctx *C = E->C; const or_graph *g = &C->g; const or_plan *P = &C->P;
    int64_t d = P->delta;
    if (q == P->ntree) {
        E->count++;
        if (E->list_out && E->list_len < E->list_cap)
            for (int k = 0; k < P->ntree; ++k) E->list_out[E->list_len * P->ntree + k] = E->tree_by_order[k];
        E->list_len++;
        if (E->do_count_motifs) {
            uint64_t contrib = 0; int ovf = 0;
            if (validate_and_count(C, E->tree_by_order, &contrib, &ovf) == RS_VALID) E->sum2 += contrib;
            if (ovf) E->overflow = 1;
        }
        return;
    }
    int c = P->order[q];
    if (q == 0) {
        for (int64_t e = 0; e < g->m; ++e) {
            if (!in_window(g->t[e], E->wi, P->wd)) continue;
            E->match[c] = (uint32_t)e; E->tree_by_order[0] = (uint32_t)e;
            enum_rec(E, 1);
        }
        return;
    }
    int s = P->parent[c], z = P->meet[c], o = other_end(P, s, z);
    uint32_t es = E->match[s];
    uint32_t zg = (P->a[s] == z) ? g->src[es] : g->dst[es];
    uint32_t og = (P->a[s] == o) ? g->src[es] : g->dst[es];
    int out_dir = (P->a[c] == z);
    const uint32_t *list = out_dir ? g->out_gid : g->in_gid;
    const int64_t *beg = out_dir ? g->out_beg : g->in_beg;
    for (int64_t x = beg[zg]; x < beg[zg + 1]; ++x) {
        uint32_t e = list[x];
        uint32_t nbr = out_dir ? g->dst[e] : g->src[e];
        int64_t t = g->t[e], ts = g->t[es];
        if (!in_window(t, E->wi, P->wd)) continue;                   /* C3 */
        if (P->rank[c] > P->rank[s]) { if (!(t > ts && t <= ts + d)) continue; }  /* C1 */
        else { if (!(t < ts && t >= ts - d)) continue; }
        if (P->c2 && nbr == og) continue;                            /* C2 */
        E->match[c] = e; E->tree_by_order[q] = e;
        enum_rec(E, q + 1);
    }
}

/* O2: number of delta-partial matches inside window i; optional list of them
 * (tree gids in sampling order). */
int or_partial_count(const or_ctx *C, int64_t wi, uint64_t *count, uint32_t *list_out, int64_t list_cap, int64_t *list_len)
{
    if (!C->have_plan || wi < 0 || wi >= C->nwin) return OR_E_ARG;
    enum_state E; memset(&E, 0, sizeof(E));
    E.C = C; E.wi = wi; E.list_out = list_out; E.list_cap = list_cap;
    enum_rec(&E, 0);
    *count = E.count;
    if (list_len) *list_len = E.list_len;
    return OR_OK;
}

/* O4: exact C = (sum over windows and partial matches of 2*cnt/N_phi) / 2. */
int or_exact_by_trees(const or_ctx *C, uint64_t *sum2_lo, uint64_t *sum2_hi)
{
    if (!C->have_plan) return OR_E_STATE;
    u128 total = 0; int ovf = 0;
    for (int64_t wi = 0; wi < C->nwin; ++wi) {
        enum_state E; memset(&E, 0, sizeof(E));
        E.C = C; E.wi = wi; E.do_count_motifs = 1;
        enum_rec(&E, 0);
        total += E.sum2;
        ovf |= E.overflow;
    }
    *sum2_lo = (uint64_t)total; *sum2_hi = (uint64_t)(total >> 64);
    return ovf ? OR_E_OVERFLOW : OR_OK;
}

/* ------------------------------------------------------------------------ */
/* O1: exact count by chronological backtracking (Def. 1.2).  Motif edges   */
/* are mapped in pi order; each graph edge is tried directly against the    */
/* vertex map built so far; times strictly increase and stay within delta   */
/* of the first edge; the vertex map is injective.                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    const or_ctx *C;
    const or_plan *P;
    int32_t phi[OR_MAXV];
    uint64_t count;
    int overflow;
} brute_state;

static void brute_rec(brute_state *B, int pos, int64_t prev, int64_t first);

static int vertex_used(const brute_state *B, uint32_t x)
{
    for (int v = 0; v < B->P->nv; ++v) if (B->phi[v] >= 0 && (uint32_t)B->phi[v] == x) return 1;
    return 0;
}

static void brute_try(brute_state *B, int pos, int64_t first, uint32_t ge, int a, int b)
{
    const or_graph *g = &B->C->g;
    uint32_t u = g->src[ge], v = g->dst[ge];
    int32_t pa = B->phi[a], pb = B->phi[b];
    if (pa >= 0 && (uint32_t)pa != u) return;
    if (pb >= 0 && (uint32_t)pb != v) return;
    int seta = 0, setb = 0;
    if (pa < 0) { if (vertex_used(B, u)) return; B->phi[a] = (int32_t)u; seta = 1; }
    if (pb < 0) {
        if (vertex_used(B, v)) { if (seta) B->phi[a] = -1; return; }
        B->phi[b] = (int32_t)v; setb = 1;
    }
    int64_t t = g->t[ge];
    brute_rec(B, pos + 1, t, pos == 0 ? t : first);
    if (seta) B->phi[a] = -1;
    if (setb) B->phi[b] = -1;
}

static void brute_rec(brute_state *B, int pos, int64_t prev, int64_t first)
{
    const or_graph *g = &B->C->g; const or_plan *P = B->P;
    if (pos == P->ne) { if (++B->count == 0) B->overflow = 1; return; }
    int e = P->pos_edge[pos];
    int a = P->a[e], b = P->b[e];
    int64_t lo = (pos == 0) ? 0 : prev + 1;          /* strictly later */
    int64_t hi = (pos == 0) ? g->T : first + P->delta; /* within delta of the first */
    int32_t pa = B->phi[a], pb = B->phi[b];
    /* The graph edges that can match motif edge (a,b): the multi-edge list
     * when both ends are mapped, the out-list of phi(a) or the in-list of
     * phi(b) when one is, every edge otherwise; each is then checked. */
    if (pa >= 0 && pb >= 0) {
        int64_t beg, end;
        pair_range(g, (uint32_t)pa, (uint32_t)pb, &beg, &end);
        for (int64_t x = lower_time(g, g->pair_gid, beg, end, lo); x < end && g->t[g->pair_gid[x]] <= hi; ++x)
            brute_try(B, pos, first, g->pair_gid[x], a, b);
    } else if (pa >= 0) {
        int64_t beg = g->out_beg[pa], end = g->out_beg[pa + 1];
        for (int64_t x = lower_time(g, g->out_gid, beg, end, lo); x < end && g->t[g->out_gid[x]] <= hi; ++x)
            brute_try(B, pos, first, g->out_gid[x], a, b);
    } else if (pb >= 0) {
        int64_t beg = g->in_beg[pb], end = g->in_beg[pb + 1];
        for (int64_t x = lower_time(g, g->in_gid, beg, end, lo); x < end && g->t[g->in_gid[x]] <= hi; ++x)
            brute_try(B, pos, first, g->in_gid[x], a, b);
    } else {
        int64_t L = 0, R = g->m;
        while (L < R) { int64_t mid = (L + R) / 2; if (g->t[mid] < lo) L = mid + 1; else R = mid; }
        for (int64_t ge = L; ge < g->m && g->t[ge] <= hi; ++ge)
            brute_try(B, pos, first, (uint32_t)ge, a, b);
    }
}

/* O1 needs only the motif (no tree): pass ne edges, ranks and delta. */
int or_brute_count(const or_ctx *C, int nv, int ne, const int32_t *ea, const int32_t *eb,
                   const int32_t *rank, int64_t delta, uint64_t *count)
{
    or_plan P; memset(&P, 0, sizeof(P));
    if (nv < 1 || nv > OR_MAXV || ne < 1 || ne > OR_MAXE || delta <= 0) return OR_E_MOTIF;
    int seen[OR_MAXE] = {0};
    P.nv = nv; P.ne = ne; P.delta = delta;
    for (int i = 0; i < ne; ++i) {
        if (ea[i] < 0 || ea[i] >= nv || eb[i] < 0 || eb[i] >= nv || ea[i] == eb[i]) return OR_E_MOTIF;
        if (rank[i] < 0 || rank[i] >= ne || seen[rank[i]]) return OR_E_MOTIF;
        seen[rank[i]] = 1;
        P.a[i] = ea[i]; P.b[i] = eb[i]; P.rank[i] = rank[i]; P.pos_edge[rank[i]] = i;
    }
    brute_state B; memset(&B, 0, sizeof(B));
    B.C = C; B.P = &P;
    for (int v = 0; v < OR_MAXV; ++v) B.phi[v] = -1;
    brute_rec(&B, 0, -1, -1);
    *count = B.count;
    return B.overflow ? OR_E_OVERFLOW : OR_OK;
}
