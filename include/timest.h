/*
 * timest.h -- C ABI of the GB300-native TIMEST temporal-motif estimator.
 *
 * TIMEST (Pan, Bhalerao, Seshadhri, Talati, arXiv 2507.20441) estimates the
 * number C of M-matches of a temporal motif M = (H, pi, delta) in a directed
 * temporal multigraph G (Def. 1.1-1.2): it picks a spanning tree S of H rooted
 * at an edge c, computes per-edge weights w_{s,e} by a dynamic program over
 * the tree inside overlapping 2*delta windows (Sec. 3.1, Claims 3.1-3.4,
 * Alg. 1-2), samples k partial matches of S with probability N_phi / W
 * (Sec. 3.2, Alg. 3, Lemma 3.5), validates each and counts its completions to
 * M (Sec. 3.3, Alg. 4-5) and returns C_hat = W * sum(cnt / N_phi) / k
 * (Alg. 6, Lemma 3.6).  All arithmetic is exact integer: weights are unsigned
 * 64-bit, totals 128-bit.
 *
 * Conventions (all entry points):
 *   - Every function returns a status (TM_OK = 0 or a TM_E_* code); on error
 *     tm_last_error(ctx) holds a one-line message.  No call traps or aborts.
 *   - Host pointers are plain CPU memory; "device" pointers are CUDA global
 *     memory of the context's device.  The caller owns every array it passes
 *     and may free it as soon as the call returns; the library copies what it
 *     keeps.  The context owns all device memory it allocates.
 *   - Calls on one context are serialised by the caller and run on the
 *     context's CUDA stream.  tm_serve_submit / tm_serve_poll are thread safe.
 *   - Time t' = t - t_min (Sec. 3 preamble).  The graph's time span
 *     t_max - t_min must be < 2^32 - 1 and m, n < 2^32 - 1 (TM_E_LIMIT).
 *   - Windows are [i*delta, (i+2)*delta) in t', i = 0..floor(T/delta)
 *     (Constraint 3, Sec. 2.1, Alg. 1).  Constraint 1 puts a later child edge
 *     in (t, t+delta] and an earlier one in [t-delta, t).
 */
#ifndef TIMEST_GB300_H
#define TIMEST_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
enum {
    TM_OK = 0,
    TM_E_ARG = 1,       /* bad argument (null pointer, out-of-range id, ...) */
    TM_E_DUP = 2,       /* repeated (u,v,t) tuple; Sec. 1.1 forbids it       */
    TM_E_SELFLOOP = 3,  /* u == v; never part of an injective match          */
    TM_E_MOTIF = 4,     /* motif or tree invalid (disconnected, self loop,   */
                        /* order not a permutation, delta <= 0, nv > 8, ...) */
    TM_E_NOMEM = 5,     /* device allocation failed                          */
    TM_E_OVERFLOW = 6,  /* an exact count does not fit its integer width     */
    TM_E_STATE = 7,     /* call out of order (e.g. sample before weights)    */
    TM_E_TIMEOUT = 8,   /* a bounded wait ran out                            */
    TM_E_CUDA = 9,      /* a CUDA runtime call failed                        */
    TM_E_LIMIT = 10,    /* size beyond a stated limit                        */
    TM_E_PENDING = 11   /* a served query has not finished yet (poll again)  */
};

/* ---- tm_graph_load flags ------------------------------------------------ */
enum {
    TM_HOST = 0,        /* src/dst/t are host pointers                        */
    TM_DEVICE = 1,      /* src/dst/t are device pointers                      */
    TM_DEDUP = 2,       /* drop repeated (u,v,t) tuples instead of TM_E_DUP   */
    TM_DROP_SELF = 4,   /* drop self loops instead of TM_E_SELFLOOP           */
    TM_PREPROCESS = 8   /* also run tm_preprocess in the same call; with      */
                        /* TM_DEVICE the arrays are read in place (no staged  */
                        /* copy), so they must stay valid until it returns    */
};

typedef struct tm_ctx tm_ctx;
typedef struct tm_motif tm_motif;

/* Unsigned 128-bit integer as two 64-bit halves. */
typedef struct { uint64_t lo, hi; } tm_u128;

/* Optional device allocator.  alloc returns a device pointer (or NULL on
 * failure) of at least `bytes` bytes usable on `stream`; free releases it. */
typedef void *(*tm_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*tm_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

typedef struct {
    tm_alloc_fn alloc;      /* NULL: cudaMallocAsync on the context stream */
    tm_free_fn free;
    void *alloc_user;
    int device;             /* CUDA device ordinal (default 0)              */
    int sample_threads;     /* threads per block of the sampler (0 = auto)  */
    int sample_tile;        /* samples per work item of batched runs (0 = auto) */
    int profile;            /* 1: time every phase with CUDA events;
                               2: also every kernel launch (tm_kernel_times) */
    int reserved[7];
} tm_config;

/* Result of one estimate.  estimate = W * hits2 / (2k) (Alg. 6 with the
 * per-sample count cnt * 2 / N_phi kept integral). */
typedef struct {
    tm_u128 W;              /* total number of (window, partial match) pairs */
    tm_u128 hits2;          /* sum over samples of cnt * 2 / N_phi           */
    uint64_t k;             /* samples drawn                                 */
    uint64_t valid;         /* samples passing Alg. 4's three checks         */
    uint64_t rej_vertex;    /* rejected: vertex map not 1-1                  */
    uint64_t rej_delta;     /* rejected: tree edges span more than delta     */
    uint64_t rej_order;     /* rejected: tree edges out of pi order          */
    double estimate;        /* C_hat                                         */
} tm_result;

/* Fill *cfg with defaults. */
void tm_config_default(tm_config *cfg);

/* Create a context on cfg->device.  cuda_stream is a cudaStream_t to run on
 * (NULL: the context creates its own).  *out receives the context. */
int tm_create(tm_ctx **out, const tm_config *cfg, void *cuda_stream);

/* Destroy a context and every device buffer it owns (motifs must be freed
 * first with tm_motif_free). */
void tm_destroy(tm_ctx *ctx);

/* One-line message for the last failing call on ctx (never NULL). */
const char *tm_last_error(tm_ctx *ctx);

/* Load a temporal graph: m tuples (src[i], dst[i], t[i]) over n vertices
 * (Sec. 1.1).  flags: TM_HOST or TM_DEVICE for where the three arrays live,
 * plus TM_DEDUP / TM_DROP_SELF, and TM_PREPROCESS to build the adjacency in
 * the same call (then device arrays are read in place instead of staged, and
 * the call returns once they are no longer read).  Ids must be < n.  Replaces
 * any previous graph (and invalidates motifs' weights).  Errors: TM_E_ARG,
 * TM_E_DUP, TM_E_SELFLOOP, TM_E_LIMIT, TM_E_NOMEM, TM_E_CUDA. */
int tm_graph_load(tm_ctx *ctx, uint32_t n, uint64_t m, const uint32_t *src,
                  const uint32_t *dst, const int64_t *t, int flags);

/* Build the time-sorted adjacency of the loaded graph on the device (Sec. 3
 * preamble; Defs. 3.1-3.3): the GLOBAL order (t', src, dst) that numbers the
 * edges, per-vertex out-lists (t', dst), in-lists (t', src), and per-pair
 * multi-edge lists El_{u,v} (t').  Duplicates / self loops are reported here
 * when tm_graph_load was given device pointers.  The graph takes about 80
 * bytes of device memory per edge (20 u32 arrays of m entries, the pair tables
 * among them, plus three bit sets of m bits and 12 bytes per vertex). */
int tm_preprocess(tm_ctx *ctx);

/* Number of edges kept, t_min and T = max t' of the preprocessed graph. */
int tm_graph_info(tm_ctx *ctx, uint64_t *m, int64_t *t_min, int64_t *T);

/* Copy the GLOBAL order to host arrays of m entries (tests and debugging). */
int tm_edges_export(tm_ctx *ctx, uint32_t *src, uint32_t *dst, uint32_t *tprime);

/* One array of the temporal CSR (Sec. 3 preamble, Defs. 3.1-3.3), for tests
 * and debugging.  gid = position in GLOBAL order (t', src, dst); the OUT order
 * is (src, t', dst), the IN order (dst, t', src), the MULTI order
 * (src, dst, t'); all positions are 0-based indexes into those orders.
 *   OUT_OFF, IN_OFF, VPAIR_OFF : n+1 list starts (VPAIR_OFF: first pair of
 *                                each source in (src, dst) order)
 *   OUT_T/NBR/GID/SRC          : m, per OUT position: t', dst, gid, src
 *   IN_T/NBR/GID/DST           : m, per IN position: t', src, gid, dst
 *   OUT_POS, IN_POS            : m, per gid: its OUT / IN position
 *   OUT_XRANK                  : m, per OUT position x (owner z, time t'):
 *                                the first IN position of z's list with time
 *                                >= t' (z's in-list end if none); IN_XRANK the
 *                                same with the roles swapped
 *   IN_TO_OUT, MULTI_TO_OUT    : m, per IN / MULTI position: the OUT position
 *   MULTI_T                    : m, per MULTI position: t'
 *   PAIR_OFF, PAIR_DST         : P+1 run starts in MULTI order, P heads
 *   OWN_OUT/IN/MULTI           : m/32+1 words, bit x set when position x
 *                                starts a new owner (vertex, vertex, pair)
 * host_out holds cap entries; *len (if not null) receives the array's length
 * whether or not it is copied (host_out null copies nothing).  Errors:
 * TM_E_ARG (unknown array, cap below the length), TM_E_STATE (no graph). */
enum {
    TM_CSR_OUT_OFF = 0, TM_CSR_OUT_T, TM_CSR_OUT_NBR, TM_CSR_OUT_GID, TM_CSR_OUT_SRC, TM_CSR_OUT_POS,
    TM_CSR_OUT_XRANK, TM_CSR_IN_OFF, TM_CSR_IN_T, TM_CSR_IN_NBR, TM_CSR_IN_GID, TM_CSR_IN_DST, TM_CSR_IN_POS,
    TM_CSR_IN_XRANK, TM_CSR_IN_TO_OUT, TM_CSR_VPAIR_OFF, TM_CSR_PAIR_OFF, TM_CSR_PAIR_DST, TM_CSR_MULTI_T,
    TM_CSR_MULTI_TO_OUT, TM_CSR_OWN_OUT, TM_CSR_OWN_IN, TM_CSR_OWN_MULTI, TM_CSR_NUM_ARRAYS
};
int tm_csr_export(tm_ctx *ctx, int array, uint32_t *host_out, uint64_t cap, uint64_t *len);

/* Define motif M = (H, pi, delta) (Def. 1.1): nv <= 8 vertices, ne <= 16
 * edges; edges[2i], edges[2i+1] are the tail and head of edge i; order[i] is
 * the position of edge i in pi (a permutation of 0..ne-1); delta >= 1.
 * Picks a default spanning tree and root: the tree of least constraint
 * looseness (Alg. 8, read over tree edges), ties to the lexicographically
 * smallest edge set, rooted at the edge of least eccentricity.
 * Errors: TM_E_ARG, TM_E_MOTIF. */
int tm_set_motif(tm_ctx *ctx, uint32_t nv, uint32_t ne, const uint32_t *edges,
                 const uint32_t *order, int64_t delta, tm_motif **out);

/* Pin the spanning tree (nv-1 motif-edge ids) and its root edge
 * (Def. 3.5).  Invalidates cached weights.  Errors: TM_E_MOTIF. */
int tm_set_tree(tm_motif *mo, const uint32_t *tree_edge_ids, uint32_t root_edge);

/* Constraint toggles of the ablation (the paper's table of constraints):
 * TM_C2 keeps Constraint 2 (a child's candidate list leaves out the
 * multi-edges to the parent's other endpoint), TM_C3 keeps Constraint 3 (the
 * 2*delta windows).  Constraint 1 always holds.  Without TM_C3 one window
 * holds every edge (window unit 2^33 > any t' span), so every N_phi is 1.
 * The estimate stays unbiased under every setting; only the valid-sample rate
 * and the variance change.  Default (tm_set_motif): TM_C2 | TM_C3.  Invalidates
 * cached weights.  Errors: TM_E_ARG (unknown flag). */
enum { TM_C2 = 1, TM_C3 = 2 };
int tm_set_constraints(tm_motif *mo, int flags);

/* Every spanning tree of motif (nv, ne, edges, order) (the arguments of
 * tm_set_motif), ranked as in Alg. 7 by constraint looseness (Alg. 8, read
 * over unordered pairs of tree edges sharing a vertex: sum of
 * |pi(e1) - pi(e2)| - 1), smallest first, ties to the lexicographically
 * smallest edge set.  Writes the first min(max_out, total) trees: masks_out[i]
 * has bit j set when motif edge j is a tree edge, looseness_out[i] its
 * looseness (either array may be null); *n_total = number of spanning trees.
 * Host only: no context, no device.  Errors: TM_E_ARG, TM_E_MOTIF. */
int tm_tree_candidates(uint32_t nv, uint32_t ne, const uint32_t *edges, const uint32_t *order,
                       uint32_t max_out, uint32_t *masks_out, uint32_t *looseness_out,
                       uint32_t *n_total);

/* One evaluated (tree, root) candidate of tm_select_tree. */
typedef struct {
    uint32_t tree_mask;     /* bit j set: motif edge j is a tree edge        */
    uint32_t root;          /* root edge (a tree edge)                       */
    uint32_t looseness;     /* of the tree (Alg. 8)                          */
    int32_t status;         /* TM_OK, or the weight pass's error (overflow)  */
    tm_u128 W;              /* exact W of the weight pass (0 on error)       */
} tm_tree_cand;

/* Spanning tree and root selection (Alg. 7): the n_c trees of least
 * looseness (order of tm_tree_candidates) are evaluated by the exact W of a
 * full weight pass on the current graph, each with every tree edge as root
 * (all_roots != 0) or with the default root of least eccentricity; the
 * candidate of least W wins (ties: the earlier evaluated, i.e. better ranked
 * tree, then lower root edge id).  Candidates are evaluated in that order and
 * recorded in cands[0 .. min(max_cand, evaluated)) when cands is not null;
 * *n_cand = number evaluated.  *out receives the winning motif with its
 * weights already computed (free it with tm_motif_free); the others' weights
 * are freed as the search goes.  A candidate whose weight pass overflows is
 * skipped.  Errors: TM_E_ARG, TM_E_MOTIF, TM_E_STATE (no preprocessed graph),
 * TM_E_OVERFLOW (every candidate overflowed), TM_E_NOMEM, TM_E_CUDA. */
int tm_select_tree(tm_ctx *ctx, uint32_t nv, uint32_t ne, const uint32_t *edges,
                   const uint32_t *order, int64_t delta, uint32_t n_c, int all_roots,
                   tm_motif **out, tm_tree_cand *cands, uint32_t max_cand, uint32_t *n_cand);

/* Read the tree plan: order[q] = motif edge sampled q-th (q < nv-1),
 * parent[q] = index in order of its parent (-1 for the root). */
int tm_motif_plan(tm_motif *mo, int32_t *order, int32_t *parent);

/* Weight pass (Sec. 3.1): windows, the DP over the tree in height order
 * (Claim 3.2, Alg. 2), segmented prefix sums and the root CDF (Claim 3.4).
 * *W_out receives W = sum over windows of W_i.  Weights stay resident in the
 * motif until it is freed or the graph changes.
 * Errors: TM_E_STATE (no graph), TM_E_OVERFLOW, TM_E_NOMEM, TM_E_CUDA. */
int tm_weights(tm_ctx *ctx, tm_motif *mo, tm_u128 *W_out);

/* Copy w_{s,e} of tree edge `tree_edge` (a motif-edge id) in window layer
 * `layer` (0: windows with even i, 1: odd i) for every edge, in GLOBAL order,
 * to host_out[m].  Edges outside any window of the layer read 0. */
int tm_weights_export(tm_ctx *ctx, tm_motif *mo, uint32_t tree_edge, uint32_t layer,
                      uint64_t *host_out);

/* Per-window totals W_i, i = 0..floor(T/delta), to host_out[cap];
 * *nwin receives floor(T/delta)+1. */
int tm_window_totals(tm_ctx *ctx, tm_motif *mo, uint64_t *host_out, uint64_t cap,
                     uint64_t *nwin);

/* Motif listing (Alg. 5 emitting the instances it counts): samples
 * first_index .. first_index+k-1 are drawn as tm_sample draws them; for every
 * valid sample, each M-match (Def. 1.2) whose tree edges are the sampled tree
 * is one instance.  Instance rows are ordered by sample id, then depth first
 * over the non-tree edges in pi order, each multi-edge list in time order.
 * Row r: inst_gids[r*ne + e] = edge id (GLOBAL order) matched to motif edge
 * e, inst_sample[r] = its sample id.  At most max_inst rows are written (host
 * arrays of max_inst*ne and max_inst entries); *n_inst receives the total
 * number of instances, which may exceed max_inst.  Two passes: counts per
 * sample, then the instances (the second checks that it finds as many as
 * DeriveCnt counted).  Errors: TM_E_STATE (no weights), TM_E_ARG,
 * TM_E_OVERFLOW, TM_E_NOMEM, TM_E_CUDA. */
int tm_sample_list(tm_ctx *ctx, tm_motif *mo, uint64_t k, uint64_t seed, uint64_t first_index,
                   uint64_t max_inst, uint32_t *inst_gids, uint64_t *inst_sample, uint64_t *n_inst);

/* Several motifs per sampling run (the paper counts related motifs, e.g.
 * M4-1..M4-4, from one run): motifs[0..nm), 1 <= nm <= 8, whose spanning
 * trees (after tm_set_motif / tm_set_tree) are the same temporal pattern -
 * same vertex count and delta, and per tree node the same endpoint vertex
 * ids, parent, meeting side, direction, leaf flag and pi relation to its
 * parent, with the tree edges in the same pi order - share motifs[0]'s
 * weights (which must be computed) and one stream of sampled trees.  Each
 * sample is drawn and validated once and completed (Alg. 5) once per motif.
 * results[i] equals tm_sample(ctx, motifs[i], k, seed, first_index) bit for
 * bit (W, hits2, counters, estimate).  Errors: TM_E_ARG, TM_E_STATE (no
 * weights on motifs[0]), TM_E_MOTIF (a tree pattern differs), TM_E_LIMIT
 * (nm > 8), TM_E_OVERFLOW, TM_E_CUDA. */
int tm_sample_group(tm_ctx *ctx, tm_motif *const *motifs, uint32_t nm, uint64_t k, uint64_t seed,
                    uint64_t first_index, tm_result *results);

/* Draw k samples with ids first_index .. first_index+k-1 from seed (Sec. 3.2
 * with the counter-based draw protocol: Philox4x32-10, key = seed, counter =
 * (sample id, draw number)), validate and count them (Sec. 3.3) and reduce
 * (Alg. 6).  Disjoint id ranges add exactly, so a job can be split or
 * resumed.  Errors: TM_E_STATE (no weights), TM_E_OVERFLOW, TM_E_CUDA. */
int tm_sample(tm_ctx *ctx, tm_motif *mo, uint64_t k, uint64_t seed, uint64_t first_index,
              tm_result *out);

/* Like tm_sample, and also copies each sample's tree edges (GLOBAL-order ids,
 * in plan order; k*(nv-1) entries), its contribution cnt*2/N_phi and its
 * outcome (0 valid, 1 vertex, 2 delta, 3 order) to host arrays. */
int tm_sample_trace(tm_ctx *ctx, tm_motif *mo, uint64_t k, uint64_t seed, uint64_t first_index,
                    uint32_t *tree_gids, uint64_t *contrib, int32_t *reason, tm_result *out);

/* Allocation-free variant of tm_sample, for callers that cannot allocate
 * device memory while sampling (a serving loop whose memory pool is held by
 * resident weights, a host framework that owns the allocator, a loop that
 * cannot afford an allocator call).  The paper has no counterpart: it is an
 * interface choice of this library.  Results are bit-identical to tm_sample
 * with the same arguments.  The call allocates nothing: its scratch (the
 * device copy of the motif plan and the result accumulators) is a fixed
 * 4096-byte array that every device loading the library holds until the
 * process exits; a plan that does not fit returns TM_E_LIMIT.  The first
 * call on a device looks up the array's device address (once per device,
 * with that device current), so make that first call before any stream
 * capture.  The accumulators are cleared at the start of every call, but all
 * calls share the one array: calls whose GPU work overlaps (on different
 * streams or contexts of one device) race.  Weights must already exist
 * (tm_weights).  Errors: TM_E_STATE, TM_E_LIMIT, TM_E_OVERFLOW, TM_E_CUDA. */
int tm_sample_noalloc(tm_ctx *ctx, tm_motif *mo, uint64_t k, uint64_t seed, uint64_t first_index,
                      tm_result *out);

/* Batched estimate: nq queries (motifs with weights, sample counts, seeds)
 * run as one persistent launch over a shared queue of sample tiles.  out[q]
 * is bit-identical to tm_sample(ctx, motifs[q], k[q], seed[q], 0, ...). */
int tm_batch_run(tm_ctx *ctx, uint32_t nq, tm_motif *const *motifs, const uint64_t *k,
                 const uint64_t *seed, tm_result *out);

/* ---- serving: continuous batching over a resident graph ----------------
 * Between tm_serve_start and tm_serve_stop only the tm_serve_* calls (and
 * tm_last_error) may be made on ctx; submit and poll are thread safe.
 * Each query runs on its motif's default tree (tm_set_motif), or on the plan
 * of the motif handle given to tm_serve_submit_motif, with sample ids 0..k-1,
 * so its result equals tm_sample on that plan with the same k and seed
 * whatever else is being served. */
typedef struct {
    uint32_t max_active;      /* queries sampled concurrently (0 = 64)                 */
    uint32_t tile;            /* samples per work item (0 = 4096)                      */
    uint32_t round_tiles;     /* work items per scheduling round (0 = 2 per SM, >= 64) */
    int32_t poll_timeout_ms;  /* bound on each wait for a round on the GPU (0 = 60 s)  */
    uint64_t weight_budget;   /* device bytes for resident weights (0 = half the free
                                 memory at start); least recently used weights that no
                                 query holds are evicted to admit new ones            */
    int32_t reserved[8];
} tm_serve_cfg;

typedef struct {
    uint64_t submitted, completed, failed;
    uint64_t cache_hits, cache_misses, evictions, rounds;
    uint64_t resident_bytes, waiting, active;
    double p50_ms, p99_ms, mean_ms;   /* submit-to-completion latency          */
    double qps;                       /* completed / (last completion - first submit) */
    uint64_t nomem_retries;           /* back-offs after a device allocation failed:
                                         a weight pass retried by admission or a
                                         sampling round run again              */
} tm_serve_stats_t;

/* Start the admission and scheduling threads on a preprocessed graph.
 * Errors: TM_E_STATE (already serving, no graph), TM_E_NOMEM, TM_E_CUDA. */
int tm_serve_start(tm_ctx *ctx, const tm_serve_cfg *cfg);

/* Queue a query M = (H, pi, delta) (arguments as tm_set_motif) with k samples
 * from seed; *ticket identifies it.  Errors: TM_E_STATE (not serving),
 * TM_E_MOTIF, TM_E_ARG.
 * Admission: when a query's weight pass (or a sampling round) runs out of
 * device memory, the server frees cached weights that no query holds, waits
 * for queries in flight and retries (up to 200 times, 20 ms apart) before the
 * query fails with TM_E_NOMEM; tm_serve_stats counts these back-offs. */
int tm_serve_submit(tm_ctx *ctx, uint32_t nv, uint32_t ne, const uint32_t *edges, const uint32_t *order,
                    int64_t delta, uint64_t k, uint64_t seed, uint64_t *ticket);

/* Queue a query on a motif handle of this context with its plan as it stands:
 * the spanning tree and root pinned by tm_set_tree (Alg. 7's choice, e.g. the
 * winner of tm_select_tree) and the constraint settings of tm_set_constraints.
 * The server copies the plan (mo stays the caller's, and may be freed or
 * changed after the call) and computes or reuses the weights of that exact
 * plan; the result equals tm_sample on mo with the same k and seed.
 * Errors: TM_E_STATE (not serving), TM_E_ARG (null, or a motif of another
 * context). */
int tm_serve_submit_motif(tm_ctx *ctx, const tm_motif *mo, uint64_t k, uint64_t seed, uint64_t *ticket);

/* Wait at most timeout_ms for a query; on completion copy its result and
 * release the ticket.  Returns the query's own status (TM_OK, or e.g.
 * TM_E_TIMEOUT if a bounded device wait ran out), or TM_E_PENDING while it is
 * still running (the ticket stays valid). */
int tm_serve_poll(tm_ctx *ctx, uint64_t ticket, tm_result *out, int timeout_ms);

/* Counters, cache behaviour and latency percentiles since tm_serve_start. */
int tm_serve_stats(tm_ctx *ctx, tm_serve_stats_t *out);

/* Stop serving: queries being sampled finish their rounds, queued ones are
 * dropped, cached weights are freed. */
int tm_serve_stop(tm_ctx *ctx);

/* Phases timed when cfg.profile = 1 (CUDA events on the context stream). */
enum {
    TM_PH_LOAD = 0,     /* tm_graph_load copy                               */
    TM_PH_CSR = 1,      /* tm_preprocess: sorts, offsets, pair tables       */
    TM_PH_WINDOWS = 2,  /* window lists of both layers                      */
    TM_PH_DP = 3,       /* weight DP kernels (Claim 3.2)                    */
    TM_PH_PREFIX = 4,   /* segmented prefix sums of child weights           */
    TM_PH_ROOT = 5,     /* root CDF and window totals (Claim 3.4)           */
    TM_PH_SAMPLE = 6,   /* sampler + validator + DeriveCnt + reduction      */
    TM_PH_BATCH = 7,    /* batched sampler                                  */
    /* parts of TM_PH_CSR (also counted in it) */
    TM_PH_CSR_STATS = 8,   /* input checks, t range, compaction             */
    TM_PH_CSR_GLOBAL = 9,  /* sort into (t', src, dst) order and duplicates */
    TM_PH_CSR_OUT = 10,    /* out- and in-list sort (one two-array sort)    */
    TM_PH_CSR_IN = 11,     /* out- and in-list gathers and offsets          */
    TM_PH_CSR_MULTI = 12,  /* multi-edge lists and pair tables              */
    TM_NUM_PHASES = 13
};

/* Accumulated milliseconds and kernel-launch counts per phase since the last
 * call (ms[cap], launches[cap]; either may be NULL); resets the counters.
 * Returns TM_NUM_PHASES in *nphases. */
int tm_phase_times(tm_ctx *ctx, double *ms, uint64_t *launches, int cap, int *nphases);

/* Per-kernel device time, recorded when the context was created with
 * cfg.profile >= 2: an event pair on the context stream around every launch
 * (tracing; adds two event records per launch). */
typedef struct {
    char name[96];        /* kernel name, e.g. "k_sample_reg<4>" (truncated) */
    double ms;            /* summed device time since the last call           */
    uint64_t launches;
} tm_kernel_time;

/* Kernels launched on ctx since the last reset, in first-launch order: fills
 * out[0 .. min(cap, *n) - 1] and sets *n to the number of distinct kernels; a
 * call with cap > 0 then resets the sums (cap = 0 only counts).  Synchronizes
 * the context stream.  Errors: TM_E_ARG. */
int tm_kernel_times(tm_ctx *ctx, tm_kernel_time *out, uint32_t cap, uint32_t *n);

/* Host->device and device->host bytes copied by the library on ctx since the
 * last call (inputs, results, counts and status words); resets them. */
int tm_io_bytes(tm_ctx *ctx, uint64_t *h2d, uint64_t *d2h);

/* One measured shape of the batched sampler. */
typedef struct {
    int tile;            /* samples per work item             */
    int threads;         /* threads per block (128 or 256)    */
    int smem_records;    /* per-sample records in shared (1) or local (0) memory */
    int coop_min;        /* lanes per long search: 0 = one lane per sample's search;
                            n = the warp's active lanes together on searches of at
                            least n entries (tm_coop_search) */
    double ms;           /* best of two timed launches        */
} tm_tune_entry;

/* Autotune tm_batch_run for this batch: time every shape (6 tile sizes x 2
 * block sizes x 2 record placements x 2 search modes) on the same queries
 * with their sample counts scaled to about target_samples in total (0 =
 * 4e6), keep the fastest in ctx and report it in *best (and every shape in
 * table[table_cap]).  A shape changes speed only: every sample's outcome
 * depends on its seed and id alone.  Errors: TM_E_STATE (no weights),
 * TM_E_CUDA. */
int tm_autotune(tm_ctx *ctx, uint32_t nq, tm_motif *const *motifs, const uint64_t *k, const uint64_t *seed,
                uint64_t target_samples, tm_tune_entry *table, uint32_t table_cap, uint32_t *nentries,
                tm_tune_entry *best);

/* Pin the batched sampler's shape: tile (samples per work item, 0 = 2048),
 * threads per block (128 or 256; 0 = 256), per-sample records in shared (1)
 * or local (0) memory.  Errors: TM_E_ARG. */
int tm_batch_shape(tm_ctx *ctx, int tile, int threads, int smem_records);

/* Warp-cooperative searches in the samplers of ctx (tm_sample, the batched
 * and served samplers): a sample whose candidate-list pick or pair-list
 * search spans at least min_entries entries is searched by all active lanes
 * of its warp at once, each step probing one position per lane and keeping
 * the bracket a ballot finds (an (n+1)-way split instead of a halving); the
 * other samples' searches stay one lane each.  0 turns it off (the default).
 * Changes speed only: every result is identical.  Errors: TM_E_ARG. */
int tm_coop_search(tm_ctx *ctx, uint32_t min_entries);

/* Free a motif and its device weights. */
void tm_motif_free(tm_motif *mo);

#ifdef __cplusplus
}
#endif
#endif /* TIMEST_GB300_H */
