// Internal declarations shared by the TIMEST CUDA translation units.
// Host-side structures (context, motif, device plan) and kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/timest.h"

namespace timest {

constexpr int kMaxV = 8;
constexpr int kMaxE = 16;
constexpr int kMaxTree = kMaxV - 1;
constexpr uint32_t kNone = 0xFFFFFFFFu;

// Device status word bits (latched by kernels, read by the host at syncs).
enum : uint32_t {
    ST_OVERFLOW = 1u,      // an exact integer exceeded its width
    ST_BADSTATE = 2u,      // an internal invariant failed (e.g. empty candidate list)
    ST_TIMEOUT = 4u,       // a bounded wait ran out
    ST_DUP = 8u,
    ST_SELFLOOP = 16u,
    ST_RANGE = 32u         // an id out of range
};

// Guide table of the window pick: draws r in [j 2^s, (j+1) 2^s) fall in a
// window between wguide[j] and wguide[j+1].  s = max(0, bitlen(W) -
// bitlen(nw) - 1), so there are at most 4 nw buckets; the same function
// sizes the table (weight pass) and reads it (sampler).
__host__ __device__ inline uint32_t wguide_shift(uint64_t W_lo, uint64_t W_hi, uint32_t nw)
{
    int bw = 0;
    for (uint64_t x = W_hi; x; x >>= 1) ++bw;
    if (bw) bw += 64;
    else for (uint64_t x = W_lo; x; x >>= 1) ++bw;
    int bn = 0;
    for (uint32_t x = nw; x; x >>= 1) ++bn;
    const int s = bw - bn - 1;
    return s > 0 ? (uint32_t)s : 0u;
}

// Windows by one quotient.  With q = floor(t' / d), t' lies in windows q - 1
// and q (the windows i with i*d <= t' < (i+2)*d); the one of layer p is the
// one with parity p: q - ((q xor p) & 1), absent (-1) when that is negative.
// The quotient uses the division by an invariant integer of Granlund and
// Montgomery ("Division by invariant integers using multiplication", PLDI
// 1994, Fig. 4.1) for 32-bit dividends: with l = ceil(log2 d) and
// m' = floor(2^32 (2^l - d) / d) + 1, floor(n / d) = (t1 + ((n - t1) >> sh1)) >> sh2
// where t1 = mulhi(m', n), sh1 = min(l, 1), sh2 = max(l - 1, 0).  A unit of
// 2^32 or more leaves every t' < 2^32 in quotient 0.
struct WinDiv {
    uint32_t mul;       // m'
    uint32_t sh1, sh2;
    uint32_t big;       // 1: d >= 2^32, every quotient is 0
    int64_t d;          // the window unit
    __device__ __forceinline__ uint32_t quot(uint32_t n) const
    {
        if (big) return 0u;
        const uint32_t t1 = __umulhi(mul, n);
        return (t1 + ((n - t1) >> sh1)) >> sh2;
    }
    // window index of layer p for quotient q, or -1
    __device__ __forceinline__ static int64_t win_of(uint32_t q, int p)
    {
        return (int64_t)q - (int64_t)((q ^ (uint32_t)p) & 1u);
    }
    __device__ __forceinline__ int64_t win(uint32_t t, int p) const { return win_of(quot(t), p); }
};

inline WinDiv make_windiv(int64_t d)
{
    WinDiv w{};
    w.d = d;
    if (d >= ((int64_t)1 << 32)) { w.big = 1; w.mul = 0; w.sh1 = w.sh2 = 0; return w; }
    const uint64_t D = (uint64_t)d;
    uint32_t l = 0;
    while (l < 32 && ((uint64_t)1 << l) < D) ++l;   // l = ceil(log2 d)
    w.mul = (uint32_t)(((((uint64_t)1 << l) - D) << 32) / D + 1);
    w.sh1 = l < 1 ? l : 1;
    w.sh2 = l > 1 ? l - 1 : 0;
    w.big = 0;
    return w;
}


// The temporal graph in HBM, all structure-of-arrays, 32-bit ids.
// gid = position in GLOBAL order (t', src, dst).
struct DevGraph {
    uint32_t n = 0;
    uint32_t m = 0;
    uint32_t npairs = 0;
    int64_t tmin = 0;
    uint32_t T = 0;                      // max t'
    // GLOBAL order
    uint32_t *g_t = nullptr, *g_src = nullptr, *g_dst = nullptr;
    // out-lists: per vertex, (t', dst) order; owner (src) per position
    uint32_t *out_off = nullptr, *out_t = nullptr, *out_nbr = nullptr, *out_gid = nullptr;
    uint32_t *out_src = nullptr;
    uint32_t *out_xrank = nullptr;       // where each out-list time falls in the owner's in-list
    uint32_t *out_pos = nullptr;         // [gid] position of the edge in its source's out-list
    // in-lists: per vertex, (t', src) order; owner (dst) per position
    uint32_t *in_off = nullptr, *in_t = nullptr, *in_nbr = nullptr, *in_gid = nullptr;
    uint32_t *in_dst = nullptr;
    uint32_t *in_xrank = nullptr;        // where each in-list time falls in the owner's out-list
    uint32_t *in_pos = nullptr;          // [gid] position of the edge in its destination's in-list
    // multi-edge lists: pairs sorted by (src, dst); entries in t' order
    uint32_t *vpair_off = nullptr;       // [n+1] first pair of each source vertex
    uint32_t *pair_dst = nullptr;        // [P]
    uint32_t *pair_off = nullptr;        // [P+1] into multi_*
    uint32_t *multi_t = nullptr;
    // position maps between the list orders (same edge): in->out, multi->out
    uint32_t *in_to_out = nullptr, *multi_to_out = nullptr;
    // bit sets over list positions: bit x set when position x starts a new
    // owner (vertex for the out/in orders, pair for the multi order); m/32+1 words
    uint32_t *own_out = nullptr, *own_in = nullptr, *own_multi = nullptr;
};

// Device plan of a motif with its rooted spanning tree (Defs. 3.4-3.5).
// Tree edges are indexed by q = position in the sampling order (breadth
// first from the root edge c).
struct DevPlan {
    int32_t nv, ne, ntree;
    int32_t c2;                          // 1: Constraint 2 (distinct far endpoints) enforced
    int64_t delta;                       // capped at 2^33 (no change of meaning)
    int64_t wdelta;                      // window unit: delta, or 2^33 without Constraint 3
    int32_t ea[kMaxE], eb[kMaxE], rank[kMaxE];
    int32_t pos_edge[kMaxE];             // motif edge at pi position
    int32_t is_tree[kMaxE];
    int32_t tedge[kMaxTree];             // motif edge id of tree node q
    int32_t tparent[kMaxTree];           // parent node (-1 for the root)
    int32_t tleaf[kMaxTree];             // 1: no children (weight 1)
    int32_t tzside[kMaxTree];            // meeting vertex = parent's tail (0) / head (1)
    int32_t tout[kMaxTree];              // 1: child leaves the meeting vertex (out-list)
    int32_t tlater[kMaxTree];            // 1: child comes after the parent in pi
    int32_t tslot[kMaxTree];             // prefix-array slot (non-root, non-leaf) or -1
    int32_t nchild[kMaxTree];
    int32_t child[kMaxTree][kMaxTree];
    int32_t height[kMaxTree];
    int32_t nslots;
    // DeriveCnt layout (Alg. 5): non-tree edges by pi position
    int32_t tnode_of_edge[kMaxE];        // tree node of a motif edge, -1 if non-tree
    int32_t nnt;                         // number of non-tree edges
    int32_t nt_pos[kMaxE];               // their pi positions, increasing
    int32_t nt_prev[kMaxE];              // tree node at the previous tree position (-1: none)
    int32_t nt_next[kMaxE];              // tree node at the next tree position (-1: none)
    int32_t derive_simple;               // every run of consecutive non-tree positions has length 1
    int32_t coupled;                     // the first and the last pi positions are both non-tree
};

// Per-motif resident weight data (one window layer p = 0, 1 each).
struct LayerData {
    uint32_t nwin = 0;                   // non-empty windows of this layer
    uint32_t *win_beg = nullptr;         // [nwin+1] gid ranges (win_beg[nwin] = m)
    uint32_t *win_id = nullptr;          // [nwin] window index i
    uint64_t *root_cdf = nullptr;        // [m] running sum of w_c inside its window
    // guide table of the root search: window kk's draws r in [j 2^s, (j+1) 2^s)
    // (s = win_gshift[kk]) have their root edge in [guide[o + j], guide[o + j + 1]]
    // (o = win_goff[kk]); guide[o + j] is the first edge whose CDF exceeds j 2^s
    uint32_t *win_gshift = nullptr;      // [nwin]
    uint32_t *win_goff = nullptr;        // [nwin + 1]
    uint32_t *guide = nullptr;           // [m/4 + 3 nwin + 1]
};

struct Server;

}  // namespace timest

struct tm_motif {
    tm_ctx *ctx = nullptr;
    uint32_t nv = 0, ne = 0;
    uint32_t ea[timest::kMaxE] = {}, eb[timest::kMaxE] = {}, rank[timest::kMaxE] = {};
    int64_t delta = 0;
    uint32_t tree[timest::kMaxTree] = {};
    uint32_t root = 0;
    timest::DevPlan plan{};
    bool have_weights = false;
    uint64_t graph_epoch = 0;
    timest::LayerData layer[2];
    // per prefix slot (non-root, non-leaf tree node): the segmented prefix of
    // its weights in the order its parent scans (out- or in-list) and in the
    // multi-edge order, as (layer 0, layer 1) pairs per position
    ulonglong2 *pref_dir[timest::kMaxTree] = {};
    ulonglong2 *pref_multi[timest::kMaxTree] = {};
    uint64_t *wcum = nullptr;            // [2*(nw0+nw1+1)] u128 window cumulative (lo,hi)
    uint32_t *wguide = nullptr;          // [4*(nw0+nw1)+2] guide table of the window pick
    uint32_t nwtot = 0;
    tm_u128 W{0, 0};
    size_t bytes = 0;                    // device bytes held
    std::vector<std::pair<void *, size_t>> bufs;
};

struct tm_ctx {
    tm_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    std::string err;
    // graph
    uint64_t epoch = 0;
    bool loaded = false, preprocessed = false;
    uint32_t n = 0;
    uint64_t m_in = 0;
    int load_flags = 0;
    uint32_t *in_src = nullptr, *in_dst = nullptr;  // staged input (device)
    int64_t *in_t = nullptr;
    bool in_borrowed = false;                        // in_* point at the caller's arrays
    timest::DevGraph g;
    std::vector<std::pair<void *, size_t>> graph_bufs;
    uint32_t *status = nullptr;          // device status word
    uint32_t *status_host = nullptr;     // pinned: [0] status mirror, [1] the CSR build's pair count
    int num_sms = 0;
    // phase timing (cfg.profile)
    struct PendingPhase { int phase; cudaEvent_t a, b; uint64_t launches; };
    std::vector<cudaEvent_t> ev_pool;
    std::vector<PendingPhase> pending;
    double phase_ms[TM_NUM_PHASES] = {};
    uint64_t h2d_bytes = 0, d2h_bytes = 0;     // host<->device traffic issued
    uint64_t kernel_launches = 0;              // kernels launched by this context
    // scratch arena: device chunks reused last-in first-out across calls
    struct ArenaChunk { char *base; size_t size; size_t used; };
    std::vector<ArenaChunk> arena;
    size_t arena_cur = 0;
    // large blocks freed through dfree, kept for reuse by a later dalloc of a
    // similar size (stream-ordered on this context's stream)
    std::vector<std::pair<void *, size_t>> spare;
    timest::Server *server = nullptr;          // serving loop (serve.cu), if running
    int batch_threads = 256;                   // batched sampler shape (set by tm_autotune)
    int batch_smem_recs = 0;
    uint32_t coop_min = 0xFFFFFFFFu;           // warp-cooperative searches from this length (tm_coop_search)
    void *pinned_acc = nullptr;                // staging for batched sums (device -> host)
    size_t pinned_acc_bytes = 0;
    uint64_t phase_launches[TM_NUM_PHASES] = {};
    // per-kernel timing (cfg.profile >= 2): an event pair around every launch
    struct PendingKernel { const void *fn; cudaEvent_t a, b; };
    std::vector<PendingKernel> pending_k;
    std::vector<std::pair<const void *, std::pair<double, uint64_t>>> kernel_ms;   // fn -> (ms, launches)
};

namespace timest {

// ---- allocation helpers (api.cu) ----
void *dalloc(tm_ctx *ctx, size_t bytes);
void dfree(tm_ctx *ctx, void *p, size_t bytes);

// ---- scratch arena (api.cu) ----
// salloc hands out 256-byte aligned scratch from the context's chunks; a
// ScratchScope returns everything allocated inside it when it closes.  All
// work runs on the context stream, so reuse is ordered after earlier use.
void *salloc(tm_ctx *ctx, size_t bytes);
struct ScratchScope {
    tm_ctx *ctx;
    size_t cur, used;
    explicit ScratchScope(tm_ctx *c);
    ~ScratchScope();
};
void arena_free(tm_ctx *ctx);
void spare_free(tm_ctx *ctx);

// ---- CSR build (csr.cu) ----
int build_csr(tm_ctx *ctx);

// ---- weights (weights.cu) ----
int compute_weights(tm_ctx *ctx, tm_motif *mo);
int export_weights(tm_ctx *ctx, tm_motif *mo, int q, int layer, uint64_t *host_out);

// ---- sampler (sampler.cu) ----
struct SampleJob {
    const DevPlan *plan;                 // device pointer
    const uint64_t *wcum;                // u128 pairs
    const uint32_t *wguide;              // guide table of the window pick (shift wshift)
    uint32_t wshift;
    WinDiv wv;                           // divider of the window unit (N_phi)
    uint32_t coop_min;                   // searches of at least this many entries are warp-cooperative
    uint32_t nwtot, nw0;
    const uint32_t *win_beg0, *win_beg1, *win_id0, *win_id1;
    const uint64_t *root_cdf0, *root_cdf1;
    const uint32_t *win_gshift0, *win_gshift1, *win_goff0, *win_goff1, *guide0, *guide1;
    const ulonglong2 *pref_dir[kMaxTree];     // (layer 0, layer 1) prefix pairs per slot
    const ulonglong2 *pref_multi[kMaxTree];
    uint64_t W_lo, W_hi;
};
int run_samples(tm_ctx *ctx, tm_motif *mo, uint64_t k, uint64_t seed, uint64_t first,
                tm_result *out, uint32_t *trace_gids, uint64_t *trace_contrib, int32_t *trace_reason);
int run_list(tm_ctx *ctx, tm_motif *mo, uint64_t k, uint64_t seed, uint64_t first, uint64_t max_inst,
             uint32_t *inst_gids, uint64_t *inst_sample, uint64_t *n_inst);
constexpr uint32_t kMaxGroup = 8;         // motifs per group sampling run
int run_group(tm_ctx *ctx, tm_motif *const *motifs, uint32_t nm, uint64_t k, uint64_t seed, uint64_t first,
              tm_result *out);
int run_batch(tm_ctx *ctx, uint32_t nq, tm_motif *const *motifs, const uint64_t *k,
              const uint64_t *seed, tm_result *out);

// Sums of one sample range (device accumulators, host copy).
struct SampleAcc {
    unsigned long long hits_lo, hits_hi, valid, rv, rd, ro;
};
// One query's share of a batched launch: sample ids first .. first+count-1.
struct BatchItem {
    tm_motif *mo;
    uint64_t seed, first, count;
};
// Launch the persistent batched sampler over the items (tiles of `tile`
// samples) and copy each item's sums to acc[i].  wait_ms > 0 bounds the wait
// for the GPU (TM_E_TIMEOUT when it runs out); 0 waits for completion.
int run_batch_items(tm_ctx *ctx, const BatchItem *items, uint32_t n, uint32_t tile, SampleAcc *acc, int wait_ms);
// Fold sums into a result (estimate = W * hits2 / (2k)).
void finish_result_acc(tm_motif *mo, uint64_t k, const SampleAcc &a, tm_result *out);

// ---- phase timing ----
// Scope that records CUDA events around a group of launches of one phase;
// the elapsed time is folded in by prof_collect() after the next sync.
struct PhaseScope {
    tm_ctx *ctx;
    int phase;
    cudaEvent_t a = nullptr;
    uint64_t launches0 = 0;
    PhaseScope(tm_ctx *c, int ph);
    ~PhaseScope();
};

// Per-kernel timing of one launch (cfg.profile >= 2): events recorded on the
// context stream before and after it; folded in by prof_collect().
struct KernelTimer {
    tm_ctx *ctx;
    const void *fn;
    cudaEvent_t a = nullptr;
    KernelTimer(tm_ctx *c, const void *f);
    ~KernelTimer();
};

// Every kernel of the library is launched through here (counted per context,
// timed per kernel when cfg.profile >= 2).
#ifdef __CUDACC__
template <typename... KArgs, typename... Args>
inline void launch(tm_ctx *ctx, void (*kernel)(KArgs...), dim3 grid, dim3 block, Args &&...args)
{
    ++ctx->kernel_launches;
    KernelTimer kt(ctx, (const void *)kernel);
    kernel<<<grid, block, 0, ctx->stream>>>(static_cast<KArgs>(args)...);
}
// The same with dynamic shared memory.
template <typename... KArgs, typename... Args>
inline void launch_smem(tm_ctx *ctx, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, Args &&...args)
{
    ++ctx->kernel_launches;
    KernelTimer kt(ctx, (const void *)kernel);
    kernel<<<grid, block, smem, ctx->stream>>>(static_cast<KArgs>(args)...);
}
#endif
void prof_collect(tm_ctx *ctx);   // call after the stream is synchronized

// ---- counted host<->device copies on the context stream ----
void copy_h2d(tm_ctx *ctx, void *dst, const void *src, size_t bytes);
void copy_d2h(tm_ctx *ctx, void *dst, const void *src, size_t bytes);

// ---- common ----
int check_cuda(tm_ctx *ctx, cudaError_t e, const char *what);
int set_err(tm_ctx *ctx, int code, const std::string &msg);
int read_status(tm_ctx *ctx, uint32_t *bits);   // syncs the stream
void fill_job(tm_motif *mo, SampleJob &job, const DevPlan *dplan);

}  // namespace timest
