// C-ABI entry points, context and allocation, and the motif / spanning-tree
// compiler (Defs. 3.4-3.5; Sec. 3.5).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <cxxabi.h>
#include <stdlib.h>

#include <algorithm>
#include <string>
#include <vector>

#include "tm_internal.h"

namespace timest {

int set_err(tm_ctx *ctx, int code, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

int check_cuda(tm_ctx *ctx, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return TM_OK;
    cudaGetLastError();
    return set_err(ctx, TM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Blocks of at least kSpareMin bytes freed with the stream-ordered pool are
// kept (at most kSpareMax of them) and handed back to a later request of
// between half and all of their size: rebuilding a graph or a motif's weights
// then reuses its blocks without a trip through the pool, which costs
// 0.2-0.8 ms of host time per gigabyte-sized block while the stream idles.
constexpr size_t kSpareMin = (size_t)4 << 20;
constexpr size_t kSpareMax = 8;

void spare_free(tm_ctx *ctx)
{
    for (auto &b : ctx->spare) cudaFreeAsync(b.first, ctx->stream);
    ctx->spare.clear();
}

void *dalloc(tm_ctx *ctx, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (ctx->cfg.alloc) {
        p = ctx->cfg.alloc(bytes, (void *)ctx->stream, ctx->cfg.alloc_user);
    } else {
        if (bytes >= kSpareMin) {
            size_t best = ctx->spare.size();
            for (size_t i = 0; i < ctx->spare.size(); ++i) {
                const size_t sz = ctx->spare[i].second;
                if (sz >= bytes && sz / 2 <= bytes && (best == ctx->spare.size() || sz < ctx->spare[best].second))
                    best = i;
            }
            if (best < ctx->spare.size()) {
                p = ctx->spare[best].first;
                ctx->spare.erase(ctx->spare.begin() + (long)best);
                return p;
            }
        }
        if (cudaMallocAsync(&p, bytes, ctx->stream) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            if (!ctx->spare.empty()) {   // give the kept blocks back and retry once
                spare_free(ctx);
                if (cudaMallocAsync(&p, bytes, ctx->stream) != cudaSuccess) {
                    cudaGetLastError();
                    p = nullptr;
                }
            }
        }
    }
    if (!p) set_err(ctx, TM_E_NOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    return p;
}

// `bytes` must be the size the block was allocated with.
void dfree(tm_ctx *ctx, void *p, size_t bytes)
{
    if (!p) return;
    if (bytes == 0) bytes = 16;
    if (ctx->cfg.free) {
        ctx->cfg.free(p, bytes, (void *)ctx->stream, ctx->cfg.alloc_user);
        return;
    }
    if (bytes >= kSpareMin) {
        if (ctx->spare.size() >= kSpareMax) {
            cudaFreeAsync(ctx->spare.front().first, ctx->stream);
            ctx->spare.erase(ctx->spare.begin());
        }
        ctx->spare.push_back({p, bytes});
        return;
    }
    cudaFreeAsync(p, ctx->stream);
}

void *salloc(tm_ctx *ctx, size_t bytes)
{
    bytes = ((bytes ? bytes : 1) + 255) / 256 * 256;
    auto &A = ctx->arena;
    if (!A.empty()) {
        auto &c = A[ctx->arena_cur];
        if (c.used + bytes <= c.size) {
            void *p = c.base + c.used;
            c.used += bytes;
            return p;
        }
        for (size_t j = ctx->arena_cur + 1; j < A.size(); ++j)
            if (A[j].size >= bytes) {
                ctx->arena_cur = j;
                A[j].used = bytes;
                return A[j].base;
            }
    }
    size_t total = 0;
    for (auto &c : A) total += c.size;
    size_t size = std::max<size_t>(bytes, std::max<size_t>((size_t)64 << 20, total / 2));
    size = (size + 255) / 256 * 256;
    char *base = (char *)dalloc(ctx, size);
    if (!base) return nullptr;
    A.push_back({base, size, bytes});
    ctx->arena_cur = A.size() - 1;
    return base;
}

ScratchScope::ScratchScope(tm_ctx *c) : ctx(c), cur(c->arena_cur), used(c->arena.empty() ? 0 : c->arena[c->arena_cur].used) {}

ScratchScope::~ScratchScope()
{
    auto &A = ctx->arena;
    if (A.empty()) return;
    if (cur < A.size()) A[cur].used = used;
    for (size_t j = cur + 1; j < A.size(); ++j) A[j].used = 0;
    ctx->arena_cur = cur < A.size() ? cur : 0;
}

void arena_free(tm_ctx *ctx)
{
    for (auto &c : ctx->arena) dfree(ctx, c.base, c.size);
    ctx->arena.clear();
    ctx->arena_cur = 0;
}

void copy_h2d(tm_ctx *ctx, void *dst, const void *src, size_t bytes)
{
    ctx->h2d_bytes += bytes;
    cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream);
}

void copy_d2h(tm_ctx *ctx, void *dst, const void *src, size_t bytes)
{
    ctx->d2h_bytes += bytes;
    cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->stream);
}

int read_status(tm_ctx *ctx, uint32_t *bits)
{
    copy_d2h(ctx, ctx->status_host, ctx->status, 4);
    int rc = check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "stream synchronize");
    *bits = rc ? 0 : *ctx->status_host;
    if (!rc) prof_collect(ctx);
    return rc;
}

void release_weights(tm_ctx *ctx, tm_motif *mo);

static cudaEvent_t take_event(tm_ctx *ctx)
{
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return e;
}

PhaseScope::PhaseScope(tm_ctx *c, int ph) : ctx(c), phase(ph), launches0(c->kernel_launches)
{
    if (ctx->cfg.profile) {
        a = take_event(ctx);
        if (a) cudaEventRecord(a, ctx->stream);
    }
}

PhaseScope::~PhaseScope()
{
    uint64_t launches = ctx->kernel_launches - launches0;
    if (!a) {
        ctx->phase_launches[phase] += launches;
        return;
    }
    cudaEvent_t b = take_event(ctx);
    if (!b) { ctx->ev_pool.push_back(a); ctx->phase_launches[phase] += launches; return; }
    cudaEventRecord(b, ctx->stream);
    ctx->pending.push_back({phase, a, b, launches});
}

KernelTimer::KernelTimer(tm_ctx *c, const void *f) : ctx(c), fn(f)
{
    if (ctx->cfg.profile >= 2) {
        a = take_event(ctx);
        if (a) cudaEventRecord(a, ctx->stream);
    }
}

KernelTimer::~KernelTimer()
{
    if (!a) return;
    cudaEvent_t b = take_event(ctx);
    if (!b) { ctx->ev_pool.push_back(a); return; }
    cudaEventRecord(b, ctx->stream);
    ctx->pending_k.push_back({fn, a, b});
}

void prof_collect(tm_ctx *ctx)
{
    for (auto &p : ctx->pending_k) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            auto it = std::find_if(ctx->kernel_ms.begin(), ctx->kernel_ms.end(),
                                   [&](const std::pair<const void *, std::pair<double, uint64_t>> &e) { return e.first == p.fn; });
            if (it == ctx->kernel_ms.end()) ctx->kernel_ms.push_back({p.fn, {(double)ms, 1}});
            else { it->second.first += ms; it->second.second += 1; }
        } else {
            cudaGetLastError();
        }
        ctx->ev_pool.push_back(p.a);
        ctx->ev_pool.push_back(p.b);
    }
    ctx->pending_k.clear();
    for (auto &p : ctx->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
            ctx->phase_ms[p.phase] += ms;
        else cudaGetLastError();
        ctx->phase_launches[p.phase] += p.launches;
        ctx->ev_pool.push_back(p.a);
        ctx->ev_pool.push_back(p.b);
    }
    ctx->pending.clear();
}

static void free_graph(tm_ctx *ctx)
{
    for (auto &b : ctx->graph_bufs) dfree(ctx, b.first, b.second);
    ctx->graph_bufs.clear();
    ctx->g = DevGraph();
    ctx->preprocessed = false;
}

static void free_input(tm_ctx *ctx)
{
    // in_t heads the single staging block (t, then src, then dst); borrowed
    // caller arrays are not ours to free
    if (ctx->in_t && !ctx->in_borrowed) dfree(ctx, ctx->in_t, ctx->m_in * 16);
    ctx->in_borrowed = false;
    ctx->in_src = ctx->in_dst = nullptr;
    ctx->in_t = nullptr;
}

// ---- motif compiler ------------------------------------------------------
struct MotifDesc {
    int nv, ne;
    int a[kMaxE], b[kMaxE], rank[kMaxE];
};

static bool connected(const MotifDesc &M, const int *edges, int cnt)
{
    int comp[kMaxV];
    for (int v = 0; v < M.nv; ++v) comp[v] = v;
    for (int i = 0; i < cnt; ++i) {
        int ca = comp[M.a[edges[i]]], cb = comp[M.b[edges[i]]];
        if (ca == cb) continue;
        for (int v = 0; v < M.nv; ++v) if (comp[v] == cb) comp[v] = ca;
    }
    for (int v = 1; v < M.nv; ++v) if (comp[v] != comp[0]) return false;
    return true;
}

static bool is_spanning_tree(const MotifDesc &M, const int *edges)
{
    int comp[kMaxV];
    for (int v = 0; v < M.nv; ++v) comp[v] = v;
    for (int i = 0; i < M.nv - 1; ++i) {
        int e = edges[i];
        if (e < 0 || e >= M.ne) return false;
        int ca = comp[M.a[e]], cb = comp[M.b[e]];
        if (ca == cb) return false;
        for (int v = 0; v < M.nv; ++v) if (comp[v] == cb) comp[v] = ca;
    }
    return true;
}

// Constraint looseness of a tree (Alg. 8, summed over pairs of tree edges
// that share a vertex): sum of |pi(e1) - pi(e2)| - 1.
static int looseness(const MotifDesc &M, const int *edges)
{
    int L = 0;
    for (int v = 0; v < M.nv; ++v)
        for (int i = 0; i < M.nv - 1; ++i)
            for (int j = i + 1; j < M.nv - 1; ++j) {
                int e1 = edges[i], e2 = edges[j];
                bool in1 = M.a[e1] == v || M.b[e1] == v, in2 = M.a[e2] == v || M.b[e2] == v;
                if (in1 && in2) L += std::abs(M.rank[e1] - M.rank[e2]) - 1;
            }
    return L;
}

// Root of least eccentricity in the tree's edge-adjacency graph (ties: lower id).
static int default_root(const MotifDesc &M, const int *edges)
{
    int nt = M.nv - 1, best = -1, bestecc = 1 << 30;
    for (int i = 0; i < nt; ++i) {
        int dist[kMaxTree];
        for (int j = 0; j < nt; ++j) dist[j] = -1;
        dist[i] = 0;
        int queue[kMaxTree], h = 0, t = 0;
        queue[t++] = i;
        while (h < t) {
            int x = queue[h++];
            for (int y = 0; y < nt; ++y) {
                if (dist[y] >= 0) continue;
                int ex = edges[x], ey = edges[y];
                bool adj = M.a[ex] == M.a[ey] || M.a[ex] == M.b[ey] || M.b[ex] == M.a[ey] || M.b[ex] == M.b[ey];
                if (adj) { dist[y] = dist[x] + 1; queue[t++] = y; }
            }
        }
        int ecc = 0;
        for (int j = 0; j < nt; ++j) ecc = std::max(ecc, dist[j]);
        if (ecc < bestecc || (ecc == bestecc && edges[i] < best)) { bestecc = ecc; best = edges[i]; }
    }
    return best;
}

// Every spanning tree, ranked as in Alg. 7: least looseness first, ties to
// the lexicographically smallest edge set (the enumeration order, kept by a
// stable sort).
struct RankedTree {
    uint32_t mask;
    int L;
    int edges[kMaxTree];
};

static void rank_trees(const MotifDesc &M, std::vector<RankedTree> &out)
{
    out.clear();
    const int k = M.nv - 1;
    int idx[kMaxTree];
    for (int i = 0; i < k; ++i) idx[i] = i;
    // lexicographic enumeration of k-subsets of the ne edges
    for (;;) {
        if (is_spanning_tree(M, idx)) {
            RankedTree r;
            r.mask = 0;
            for (int i = 0; i < k; ++i) { r.edges[i] = idx[i]; r.mask |= 1u << idx[i]; }
            r.L = looseness(M, idx);
            out.push_back(r);
        }
        int i = k - 1;
        while (i >= 0 && idx[i] == M.ne - k + i) --i;
        if (i < 0) break;
        ++idx[i];
        for (int j = i + 1; j < k; ++j) idx[j] = idx[j - 1] + 1;
    }
    std::stable_sort(out.begin(), out.end(), [](const RankedTree &a, const RankedTree &b) { return a.L < b.L; });
}

static void default_tree(const MotifDesc &M, int *tree_out, int *root_out)
{
    std::vector<RankedTree> R;
    rank_trees(M, R);   // a connected motif has at least one spanning tree
    for (int i = 0; i < M.nv - 1; ++i) tree_out[i] = R[0].edges[i];
    *root_out = default_root(M, tree_out);
}

// Check a motif description (the arguments of tm_set_motif) and fill M.
static int parse_motif(uint32_t nv, uint32_t ne, const uint32_t *edges, const uint32_t *order, MotifDesc &M,
                       const char **why)
{
    *why = "";
    if (!edges || !order) { *why = "null motif array"; return TM_E_ARG; }
    if (nv < 2 || nv > (uint32_t)kMaxV || ne < nv - 1 || ne > (uint32_t)kMaxE) {
        *why = "motif needs 2..8 vertices and nv-1..16 edges";
        return TM_E_MOTIF;
    }
    M.nv = (int)nv; M.ne = (int)ne;
    bool seen[kMaxE] = {};
    for (uint32_t i = 0; i < ne; ++i) {
        uint32_t a = edges[2 * i], b = edges[2 * i + 1];
        if (a >= nv || b >= nv || a == b) { *why = "motif edge out of range or self loop"; return TM_E_MOTIF; }
        if (order[i] >= ne || seen[order[i]]) { *why = "order is not a permutation"; return TM_E_MOTIF; }
        seen[order[i]] = true;
        M.a[i] = (int)a; M.b[i] = (int)b; M.rank[i] = (int)order[i];
    }
    int all[kMaxE];
    for (int i = 0; i < M.ne; ++i) all[i] = i;
    if (!connected(M, all, M.ne)) { *why = "motif is not connected"; return TM_E_MOTIF; }
    return TM_OK;
}

// Root the tree at `root` and lay it out in sampling order: breadth first;
// children of the root at its tail, then at its head; a node's children in
// increasing motif-edge index (the draw order of the counter-based streams).
static int compile_plan(const MotifDesc &M, const int *tree, int root, int64_t delta, DevPlan &P)
{
    memset(&P, 0, sizeof(P));
    P.nv = M.nv; P.ne = M.ne; P.ntree = M.nv - 1;
    P.delta = std::min<int64_t>(delta, (int64_t)1 << 33);
    P.wdelta = P.delta;
    P.c2 = 1;
    bool in_tree[kMaxE] = {};
    for (int i = 0; i < P.ntree; ++i) in_tree[tree[i]] = true;
    if (!in_tree[root]) return TM_E_MOTIF;
    for (int e = 0; e < M.ne; ++e) {
        P.ea[e] = M.a[e]; P.eb[e] = M.b[e]; P.rank[e] = M.rank[e];
        P.pos_edge[M.rank[e]] = e;
        P.is_tree[e] = in_tree[e] ? 1 : 0;
    }
    int lower[kMaxTree];           // lower endpoint of each node (-1 for the root)
    bool placed[kMaxE] = {};
    int nq = 0;
    P.tedge[0] = root; P.tparent[0] = -1; lower[0] = -1; placed[root] = true; nq = 1;
    for (int h = 0; h < nq; ++h) {
        int s = P.tedge[h];
        int zs[2], nz;
        if (h == 0) { zs[0] = M.a[s]; zs[1] = M.b[s]; nz = 2; }
        else { zs[0] = lower[h]; nz = 1; }
        for (int k = 0; k < nz; ++k) {
            int z = zs[k];
            for (int e = 0; e < M.ne; ++e) {
                if (!in_tree[e] || placed[e] || (M.a[e] != z && M.b[e] != z)) continue;
                placed[e] = true;
                int q = nq++;
                P.tedge[q] = e;
                P.tparent[q] = h;
                P.tzside[q] = (M.a[s] == z) ? 0 : 1;
                P.tout[q] = (M.a[e] == z) ? 1 : 0;
                P.tlater[q] = (M.rank[e] > M.rank[s]) ? 1 : 0;
                lower[q] = (M.a[e] == z) ? M.b[e] : M.a[e];
                P.child[h][P.nchild[h]++] = q;
            }
        }
    }
    if (nq != P.ntree) return TM_E_MOTIF;
    int slot = 0;
    for (int q = P.ntree - 1; q >= 0; --q) {
        int hmax = -1;
        for (int c = 0; c < P.nchild[q]; ++c) hmax = std::max(hmax, P.height[P.child[q][c]]);
        P.height[q] = hmax + 1;
        P.tleaf[q] = P.nchild[q] == 0 ? 1 : 0;
    }
    for (int q = 0; q < P.ntree; ++q) P.tslot[q] = (q > 0 && !P.tleaf[q]) ? slot++ : -1;
    P.nslots = slot;
    // non-tree edges along pi and their neighbouring tree positions
    for (int e = 0; e < M.ne; ++e) P.tnode_of_edge[e] = -1;
    for (int q = 0; q < P.ntree; ++q) P.tnode_of_edge[P.tedge[q]] = q;
    P.nnt = 0;
    P.derive_simple = 1;
    for (int pos = 0; pos < M.ne; ++pos) {
        int e = P.pos_edge[pos];
        if (P.tnode_of_edge[e] >= 0) continue;
        int i = P.nnt++;
        P.nt_pos[i] = pos;
        P.nt_prev[i] = -1;
        P.nt_next[i] = -1;
        for (int b = pos - 1; b >= 0; --b)
            if (P.tnode_of_edge[P.pos_edge[b]] >= 0) { P.nt_prev[i] = P.tnode_of_edge[P.pos_edge[b]]; break; }
        for (int a = pos + 1; a < M.ne; ++a)
            if (P.tnode_of_edge[P.pos_edge[a]] >= 0) { P.nt_next[i] = P.tnode_of_edge[P.pos_edge[a]]; break; }
        if (pos > 0 && P.tnode_of_edge[P.pos_edge[pos - 1]] < 0) P.derive_simple = 0;
    }
    P.coupled = (P.nnt > 0 && P.nt_pos[0] == 0 && P.nt_pos[P.nnt - 1] == M.ne - 1) ? 1 : 0;
    return TM_OK;
}

// A kernel's name without namespaces and parameter list, e.g.
// "k_sample_reg<4>" (demangled when the runtime reports a mangled name).
static std::string short_kernel_name(const char *raw)
{
    std::string s = raw;
    int status = 0;
    char *dm = abi::__cxa_demangle(raw, nullptr, nullptr, &status);
    if (status == 0 && dm) s = dm;
    free(dm);
    const char *drop[] = {"timest::", "(anonymous namespace)::", "void "};
    for (const char *d : drop)
        for (size_t p; (p = s.find(d)) != std::string::npos;) s.erase(p, strlen(d));
    // cut the parameter list: the first '(' outside template brackets
    int depth = 0;
    for (size_t i = 0; i < s.size(); ++i) {
        if (s[i] == '<') ++depth;
        else if (s[i] == '>') --depth;
        else if (s[i] == '(' && depth == 0) { s.resize(i); break; }
    }
    return s;
}

}  // namespace timest

using namespace timest;

extern "C" {

void tm_config_default(tm_config *cfg)
{
    if (!cfg) return;
    memset(cfg, 0, sizeof(*cfg));
}

int tm_create(tm_ctx **out, const tm_config *cfg, void *cuda_stream)
{
    if (!out) return TM_E_ARG;
    *out = nullptr;
    tm_ctx *ctx = new tm_ctx();
    if (cfg) ctx->cfg = *cfg;
    else tm_config_default(&ctx->cfg);
    if ((ctx->cfg.alloc == nullptr) != (ctx->cfg.free == nullptr)) { delete ctx; return TM_E_ARG; }
    ctx->device = ctx->cfg.device;
    int rc = check_cuda(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    if (!rc && !ctx->cfg.alloc) {
        // keep freed blocks in this process's stream-ordered pool for reuse
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    }
    if (!rc) rc = check_cuda(ctx, cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device),
                             "device attributes");
    if (!rc) {
        if (cuda_stream) ctx->stream = (cudaStream_t)cuda_stream;
        else { rc = check_cuda(ctx, cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking), "stream"); ctx->own_stream = true; }
    }
    if (!rc) rc = check_cuda(ctx, cudaMallocHost((void **)&ctx->status_host, 64), "pinned status");
    if (!rc) {
        ctx->status = (uint32_t *)dalloc(ctx, 64);
        if (!ctx->status) rc = TM_E_NOMEM;
        else cudaMemsetAsync(ctx->status, 0, 64, ctx->stream);
    }
    if (rc) { tm_destroy(ctx); return rc; }
    *out = ctx;
    return TM_OK;
}

void tm_destroy(tm_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->server) tm_serve_stop(ctx);
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    prof_collect(ctx);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    ctx->ev_pool.clear();
    free_input(ctx);
    free_graph(ctx);
    arena_free(ctx);
    spare_free(ctx);
    if (ctx->status) dfree(ctx, ctx->status, 64);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->status_host) cudaFreeHost(ctx->status_host);
    if (ctx->pinned_acc) cudaFreeHost(ctx->pinned_acc);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char *tm_last_error(tm_ctx *ctx)
{
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

int tm_graph_load(tm_ctx *ctx, uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst, const int64_t *t,
                  int flags)
{
    if (!ctx) return TM_E_ARG;
    if (m && (!src || !dst || !t)) return set_err(ctx, TM_E_ARG, "null edge array");
    if (n == 0 || n >= 0xFFFFFFFFu) return set_err(ctx, TM_E_LIMIT, "vertex count must be in [1, 2^32-2]");
    if (m >= 0xFFFFFFFFull) return set_err(ctx, TM_E_LIMIT, "edge count must be below 2^32-1");
    cudaSetDevice(ctx->device);
    free_input(ctx);
    free_graph(ctx);
    ctx->epoch++;
    ctx->loaded = false;
    ctx->n = n;
    ctx->m_in = m;
    ctx->load_flags = flags;
    if (m && (flags & TM_DEVICE) && (flags & TM_PREPROCESS)) {
        // build straight from the caller's device arrays, valid for this call
        ctx->in_src = const_cast<uint32_t *>(src);
        ctx->in_dst = const_cast<uint32_t *>(dst);
        ctx->in_t = const_cast<int64_t *>(t);
        ctx->in_borrowed = true;
        ctx->loaded = true;
        const int rc = tm_preprocess(ctx);
        if (ctx->in_borrowed) {   // failed: the caller's arrays are not kept
            free_input(ctx);
            ctx->loaded = false;
        }
        return rc;
    }
    if (m) {
        char *blk = (char *)dalloc(ctx, m * 16);
        if (!blk) return TM_E_NOMEM;
        ctx->in_t = (int64_t *)blk;
        ctx->in_src = (uint32_t *)(blk + m * 8);
        ctx->in_dst = (uint32_t *)(blk + m * 12);
        cudaMemcpyKind kind = (flags & TM_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        {
            PhaseScope ph(ctx, TM_PH_LOAD);
            if (kind == cudaMemcpyHostToDevice) ctx->h2d_bytes += m * 16;
            cudaMemcpyAsync(ctx->in_src, src, m * 4, kind, ctx->stream);
            cudaMemcpyAsync(ctx->in_dst, dst, m * 4, kind, ctx->stream);
            cudaMemcpyAsync(ctx->in_t, t, m * 8, kind, ctx->stream);
        }
        int rc = check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "graph copy");
        prof_collect(ctx);
        if (rc) { free_input(ctx); return rc; }
    }
    ctx->loaded = true;
    return (flags & TM_PREPROCESS) ? tm_preprocess(ctx) : TM_OK;
}

int tm_preprocess(tm_ctx *ctx)
{
    if (!ctx) return TM_E_ARG;
    if (!ctx->loaded) return set_err(ctx, TM_E_STATE, "no graph loaded");
    cudaSetDevice(ctx->device);
    free_graph(ctx);
    int rc;
    {
        PhaseScope ph(ctx, TM_PH_CSR);
        rc = build_csr(ctx);
    }
    cudaStreamSynchronize(ctx->stream);
    prof_collect(ctx);
    if (rc) { free_graph(ctx); return rc; }
    free_input(ctx);
    ctx->loaded = false;
    ctx->preprocessed = true;
    return TM_OK;
}

int tm_graph_info(tm_ctx *ctx, uint64_t *m, int64_t *t_min, int64_t *T)
{
    if (!ctx) return TM_E_ARG;
    if (!ctx->preprocessed) return set_err(ctx, TM_E_STATE, "graph not preprocessed");
    if (m) *m = ctx->g.m;
    if (t_min) *t_min = ctx->g.tmin;
    if (T) *T = ctx->g.T;
    return TM_OK;
}

int tm_edges_export(tm_ctx *ctx, uint32_t *src, uint32_t *dst, uint32_t *tprime)
{
    if (!ctx) return TM_E_ARG;
    if (!ctx->preprocessed) return set_err(ctx, TM_E_STATE, "graph not preprocessed");
    size_t b = (size_t)ctx->g.m * 4;
    if (b) {
        if (src) copy_d2h(ctx, src, ctx->g.g_src, b);
        if (dst) copy_d2h(ctx, dst, ctx->g.g_dst, b);
        if (tprime) copy_d2h(ctx, tprime, ctx->g.g_t, b);
    }
    return check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "edge export");
}

int tm_csr_export(tm_ctx *ctx, int array, uint32_t *host_out, uint64_t cap, uint64_t *len)
{
    if (!ctx) return TM_E_ARG;
    if (!ctx->preprocessed) return set_err(ctx, TM_E_STATE, "graph not preprocessed");
    const DevGraph &g = ctx->g;
    const uint64_t m = g.m, n1 = (uint64_t)g.n + 1, words = m / 32 + 1;
    const uint32_t *src = nullptr;
    uint64_t cnt = m;
    switch (array) {
    case TM_CSR_OUT_OFF: src = g.out_off; cnt = n1; break;
    case TM_CSR_OUT_T: src = g.out_t; break;
    case TM_CSR_OUT_NBR: src = g.out_nbr; break;
    case TM_CSR_OUT_GID: src = g.out_gid; break;
    case TM_CSR_OUT_SRC: src = g.out_src; break;
    case TM_CSR_OUT_POS: src = g.out_pos; break;
    case TM_CSR_OUT_XRANK: src = g.out_xrank; break;
    case TM_CSR_IN_OFF: src = g.in_off; cnt = n1; break;
    case TM_CSR_IN_T: src = g.in_t; break;
    case TM_CSR_IN_NBR: src = g.in_nbr; break;
    case TM_CSR_IN_GID: src = g.in_gid; break;
    case TM_CSR_IN_DST: src = g.in_dst; break;
    case TM_CSR_IN_POS: src = g.in_pos; break;
    case TM_CSR_IN_XRANK: src = g.in_xrank; break;
    case TM_CSR_IN_TO_OUT: src = g.in_to_out; break;
    case TM_CSR_VPAIR_OFF: src = g.vpair_off; cnt = n1; break;
    case TM_CSR_PAIR_OFF: src = g.pair_off; cnt = (uint64_t)g.npairs + 1; break;
    case TM_CSR_PAIR_DST: src = g.pair_dst; cnt = g.npairs; break;
    case TM_CSR_MULTI_T: src = g.multi_t; break;
    case TM_CSR_MULTI_TO_OUT: src = g.multi_to_out; break;
    case TM_CSR_OWN_OUT: src = g.own_out; cnt = words; break;
    case TM_CSR_OWN_IN: src = g.own_in; cnt = words; break;
    case TM_CSR_OWN_MULTI: src = g.own_multi; cnt = words; break;
    default: return set_err(ctx, TM_E_ARG, "unknown CSR array");
    }
    if (len) *len = cnt;
    if (!host_out) return TM_OK;
    if (cap < cnt) return set_err(ctx, TM_E_ARG, "CSR export: cap below the array's length");
    if (cnt && src) copy_d2h(ctx, host_out, src, (size_t)cnt * 4);
    return check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "CSR export");
}

// A motif planned on (tree, root); nullptr and *rc on failure.
static tm_motif *new_motif(tm_ctx *ctx, const MotifDesc &M, const int *tree, int root, int64_t delta, int *rc)
{
    tm_motif *mo = new tm_motif();
    mo->ctx = ctx;
    mo->nv = (uint32_t)M.nv; mo->ne = (uint32_t)M.ne; mo->delta = delta;
    for (int i = 0; i < M.ne; ++i) { mo->ea[i] = M.a[i]; mo->eb[i] = M.b[i]; mo->rank[i] = M.rank[i]; }
    for (int i = 0; i < M.nv - 1; ++i) mo->tree[i] = tree[i];
    mo->root = root;
    *rc = compile_plan(M, tree, root, delta, mo->plan);
    if (*rc) { delete mo; return nullptr; }
    return mo;
}

int tm_set_motif(tm_ctx *ctx, uint32_t nv, uint32_t ne, const uint32_t *edges, const uint32_t *order, int64_t delta,
                 tm_motif **out)
{
    if (!ctx || !out || !edges || !order) return TM_E_ARG;
    *out = nullptr;
    MotifDesc M;
    const char *why;
    int rc = parse_motif(nv, ne, edges, order, M, &why);
    if (rc) return set_err(ctx, rc, why);
    if (delta <= 0) return set_err(ctx, TM_E_MOTIF, "delta must be positive");
    int tree[kMaxTree], root;
    default_tree(M, tree, &root);
    tm_motif *mo = new_motif(ctx, M, tree, root, delta, &rc);
    if (!mo) return set_err(ctx, rc, "internal: default tree did not compile");
    *out = mo;
    return TM_OK;
}

int tm_tree_candidates(uint32_t nv, uint32_t ne, const uint32_t *edges, const uint32_t *order, uint32_t max_out,
                       uint32_t *masks_out, uint32_t *looseness_out, uint32_t *n_total)
{
    MotifDesc M;
    const char *why;
    int rc = parse_motif(nv, ne, edges, order, M, &why);
    if (rc) return rc;
    std::vector<RankedTree> R;
    rank_trees(M, R);
    for (uint32_t i = 0; i < max_out && i < R.size(); ++i) {
        if (masks_out) masks_out[i] = R[i].mask;
        if (looseness_out) looseness_out[i] = (uint32_t)R[i].L;
    }
    if (n_total) *n_total = (uint32_t)R.size();
    return TM_OK;
}

static bool u128_less(const tm_u128 &a, const tm_u128 &b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

int tm_select_tree(tm_ctx *ctx, uint32_t nv, uint32_t ne, const uint32_t *edges, const uint32_t *order, int64_t delta,
                   uint32_t n_c, int all_roots, tm_motif **out, tm_tree_cand *cands, uint32_t max_cand, uint32_t *n_cand)
{
    if (!ctx || !out || !edges || !order) return TM_E_ARG;
    *out = nullptr;
    if (n_cand) *n_cand = 0;
    if (!ctx->preprocessed) return set_err(ctx, TM_E_STATE, "graph not preprocessed");
    MotifDesc M;
    const char *why;
    int rc = parse_motif(nv, ne, edges, order, M, &why);
    if (rc) return set_err(ctx, rc, why);
    if (delta <= 0) return set_err(ctx, TM_E_MOTIF, "delta must be positive");
    std::vector<RankedTree> R;
    rank_trees(M, R);
    const size_t ntry = std::min<size_t>(n_c ? n_c : 1, R.size());
    tm_motif *best = nullptr;
    tm_u128 bestW{0, 0};
    uint32_t evaluated = 0;
    for (size_t t = 0; t < ntry; ++t) {
        int roots[kMaxTree], nroots = 0;
        if (all_roots) for (int i = 0; i < M.nv - 1; ++i) roots[nroots++] = R[t].edges[i];   // increasing id
        else roots[nroots++] = default_root(M, R[t].edges);
        for (int ri = 0; ri < nroots; ++ri) {
            tm_motif *mo = new_motif(ctx, M, R[t].edges, roots[ri], delta, &rc);
            if (!mo) {
                tm_motif_free(best);
                return set_err(ctx, rc, "internal: candidate tree did not compile");
            }
            tm_u128 W{0, 0};
            const int crc = tm_weights(ctx, mo, &W);
            if (cands && evaluated < max_cand) {
                tm_tree_cand &c = cands[evaluated];
                c.tree_mask = R[t].mask;
                c.root = (uint32_t)roots[ri];
                c.looseness = (uint32_t)R[t].L;
                c.status = crc;
                c.W = crc == TM_OK ? W : tm_u128{0, 0};
            }
            ++evaluated;
            if (crc == TM_OK && (!best || u128_less(W, bestW))) {
                tm_motif_free(best);
                best = mo;
                bestW = W;
                continue;
            }
            tm_motif_free(mo);
            if (crc != TM_OK && crc != TM_E_OVERFLOW) {   // a real failure ends the search
                tm_motif_free(best);
                if (n_cand) *n_cand = evaluated;
                return crc;
            }
        }
    }
    if (n_cand) *n_cand = evaluated;
    if (!best) return set_err(ctx, TM_E_OVERFLOW, "every candidate's weight pass overflowed");
    *out = best;
    return TM_OK;
}

int tm_set_tree(tm_motif *mo, const uint32_t *tree_edge_ids, uint32_t root_edge)
{
    if (!mo || !tree_edge_ids) return TM_E_ARG;
    MotifDesc M;
    M.nv = (int)mo->nv; M.ne = (int)mo->ne;
    for (int i = 0; i < M.ne; ++i) { M.a[i] = mo->ea[i]; M.b[i] = mo->eb[i]; M.rank[i] = mo->rank[i]; }
    int tree[kMaxTree];
    for (int i = 0; i < M.nv - 1; ++i) tree[i] = (int)tree_edge_ids[i];
    if (!is_spanning_tree(M, tree)) return set_err(mo->ctx, TM_E_MOTIF, "edges do not form a spanning tree");
    DevPlan P;
    int rc = compile_plan(M, tree, (int)root_edge, mo->delta, P);
    if (rc) return set_err(mo->ctx, rc, "root edge is not a tree edge");
    release_weights(mo->ctx, mo);
    mo->plan = P;
    for (int i = 0; i < M.nv - 1; ++i) mo->tree[i] = tree[i];
    mo->root = root_edge;
    return TM_OK;
}

int tm_set_constraints(tm_motif *mo, int flags)
{
    if (!mo || (flags & ~(TM_C2 | TM_C3))) return TM_E_ARG;
    release_weights(mo->ctx, mo);
    mo->plan.c2 = (flags & TM_C2) ? 1 : 0;
    mo->plan.wdelta = (flags & TM_C3) ? mo->plan.delta : ((int64_t)1 << 33);
    return TM_OK;
}

int tm_motif_plan(tm_motif *mo, int32_t *order, int32_t *parent)
{
    if (!mo) return TM_E_ARG;
    for (int q = 0; q < mo->plan.ntree; ++q) {
        if (order) order[q] = mo->plan.tedge[q];
        if (parent) parent[q] = mo->plan.tparent[q];
    }
    return TM_OK;
}

int tm_weights(tm_ctx *ctx, tm_motif *mo, tm_u128 *W_out)
{
    if (!ctx || !mo || mo->ctx != ctx) return TM_E_ARG;
    if (!ctx->preprocessed) return set_err(ctx, TM_E_STATE, "graph not preprocessed");
    cudaSetDevice(ctx->device);
    int rc = compute_weights(ctx, mo);
    if (rc) { release_weights(ctx, mo); return rc; }
    if (W_out) *W_out = mo->W;
    return TM_OK;
}

static int need_weights(tm_ctx *ctx, tm_motif *mo)
{
    if (!ctx || !mo || mo->ctx != ctx) return TM_E_ARG;
    if (!mo->have_weights || mo->graph_epoch != ctx->epoch || !ctx->preprocessed)
        return set_err(ctx, TM_E_STATE, "weights not computed for the current graph");
    return TM_OK;
}

int tm_weights_export(tm_ctx *ctx, tm_motif *mo, uint32_t tree_edge, uint32_t layer, uint64_t *host_out)
{
    int rc = need_weights(ctx, mo);
    if (rc) return rc;
    if (layer > 1 || !host_out) return set_err(ctx, TM_E_ARG, "bad layer or null output");
    int q = -1;
    for (int i = 0; i < mo->plan.ntree; ++i) if ((uint32_t)mo->plan.tedge[i] == tree_edge) q = i;
    if (q < 0) return set_err(ctx, TM_E_ARG, "not a tree edge");
    cudaSetDevice(ctx->device);
    return export_weights(ctx, mo, q, (int)layer, host_out);
}

int tm_window_totals(tm_ctx *ctx, tm_motif *mo, uint64_t *host_out, uint64_t cap, uint64_t *nwin)
{
    int rc = need_weights(ctx, mo);
    if (rc) return rc;
    uint64_t nw = (uint64_t)ctx->g.T / (uint64_t)mo->plan.wdelta + 1;
    if (ctx->g.m == 0) nw = 1;
    if (nwin) *nwin = nw;
    if (!host_out) return TM_OK;
    // the device keeps the non-empty windows only: expand to the dense index
    std::vector<uint64_t> wc(2 * ((size_t)mo->nwtot + 1));
    std::vector<uint32_t> id0(mo->layer[0].nwin + 1), id1(mo->layer[1].nwin + 1);
    copy_d2h(ctx, wc.data(), mo->wcum, wc.size() * 8);
    copy_d2h(ctx, id0.data(), mo->layer[0].win_id, id0.size() * 4);
    copy_d2h(ctx, id1.data(), mo->layer[1].win_id, id1.size() * 4);
    rc = check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "window totals");
    if (rc) return rc;
    for (uint64_t i = 0; i < std::min(cap, nw); ++i) host_out[i] = 0;
    for (uint32_t k = 0; k < mo->nwtot; ++k) {
        uint32_t i = k < mo->layer[0].nwin ? id0[k] : id1[k - mo->layer[0].nwin];
        uint64_t tot = wc[2 * (k + 1)] - wc[2 * k];   // W_i < 2^64
        if (i < cap) host_out[i] = tot;
    }
    return TM_OK;
}

int tm_sample(tm_ctx *ctx, tm_motif *mo, uint64_t k, uint64_t seed, uint64_t first_index, tm_result *out)
{
    int rc = need_weights(ctx, mo);
    if (rc) return rc;
    if (!out) return set_err(ctx, TM_E_ARG, "null result");
    cudaSetDevice(ctx->device);
    return run_samples(ctx, mo, k, seed, first_index, out, nullptr, nullptr, nullptr);
}

int tm_sample_list(tm_ctx *ctx, tm_motif *mo, uint64_t k, uint64_t seed, uint64_t first_index, uint64_t max_inst,
                   uint32_t *inst_gids, uint64_t *inst_sample, uint64_t *n_inst)
{
    int rc = need_weights(ctx, mo);
    if (rc) return rc;
    if (!n_inst || (max_inst && (!inst_gids || !inst_sample))) return set_err(ctx, TM_E_ARG, "null listing output");
    cudaSetDevice(ctx->device);
    return run_list(ctx, mo, k, seed, first_index, max_inst, inst_gids, inst_sample, n_inst);
}

int tm_sample_group(tm_ctx *ctx, tm_motif *const *motifs, uint32_t nm, uint64_t k, uint64_t seed, uint64_t first_index,
                    tm_result *results)
{
    if (!ctx || !motifs || !results || nm == 0) return TM_E_ARG;
    if (nm > kMaxGroup) return set_err(ctx, TM_E_LIMIT, "at most 8 motifs per group");
    for (uint32_t i = 0; i < nm; ++i)
        if (!motifs[i] || motifs[i]->ctx != ctx) return set_err(ctx, TM_E_ARG, "motif of another context");
    int rc = need_weights(ctx, motifs[0]);
    if (rc) return rc;
    cudaSetDevice(ctx->device);
    return run_group(ctx, motifs, nm, k, seed, first_index, results);
}

int tm_sample_trace(tm_ctx *ctx, tm_motif *mo, uint64_t k, uint64_t seed, uint64_t first_index, uint32_t *tree_gids,
                    uint64_t *contrib, int32_t *reason, tm_result *out)
{
    int rc = need_weights(ctx, mo);
    if (rc) return rc;
    if (!out) return set_err(ctx, TM_E_ARG, "null result");
    cudaSetDevice(ctx->device);
    return run_samples(ctx, mo, k, seed, first_index, out, tree_gids, contrib, reason);
}

int tm_batch_run(tm_ctx *ctx, uint32_t nq, tm_motif *const *motifs, const uint64_t *k, const uint64_t *seed,
                 tm_result *out)
{
    if (!ctx || (nq && (!motifs || !k || !seed || !out))) return TM_E_ARG;
    for (uint32_t q = 0; q < nq; ++q) {
        int rc = need_weights(ctx, motifs[q]);
        if (rc) return rc;
    }
    cudaSetDevice(ctx->device);
    return run_batch(ctx, nq, motifs, k, seed, out);
}

int tm_io_bytes(tm_ctx *ctx, uint64_t *h2d, uint64_t *d2h)
{
    if (!ctx) return TM_E_ARG;
    if (h2d) *h2d = ctx->h2d_bytes;
    if (d2h) *d2h = ctx->d2h_bytes;
    ctx->h2d_bytes = ctx->d2h_bytes = 0;
    return TM_OK;
}

int tm_phase_times(tm_ctx *ctx, double *ms, uint64_t *launches, int cap, int *nphases)
{
    if (!ctx) return TM_E_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    prof_collect(ctx);
    for (int i = 0; i < TM_NUM_PHASES && i < cap; ++i) {
        if (ms) ms[i] = ctx->phase_ms[i];
        if (launches) launches[i] = ctx->phase_launches[i];
    }
    for (int i = 0; i < TM_NUM_PHASES; ++i) { ctx->phase_ms[i] = 0; ctx->phase_launches[i] = 0; }
    if (nphases) *nphases = TM_NUM_PHASES;
    return TM_OK;
}

int tm_kernel_times(tm_ctx *ctx, tm_kernel_time *out, uint32_t cap, uint32_t *n)
{
    if (!ctx || !n || (cap && !out)) return TM_E_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    prof_collect(ctx);
    *n = (uint32_t)ctx->kernel_ms.size();
    for (uint32_t i = 0; i < cap && i < ctx->kernel_ms.size(); ++i) {
        const auto &e = ctx->kernel_ms[i];
        memset(out[i].name, 0, sizeof(out[i].name));
        const char *raw = nullptr;
        std::string nm = "?";
        if (cudaFuncGetName(&raw, e.first) == cudaSuccess && raw) nm = short_kernel_name(raw);
        else cudaGetLastError();
        strncpy(out[i].name, nm.c_str(), sizeof(out[i].name) - 1);
        out[i].ms = e.second.first;
        out[i].launches = e.second.second;
    }
    if (cap) ctx->kernel_ms.clear();
    return TM_OK;
}

void tm_motif_free(tm_motif *mo)
{
    if (!mo) return;
    if (mo->ctx) {
        cudaSetDevice(mo->ctx->device);
        release_weights(mo->ctx, mo);
        cudaStreamSynchronize(mo->ctx->stream);
    }
    delete mo;
}

}  // extern "C"
