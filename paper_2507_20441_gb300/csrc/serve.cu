// Serving: continuous batching of (motif, delta, k, seed) queries over one
// device-resident graph.
//
// Three parties share a context while serving:
//   * callers submit queries and poll for results (thread safe);
//   * the admission thread looks each query's weights up in a cache keyed by
//     (motif, order, delta); on a miss it waits until the resident weights
//     fit the memory budget (evicting least-recently-used weights that no
//     query holds), then computes them on its own stream through a second
//     context that shares the graph, so weight passes overlap the sampling
//     rounds of queries already admitted;
//   * the scheduler thread keeps up to max_active admitted queries in flight
//     and runs rounds of the batched sampler: each round gives every active
//     query its next range of sample ids, so queries join and leave between
//     rounds and their tiles share every launch.
// Every query draws samples 0..k-1 from its own counter-based streams and the
// sums of a query's rounds are exact integers, so a result does not depend on
// which other queries it shared rounds with: it equals tm_sample on the
// query's plan (its default tree, or the tree, root and constraint settings
// of a motif handle submitted with tm_serve_submit_motif) with the same k and
// seed.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "tm_internal.h"

namespace timest {
namespace {

using Clock = std::chrono::steady_clock;

// Back-off when device memory runs out: attempts and the wait between them.
constexpr int kNoMemRetries = 200;
constexpr int kNoMemWaitMs = 20;

struct Request {
    uint64_t ticket = 0;
    std::string key;
    uint32_t nv = 0, ne = 0;
    std::vector<uint32_t> edges, order;
    int64_t delta = 0;
    // a pinned plan (tm_serve_submit_motif): tree edges, root and constraint
    // flags to apply after tm_set_motif; pinned = false keeps the default
    bool pinned = false;
    std::vector<uint32_t> tree;
    uint32_t root = 0;
    int cflags = TM_C2 | TM_C3;
    uint64_t k = 0, seed = 0;
    Clock::time_point t_submit;
    // progress
    tm_motif *mo = nullptr;
    uint64_t next = 0;
    SampleAcc acc{0, 0, 0, 0, 0, 0};
    int rc = TM_OK;
    tm_result result{};
    double latency_ms = 0.0;
};

struct CacheEntry {
    tm_motif *mo = nullptr;
    size_t bytes = 0;
    int refs = 0;
    uint64_t last_use = 0;
};

}  // namespace

struct Server {
    tm_ctx *main = nullptr;
    tm_ctx *shadow = nullptr;
    tm_serve_cfg cfg{};
    std::mutex mu;
    std::condition_variable cv_admit, cv_sched, cv_done;
    std::deque<Request *> pending, ready;
    std::vector<Request *> active;
    std::map<uint64_t, Request *> done;
    std::map<std::string, CacheEntry> cache;
    size_t resident = 0;
    uint64_t use_clock = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread admit_thr, sched_thr;
    // statistics
    uint64_t submitted = 0, completed = 0, failed = 0, hits = 0, misses = 0, evictions = 0, rounds = 0;
    uint64_t admit_retries = 0, round_retries = 0;   // back-offs after TM_E_NOMEM
    std::vector<double> latencies;
    Clock::time_point t_first_submit, t_last_done;
    bool any_submit = false;
};

namespace {

void add_acc(SampleAcc &a, const SampleAcc &b)
{
    unsigned long long lo = a.hits_lo + b.hits_lo;
    a.hits_hi += b.hits_hi + (lo < a.hits_lo ? 1 : 0);
    a.hits_lo = lo;
    a.valid += b.valid;
    a.rv += b.rv;
    a.rd += b.rd;
    a.ro += b.ro;
}

std::string make_key(uint32_t nv, uint32_t ne, const uint32_t *edges, const uint32_t *order, int64_t delta)
{
    std::string s = std::to_string(nv) + ":" + std::to_string(delta) + ":";
    for (uint32_t i = 0; i < ne; ++i)
        s += std::to_string(edges[2 * i]) + ">" + std::to_string(edges[2 * i + 1]) + "@" + std::to_string(order[i]) + ",";
    return s;
}

// Device bytes a motif's resident weights will need (root CDF and its guide
// table, prefix slots, window lists), before they are computed.
size_t estimate_bytes(const tm_motif *mo, uint64_t m, uint64_t T)
{
    uint64_t slots = (uint64_t)mo->plan.nslots;
    uint64_t nwin = T / (uint64_t)std::max<int64_t>(1, mo->plan.wdelta) + 2;
    nwin = std::min<uint64_t>(nwin, m + 2);
    // root CDF 16 B and root-search guide about 2 B per edge, 32 B per prefix slot
    return (size_t)((18 + 32 * slots) * std::max<uint64_t>(m, 1) + 96 * nwin + 4096);
}

void finish_locked(Server *S, Request *r)
{
    r->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - r->t_submit).count();
    if (r->rc == TM_OK) {
        finish_result_acc(r->mo, r->k, r->acc, &r->result);
        S->completed++;
        S->latencies.push_back(r->latency_ms);
    } else {
        S->failed++;
    }
    S->t_last_done = Clock::now();
    if (r->mo) {
        auto it = S->cache.find(r->key);
        if (it != S->cache.end() && it->second.refs > 0) it->second.refs--;
    }
    S->done[r->ticket] = r;
    S->cv_done.notify_all();
    S->cv_admit.notify_all();
}

// A request whose weights are cached joins the ready queue at once (holding
// a reference to them); false when they are not resident.  Caller holds mu.
bool admit_cached_locked(Server *S, Request *r)
{
    auto it = S->cache.find(r->key);
    if (it == S->cache.end()) return false;
    it->second.refs++;
    it->second.last_use = ++S->use_clock;
    r->mo = it->second.mo;
    S->hits++;
    S->ready.push_back(r);
    S->cv_sched.notify_all();
    return true;
}

void admit_loop(Server *S)
{
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_admit.wait(lk, [&] { return S->stop || !S->pending.empty(); });
        if (S->stop) return;
        // queued requests whose weights became resident (an earlier miss of
        // the same plan) go first: a miss's weight pass blocks no hit
        for (auto q = S->pending.begin(); q != S->pending.end();) {
            if (admit_cached_locked(S, *q)) q = S->pending.erase(q);
            else ++q;
        }
        if (S->pending.empty()) continue;
        Request *r = S->pending.front();
        // miss: build the plan, then wait for room under the budget
        lk.unlock();
        tm_motif *mo = nullptr;
        int rc = tm_set_motif(S->shadow, r->nv, r->ne, r->edges.data(), r->order.data(), r->delta, &mo);
        if (!rc && r->pinned) {
            rc = tm_set_tree(mo, r->tree.data(), r->root);
            if (!rc) rc = tm_set_constraints(mo, r->cflags);
            if (rc) { tm_motif_free(mo); mo = nullptr; }
        }
        lk.lock();
        if (rc) {
            S->pending.pop_front();
            r->rc = rc;
            finish_locked(S, r);
            continue;
        }
        size_t need = estimate_bytes(mo, S->shadow->g.m, S->shadow->g.T);
        for (;;) {
            if (S->stop) { lk.unlock(); tm_motif_free(mo); lk.lock(); return; }
            if (S->resident + need <= S->cfg.weight_budget) break;
            // evict the least recently used weights nobody holds
            auto victim = S->cache.end();
            for (auto c = S->cache.begin(); c != S->cache.end(); ++c)
                if (c->second.refs == 0 && (victim == S->cache.end() || c->second.last_use < victim->second.last_use))
                    victim = c;
            if (victim != S->cache.end()) {
                tm_motif *vm = victim->second.mo;
                S->resident -= victim->second.bytes;
                S->cache.erase(victim);
                S->evictions++;
                lk.unlock();
                tm_motif_free(vm);
                lk.lock();
                continue;
            }
            if (S->cache.empty() && S->active.empty() && S->ready.empty()) break;   // alone: admit regardless
            S->cv_admit.wait_for(lk, std::chrono::milliseconds(50));
        }
        lk.unlock();
        tm_u128 W;
        rc = tm_weights(S->shadow, mo, &W);
        lk.lock();
        // out of device memory: free the cached weights that no query holds,
        // wait for the queries in flight to release theirs, and try again a
        // bounded number of times before the query fails with TM_E_NOMEM
        for (int attempt = 0; rc == TM_E_NOMEM && attempt < kNoMemRetries && !S->stop; ++attempt) {
            S->admit_retries++;
            std::vector<tm_motif *> freed;
            for (auto c = S->cache.begin(); c != S->cache.end();) {
                if (c->second.refs == 0) {
                    freed.push_back(c->second.mo);
                    S->resident -= c->second.bytes;
                    S->evictions++;
                    c = S->cache.erase(c);
                } else {
                    ++c;
                }
            }
            lk.unlock();
            for (tm_motif *vm : freed) tm_motif_free(vm);
            lk.lock();
            S->cv_admit.wait_for(lk, std::chrono::milliseconds(kNoMemWaitMs));
            lk.unlock();
            rc = tm_weights(S->shadow, mo, &W);
            lk.lock();
        }
        S->pending.pop_front();
        if (rc) {
            r->rc = rc;
            lk.unlock();
            tm_motif_free(mo);
            lk.lock();
            finish_locked(S, r);
            continue;
        }
        CacheEntry e;
        e.mo = mo;
        e.bytes = mo->bytes;
        e.refs = 1;
        e.last_use = ++S->use_clock;
        S->cache[r->key] = e;
        S->resident += e.bytes;
        S->misses++;
        r->mo = mo;
        S->ready.push_back(r);
        S->cv_sched.notify_all();
    }
}

void sched_loop(Server *S)
{
    tm_ctx *ctx = S->main;
    cudaSetDevice(ctx->device);
    const uint32_t tile = S->cfg.tile;
    std::vector<BatchItem> items;
    std::vector<Request *> owners;
    std::vector<SampleAcc> accs;
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        while (!S->stop && !S->ready.empty() && S->active.size() < S->cfg.max_active) {
            S->active.push_back(S->ready.front());
            S->ready.pop_front();
        }
        if (S->active.empty()) {
            if (S->stop) return;
            S->cv_sched.wait(lk, [&] { return S->stop || !S->ready.empty(); });
            continue;
        }
        // one round: every active query gets its next share of sample ids
        uint64_t round = (uint64_t)S->cfg.round_tiles * tile;
        uint64_t share = std::max<uint64_t>(tile, (round / S->active.size()) / tile * tile);
        items.clear();
        owners.clear();
        for (Request *r : S->active) {
            uint64_t cnt = std::min<uint64_t>(share, r->k - r->next);
            items.push_back(BatchItem{r->mo, r->seed, r->next, cnt});
            owners.push_back(r);
        }
        accs.assign(items.size(), SampleAcc{0, 0, 0, 0, 0, 0});
        lk.unlock();
        int rc = run_batch_items(ctx, items.data(), (uint32_t)items.size(), tile, accs.data(),
                                 S->cfg.poll_timeout_ms);
        // a round that could not get its scratch memory ran nothing: back off
        // and run the same round again (bounded)
        for (int attempt = 0; rc == TM_E_NOMEM && attempt < kNoMemRetries; ++attempt) {
            {
                std::lock_guard<std::mutex> g(S->mu);
                S->round_retries++;
                if (S->stop) break;
            }
            std::this_thread::sleep_for(std::chrono::milliseconds(kNoMemWaitMs));
            accs.assign(items.size(), SampleAcc{0, 0, 0, 0, 0, 0});
            rc = run_batch_items(ctx, items.data(), (uint32_t)items.size(), tile, accs.data(), S->cfg.poll_timeout_ms);
        }
        lk.lock();
        S->rounds++;
        std::vector<Request *> still;
        for (size_t i = 0; i < owners.size(); ++i) {
            Request *r = owners[i];
            if (rc) {
                r->rc = rc;
                finish_locked(S, r);
                continue;
            }
            add_acc(r->acc, accs[i]);
            r->next += items[i].count;
            if (r->next >= r->k) finish_locked(S, r);
            else still.push_back(r);
        }
        S->active.swap(still);
    }
}

}  // namespace
}  // namespace timest

using namespace timest;

extern "C" {

int tm_serve_start(tm_ctx *ctx, const tm_serve_cfg *cfg)
{
    if (!ctx) return TM_E_ARG;
    if (ctx->server) return set_err(ctx, TM_E_STATE, "already serving");
    if (!ctx->preprocessed) return set_err(ctx, TM_E_STATE, "graph not preprocessed");
    cudaSetDevice(ctx->device);
    Server *S = new Server();
    S->main = ctx;
    if (cfg) S->cfg = *cfg;
    if (S->cfg.max_active == 0) S->cfg.max_active = 64;
    if (S->cfg.tile == 0) S->cfg.tile = 4096;
    if (S->cfg.round_tiles == 0) S->cfg.round_tiles = (uint32_t)std::max(64, ctx->num_sms * 2);
    if (S->cfg.poll_timeout_ms <= 0) S->cfg.poll_timeout_ms = 60000;
    if (S->cfg.weight_budget == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        S->cfg.weight_budget = fr / 2;
    }
    // second context on its own stream, sharing the graph (not owning it)
    tm_config c2 = ctx->cfg;
    c2.profile = 0;
    tm_ctx *sh = nullptr;
    int rc = tm_create(&sh, &c2, nullptr);
    if (rc) { delete S; return set_err(ctx, rc, "cannot create the admission context"); }
    sh->g = ctx->g;
    sh->n = ctx->n;
    sh->epoch = ctx->epoch;
    sh->preprocessed = true;
    S->shadow = sh;
    ctx->server = S;
    S->admit_thr = std::thread(admit_loop, S);
    S->sched_thr = std::thread(sched_loop, S);
    return TM_OK;
}

static int queue_request(Server *S, Request *r, uint64_t *ticket)
{
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) { delete r; return TM_E_STATE; }
    r->ticket = S->next_ticket++;
    r->t_submit = Clock::now();
    if (!S->any_submit) { S->any_submit = true; S->t_first_submit = r->t_submit; }
    S->submitted++;
    *ticket = r->ticket;
    // weights already resident: straight to the scheduler, so a hit never
    // waits behind another query's weight pass
    if (admit_cached_locked(S, r)) return TM_OK;
    S->pending.push_back(r);
    S->cv_admit.notify_all();
    return TM_OK;
}

int tm_serve_submit(tm_ctx *ctx, uint32_t nv, uint32_t ne, const uint32_t *edges, const uint32_t *order, int64_t delta,
                    uint64_t k, uint64_t seed, uint64_t *ticket)
{
    if (!ctx || !edges || !order || !ticket) return TM_E_ARG;
    Server *S = ctx->server;
    if (!S) return TM_E_STATE;
    if (nv < 2 || nv > (uint32_t)kMaxV || ne > (uint32_t)kMaxE || ne < nv - 1 || delta <= 0) return TM_E_MOTIF;
    Request *r = new Request();
    r->nv = nv; r->ne = ne;
    r->edges.assign(edges, edges + 2 * ne);
    r->order.assign(order, order + ne);
    r->delta = delta;
    r->k = k;
    r->seed = seed;
    r->key = make_key(nv, ne, edges, order, delta);
    return queue_request(S, r, ticket);
}

int tm_serve_submit_motif(tm_ctx *ctx, const tm_motif *mo, uint64_t k, uint64_t seed, uint64_t *ticket)
{
    if (!ctx || !mo || !ticket) return TM_E_ARG;
    Server *S = ctx->server;
    if (!S) return TM_E_STATE;
    if (mo->ctx != ctx) return TM_E_ARG;
    Request *r = new Request();
    r->nv = mo->nv; r->ne = mo->ne;
    for (uint32_t i = 0; i < mo->ne; ++i) {
        r->edges.push_back(mo->ea[i]);
        r->edges.push_back(mo->eb[i]);
        r->order.push_back(mo->rank[i]);
    }
    r->delta = mo->delta;
    r->pinned = true;
    r->tree.assign(mo->tree, mo->tree + (mo->nv - 1));
    r->root = mo->root;
    r->cflags = (mo->plan.c2 ? TM_C2 : 0) | (mo->plan.wdelta == mo->plan.delta ? TM_C3 : 0);
    r->k = k;
    r->seed = seed;
    // the cache key names the plan: motif, tree, root and constraint flags
    std::string key = make_key(r->nv, r->ne, r->edges.data(), r->order.data(), r->delta) + "|tree:";
    for (uint32_t e : r->tree) key += std::to_string(e) + ",";
    key += "root:" + std::to_string(r->root) + "|c:" + std::to_string(r->cflags);
    r->key = key;
    return queue_request(S, r, ticket);
}

int tm_serve_poll(tm_ctx *ctx, uint64_t ticket, tm_result *out, int timeout_ms)
{
    if (!ctx || !out) return TM_E_ARG;
    Server *S = ctx->server;
    if (!S) return TM_E_STATE;
    std::unique_lock<std::mutex> lk(S->mu);
    if (ticket == 0 || ticket >= S->next_ticket) return TM_E_ARG;
    auto ready = [&] { return S->done.count(ticket) > 0; };
    if (!ready()) {
        if (timeout_ms <= 0 || !S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
            return TM_E_PENDING;
    }
    Request *r = S->done[ticket];
    S->done.erase(ticket);
    int rc = r->rc;
    *out = r->result;
    delete r;
    return rc;
}

int tm_serve_stats(tm_ctx *ctx, tm_serve_stats_t *out)
{
    if (!ctx || !out) return TM_E_ARG;
    Server *S = ctx->server;
    if (!S) return TM_E_STATE;
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->failed = S->failed;
    out->cache_hits = S->hits;
    out->cache_misses = S->misses;
    out->evictions = S->evictions;
    out->rounds = S->rounds;
    out->resident_bytes = S->resident;
    out->waiting = S->pending.size() + S->ready.size();
    out->active = S->active.size();
    out->nomem_retries = S->admit_retries + S->round_retries;
    std::vector<double> l = S->latencies;
    std::sort(l.begin(), l.end());
    if (!l.empty()) {
        auto pct = [&](double p) { return l[std::min(l.size() - 1, (size_t)(p * (l.size() - 1) + 0.5))]; };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double s = 0;
        for (double x : l) s += x;
        out->mean_ms = s / l.size();
        double span = std::chrono::duration<double>(S->t_last_done - S->t_first_submit).count();
        out->qps = span > 0 ? (double)S->completed / span : 0.0;
    }
    return TM_OK;
}

int tm_serve_stop(tm_ctx *ctx)
{
    if (!ctx) return TM_E_ARG;
    Server *S = ctx->server;
    if (!S) return TM_E_STATE;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_admit.notify_all();
        S->cv_sched.notify_all();
    }
    S->admit_thr.join();
    S->sched_thr.join();
    // queries that never finished report TM_E_STATE; their results are freed here
    for (Request *r : S->pending) delete r;
    for (Request *r : S->ready) delete r;
    for (Request *r : S->active) delete r;
    for (auto &d : S->done) delete d.second;
    for (auto &c : S->cache) tm_motif_free(c.second.mo);
    tm_destroy(S->shadow);
    ctx->server = nullptr;
    delete S;
    return TM_OK;
}

}  // extern "C"
