// Sampler, validator and DeriveCnt of TIMEST (Sec. 3.2-3.4; Alg. 3-6).
//
// Sample j draws from its own counter-based stream (Philox4x32-10, key =
// seed, counter = (j, draw number)): a window with probability W_i / W, a
// root edge with probability w_c / W_i (inverse CDF by binary search), then
// each tree edge in breadth-first order from its candidate list L (Claim
// 3.1) with probability proportional to its weight.  L is the meeting
// vertex's out/in-list in a time range minus one multi-edge list; the pick
// is a binary search over positions of the out/in-list whose cumulative
// weight (minus the excluded entries before it, found by a nested search in
// the multi-edge list) first exceeds the draw, so no list is materialised.
// The sample is then validated (Alg. 4) and its completions to the motif
// counted (Alg. 5) by a merge over the non-tree edges' multi-edge lists.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "tm_device.cuh"
#include "tm_internal.h"

namespace timest {

namespace {

typedef SampleAcc Acc;

// Per-thread sample state: rows 0..6 tree-edge sources, 7..13 destinations,
// 14..20 times, 21..27 edge ids, 28..35 the vertex map,
// `stride` apart.  The sampler keeps them in (L1-cached) local memory; a
// shared-memory layout measured slower because it shrinks L1 for the
// searches.
constexpr int kRecRows = 4 * kMaxTree + kMaxV;

struct Recs {
    uint32_t *base;
    int stride;
    __device__ __forceinline__ uint32_t &src(int q) { return base[(0 * kMaxTree + q) * stride]; }
    __device__ __forceinline__ uint32_t &dst(int q) { return base[(1 * kMaxTree + q) * stride]; }
    __device__ __forceinline__ uint32_t &t(int q) { return base[(2 * kMaxTree + q) * stride]; }
    __device__ __forceinline__ uint32_t &gid(int q) { return base[(3 * kMaxTree + q) * stride]; }
    __device__ __forceinline__ uint32_t &phi(int v) { return base[(4 * kMaxTree + v) * stride]; }
};

// The pair id of (u, v) (or kNone): a search of u's pairs, sorted by
// destination; warp-cooperative from coop_min pairs on.
__device__ __forceinline__ uint32_t pair_of_coop(const DevGraph &g, uint32_t u, uint32_t v, uint32_t coop_min)
{
    const uint32_t lo = __ldg(g.vpair_off + u), hi = __ldg(g.vpair_off + u + 1);
    const uint32_t p = first_true_coop(ProbeGeU32{g.pair_dst, v}, lo, hi, coop_min);
    return (p < hi && __ldg(g.pair_dst + p) == v) ? p : kNone;
}

// Multi-edge list range of pair (u, v), or an empty range.
__device__ __forceinline__ void find_pair(const DevGraph &g, uint32_t u, uint32_t v, uint32_t &beg, uint32_t &end,
                                          uint32_t coop_min = 0xFFFFFFFFu)
{
    uint32_t lo = __ldg(g.vpair_off + u), hi = __ldg(g.vpair_off + u + 1);
    uint32_t p = first_true_coop(ProbeGeU32{g.pair_dst, v}, lo, hi, coop_min);
    if (p < hi && __ldg(g.pair_dst + p) == v) {
        beg = __ldg(g.pair_off + p);
        end = __ldg(g.pair_off + p + 1);
    } else {
        beg = end = 0;
    }
}

// DeriveCnt (Alg. 5) when every run of consecutive non-tree pi positions has
// length 1: each non-tree edge only has to lie strictly between its two
// neighbouring tree times (and within [tmax - delta, tmin + delta]), so the
// count is a product of range sizes of multi-edge lists.  When both the
// first and the last pi edge are non-tree their times are coupled by the
// delta span: sum over the first edge's candidates x of the last edge's
// candidates up to x + delta (two pointers over the two sorted lists).
// Rec supplies the vertex map phi(v) and the tree-node times t(q).
template <class Rec>
__device__ uint64_t derive_simple(const DevGraph &g, const DevPlan &P, Rec &R, uint32_t tmin, uint32_t tmax,
                                  bool &ovf, uint32_t coop_min = 0xFFFFFFFFu)
{
    const uint64_t d = (uint64_t)P.delta;
    const uint64_t glo = (uint64_t)tmax >= d ? (uint64_t)tmax - d : 0;
    const uint64_t ghi = (uint64_t)tmin + d;
    uint64_t prod = 1;
    uint32_t ra0 = 0, rb0 = 0, ra1 = 0, rb1 = 0;   // ranges of the coupled first / last edges
    for (int i = 0; i < P.nnt; ++i) {
        const int e = P.pos_edge[P.nt_pos[i]];
        uint32_t b, en;
        find_pair(g, R.phi(P.ea[e]), R.phi(P.eb[e]), b, en, coop_min);
        if (b == en) return 0;
        uint64_t lo = glo, hi = ghi;
        if (P.nt_prev[i] >= 0) { uint64_t x = (uint64_t)R.t(P.nt_prev[i]) + 1; lo = x > lo ? x : lo; }
        if (P.nt_next[i] >= 0) {
            uint32_t nt = R.t(P.nt_next[i]);
            if (nt == 0) return 0;
            hi = (uint64_t)nt - 1 < hi ? (uint64_t)nt - 1 : hi;
        }
        if (lo > hi) return 0;
        const uint32_t x0 = lower_idx(g.multi_t, b, en, lo);
        const uint32_t x1 = lower_idx(g.multi_t, x0, en, hi + 1);
        if (x1 == x0) return 0;
        if (P.coupled && i == 0) {
            ra0 = x0;
            rb0 = x1;
        } else if (P.coupled && i == P.nnt - 1) {
            ra1 = x0;
            rb1 = x1;
        } else {
            prod = mul_chk(prod, (uint64_t)(x1 - x0), ovf);
        }
    }
    if (!P.coupled) return prod;
    uint64_t sum = 0;
    uint32_t j = ra1;
    for (uint32_t x = ra0; x < rb0; ++x) {
        const uint64_t cap = (uint64_t)__ldg(g.multi_t + x) + d;
        while (j < rb1 && (uint64_t)__ldg(g.multi_t + j) <= cap) ++j;
        sum = add_chk(sum, (uint64_t)(j - ra1), ovf);
    }
    return mul_chk(prod, sum, ovf);
}

// DeriveCnt, general case: the lists are merged in time order (ties: later pi
// position first); acc[q] counts the increasing chains over positions 0..q
// that end at an element already passed.
__device__ __noinline__ uint64_t derive_merge(const DevGraph &g, const DevPlan &P, Recs &R, uint32_t tmin_tree, uint32_t tmax_tree,
                                 bool &ovf)
{
    const int ne = P.ne;
    const int64_t d = P.delta;
    uint32_t cur[kMaxE], end[kMaxE], fixed_t[kMaxE];
    bool is_fixed[kMaxE];
    uint64_t glo = (int64_t)tmax_tree >= d ? (uint64_t)((int64_t)tmax_tree - d) : 0;
    uint64_t ghi = (uint64_t)tmin_tree + (uint64_t)d;
    int64_t prev_t = -1;
    for (int pos = 0; pos < ne; ++pos) {
        int e = P.pos_edge[pos];
        int q = P.tnode_of_edge[e];
        if (q >= 0) {
            is_fixed[pos] = true;
            fixed_t[pos] = R.t(q);
            cur[pos] = 0; end[pos] = 1;
            prev_t = R.t(q);
        } else {
            is_fixed[pos] = false;
            uint32_t b, en;
            find_pair(g, R.phi(P.ea[e]), R.phi(P.eb[e]), b, en);
            uint64_t lo = glo;
            if (prev_t >= 0 && (uint64_t)prev_t + 1 > lo) lo = (uint64_t)prev_t + 1;
            cur[pos] = lower_idx(g.multi_t, b, en, lo);
            end[pos] = en;
            fixed_t[pos] = 0;
        }
    }
    int64_t next_t = -1;
    for (int pos = ne - 1; pos >= 0; --pos) {
        if (is_fixed[pos]) { next_t = fixed_t[pos]; continue; }
        if (next_t == 0) return 0;
        uint64_t hi = ghi;
        if (next_t > 0 && (uint64_t)next_t - 1 < hi) hi = (uint64_t)next_t - 1;
        end[pos] = lower_idx(g.multi_t, cur[pos], end[pos], hi + 1);
        if (cur[pos] >= end[pos]) return 0;
    }
    const bool coupled = !is_fixed[0] && !is_fixed[ne - 1];
    uint64_t total = 0;
    const uint32_t first_beg = cur[0], first_end = end[0];
    const uint32_t nfirst = coupled ? first_end - first_beg : 1;
    for (uint32_t f = 0; f < nfirst; ++f) {
        uint32_t c[kMaxE], en[kMaxE];
        uint64_t acc[kMaxE];
        uint64_t cap = ghi;
        for (int pos = 0; pos < ne; ++pos) { c[pos] = cur[pos]; en[pos] = end[pos]; acc[pos] = 0; }
        if (coupled) {
            c[0] = first_beg + f;
            en[0] = c[0] + 1;
            cap = (uint64_t)__ldg(g.multi_t + c[0]) + (uint64_t)d;
        }
        for (;;) {
            int best = -1;
            uint64_t bt = ~0ull;
            for (int pos = 0; pos < ne; ++pos) {
                if (c[pos] >= en[pos]) continue;
                uint64_t tp = is_fixed[pos] ? fixed_t[pos] : __ldg(g.multi_t + c[pos]);
                if (tp <= bt) { bt = tp; best = pos; }
            }
            if (best < 0 || bt > cap) break;
            uint64_t add = best == 0 ? 1 : acc[best - 1];
            acc[best] = add_chk(acc[best], add, ovf);
            c[best]++;
        }
        total = add_chk(total, acc[ne - 1], ovf);
    }
    return total;
}

__device__ __forceinline__ void load_edge(const DevGraph &g, uint32_t gid, Recs &R, int q)
{
    R.gid(q) = gid;
    R.src(q) = __ldg(g.g_src + gid);
    R.dst(q) = __ldg(g.g_dst + gid);
    R.t(q) = __ldg(g.g_t + gid);
}

// Alg. 4: 0 when the sampled tree is valid, else the reject reason (1 the
// vertex map is not 1-1, 2 the tree spans more than delta, 3 tree edges out
// of pi order); fills the vertex map and the tree's time span.
__device__ int validate_tree(const DevPlan &P, Recs R, uint32_t &tmin, uint32_t &tmax)
{
    const uint64_t d = (uint64_t)P.delta;
    tmin = 0xFFFFFFFFu;
    tmax = 0;
    for (int q = 0; q < P.ntree; ++q) {
        const int e = P.tedge[q];
        R.phi(P.ea[e]) = R.src(q);
        R.phi(P.eb[e]) = R.dst(q);
        const uint32_t tq = R.t(q);
        tmin = min(tmin, tq);
        tmax = max(tmax, tq);
    }
    for (int x = 0; x < P.nv; ++x) {
        const uint32_t px = R.phi(x);
        for (int y = x + 1; y < P.nv; ++y)
            if (px == R.phi(y)) return 1;
    }
    if ((uint64_t)tmax - (uint64_t)tmin > d) return 2;
    int64_t prev = -1;
    for (int pos = 0; pos < P.ne; ++pos) {
        const int q = P.tnode_of_edge[P.pos_edge[pos]];
        if (q < 0) continue;
        const int64_t tq = R.t(q);
        if (tq <= prev) return 3;
        prev = tq;
    }
    return 0;
}

// DeriveCnt (Alg. 5): completions of a valid tree to M-matches.
__device__ __forceinline__ uint64_t derive_cnt(const DevGraph &g, const DevPlan &P, Recs R, uint32_t tmin,
                                               uint32_t tmax, bool &ovf)
{
    return P.nnt == 0 ? 1
         : (P.derive_simple ? derive_simple(g, P, R, tmin, tmax, ovf) : derive_merge(g, P, R, tmin, tmax, ovf));
}

// DeriveCnt (Alg. 5) of a valid tree and N_phi (windows holding every tree
// edge): the sample's contribution cnt * 2 / N_phi.
// cnt * 2 / N_phi: N_phi is 2 when the tree's span [tmin, tmax] lies in two
// windows (both layers), else 1; N_phi counts windows of the window unit.
// The window quotients come from the divider of the window unit.
__device__ __forceinline__ uint64_t over_nphi(const WinDiv &wv, uint64_t cnt, uint32_t tmin, uint32_t tmax,
                                              bool &ovf)
{
    const bool two = (uint64_t)tmin >= (uint64_t)wv.d && wv.quot(tmin) == wv.quot(tmax);
    return two ? cnt : mul_chk(cnt, 2, ovf);
}

__device__ uint64_t complete_count(const DevGraph &g, const DevPlan &P, const WinDiv &wv, Recs R, uint32_t tmin,
                                   uint32_t tmax, uint32_t *status)
{
    bool ovf = false;
    const uint64_t cnt = over_nphi(wv, derive_cnt(g, P, R, tmin, tmax, ovf), tmin, tmax, ovf);
    if (ovf) latch(status, ST_OVERFLOW);
    return cnt;
}

// The first draws of sample j (Alg. 3): a window with probability W_i / W,
// then its root edge through the window's guide table and CDF.  Sets the
// layer p, the window's time range [wlo, whi] and the root edge id; 0, or -1
// on an internal inconsistency (latched as ST_BADSTATE).
__device__ __forceinline__ int sample_root(const DevPlan &P, const SampleJob &J, SampleRng &rng, uint32_t *status,
                                           int &p, uint32_t &wlo, uint32_t &whi, uint32_t &root)
{
    const u128 W = (u128)J.W_lo | ((u128)J.W_hi << 64);
    u128 r = rng.below128(W, status);
    // window: last k with wcum[k] <= r, between the guide entries of r's bucket
    const uint32_t jb = (uint32_t)(r >> J.wshift);
    uint32_t lo = __ldg(J.wguide + jb), hi = __ldg(J.wguide + jb + 1) + 1;
    if (lo >= hi || hi > J.nwtot) { latch(status, ST_BADSTATE); return -1; }
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        u128 c = (u128)__ldg(J.wcum + 2 * (size_t)mid) | ((u128)__ldg(J.wcum + 2 * (size_t)mid + 1) << 64);
        if (c <= r) lo = mid; else hi = mid;
    }
    const uint32_t k = lo;
    const u128 ck = (u128)__ldg(J.wcum + 2 * (size_t)k) | ((u128)__ldg(J.wcum + 2 * (size_t)k + 1) << 64);
    const uint64_t rr = (uint64_t)(r - ck);
    p = k < J.nw0 ? 0 : 1;
    const uint32_t kk = p ? k - J.nw0 : k;
    const uint32_t *wb = p ? J.win_beg1 : J.win_beg0;
    const uint64_t *cdf = p ? J.root_cdf1 : J.root_cdf0;
    const uint32_t wbeg = __ldg(wb + kk), wend = __ldg(wb + kk + 1);
    const uint64_t wi = __ldg((p ? J.win_id1 : J.win_id0) + kk);
    const uint64_t wd = (uint64_t)P.wdelta;
    // 32-bit bounds: the window holds the root's time, so wlo fits; whi is
    // clamped to the largest t' (no time lies beyond it)
    wlo = (uint32_t)(wi * wd);
    const uint64_t whi64 = (wi + 2) * wd - 1;
    whi = whi64 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)whi64;
    // the root edge lies between two guide entries: the first edges whose CDF
    // exceeds the bucket bounds below and above rr
    const uint32_t gsh = __ldg((p ? J.win_gshift1 : J.win_gshift0) + kk);
    const uint32_t *G = (p ? J.guide1 : J.guide0) + __ldg((p ? J.win_goff1 : J.win_goff0) + kk) + (rr >> gsh);
    const uint32_t glo = __ldg(G), ghi = __ldg(G + 1);
    if (glo < wbeg || ghi >= wend || glo > ghi) { latch(status, ST_BADSTATE); return -1; }
    root = upper_idx64(cdf, glo, ghi + 1, rr);
    if (root > ghi) { latch(status, ST_BADSTATE); return -1; }
    return 0;
}

// One tree edge of Alg. 3: the edge of tree node q, drawn by weight from its
// candidate list at the meeting vertex given its parent's edge (source ps,
// destination pd, time pt, edge id pgid), in layer p whose
// window spans [wlo, whi].  Sets the child's time, endpoints and, for a node
// with children or when `ids` is set, its edge id; 0, or -1 on an
// internal inconsistency (latched as ST_BADSTATE).
__device__ __forceinline__ int sample_child(const DevGraph &g, const DevPlan &P, const SampleJob &J, int q, int p,
                                            uint32_t wlo, uint32_t whi, SampleRng &rng, uint32_t *status,
                                            uint32_t ps, uint32_t pd, uint32_t pt, uint32_t pgid,
                                            bool ids, uint32_t &ct, uint32_t &cs, uint32_t &cd, uint32_t &cgid)
{
    const uint64_t d = (uint64_t)P.delta;
    const bool zs = P.tzside[q] != 0, out = P.tout[q] != 0, leaf = P.tleaf[q] != 0;
    const uint32_t zg = zs ? pd : ps;
    const uint32_t og = zs ? ps : pd;
    uint64_t tlo, thi;
    if (P.tlater[q]) { tlo = (uint64_t)pt + 1; thi = (uint64_t)pt + d; }
    else {
        if (pt == 0) { latch(status, ST_BADSTATE); return -1; }
        tlo = (uint64_t)pt >= d ? (uint64_t)pt - d : 0;
        thi = (uint64_t)pt - 1;
    }
    tlo = tlo < (uint64_t)wlo ? (uint64_t)wlo : tlo;
    thi = thi > (uint64_t)whi ? (uint64_t)whi : thi;
    const uint32_t *nbr = out ? g.out_nbr : g.in_nbr;
    const uint32_t *gids = out ? g.out_gid : g.in_gid;
    // the parent edge's position in the meeting vertex's out-list (z is its
    // source) or in-list (z is its destination)
    const uint32_t ppos = __ldg((zs ? g.in_pos : g.out_pos) + pgid);
    uint32_t a, b, beg;
    const uint32_t *tarr;
    child_range(g, zs ? 1 : 0, out, zg, ppos, pt, P.tlater[q] != 0, tlo, thi, a, b, beg, tarr);
    // the excluded multi-edge list (Constraint 2): zg -> og for a child
    // leaving the meeting vertex, og -> zg for one entering it (scanning a
    // short range for such entries first measured slower than this lookup)
    const uint32_t pe = !P.c2 ? kNone
                      : out ? pair_of_coop(g, zg, og, J.coop_min) : pair_of_coop(g, og, zg, J.coop_min);
    uint32_t ea = 0, eb = 0, pb = 0;
    if (pe != kNone) {
        pb = __ldg(g.pair_off + pe);
        const uint32_t pend = __ldg(g.pair_off + pe + 1);
        ea = lower_idx(g.multi_t, pb, pend, tlo);
        eb = gallop_idx(g.multi_t, ea, pend, thi + 1);
    }
    const int slot = P.tslot[q];
    const uint64_t *Pd = nullptr, *Pm = nullptr;
    uint64_t base = 0, base_m = 0, total;
    if (leaf) {
        total = (uint64_t)(b - a) - (uint64_t)(eb - ea);
    } else {
        // layer p's lane of the slot's (layer 0, layer 1) prefix pairs
        Pd = (const uint64_t *)J.pref_dir[slot] + p;
        Pm = (const uint64_t *)J.pref_multi[slot] + p;
        base = (a > beg && __ldg(tarr + a - 1) >= wlo) ? __ldg(Pd + 2 * (size_t)(a - 1)) : 0;
        base_m = (ea > pb && __ldg(g.multi_t + ea - 1) >= wlo) ? __ldg(Pm + 2 * (size_t)(ea - 1)) : 0;
        const uint64_t sr = b > a ? __ldg(Pd + 2 * (size_t)(b - 1)) - base : 0;
        const uint64_t se = eb > ea ? __ldg(Pm + 2 * (size_t)(eb - 1)) - base_m : 0;
        total = sr - se;
    }
    if (total == 0 || b <= a) { latch(status, ST_BADSTATE); return -1; }
    const uint64_t rc = rng.below(total, status);
    // smallest x in [a, b) with F(x) > rc, F(x) = weight of the
    // non-excluded entries in [a, x]
    uint32_t xl = a, xh = b - 1;
    if (eb == ea) {
        // nothing excluded: F(x) = x - a + 1 for a leaf (the pick is
        // direct), the prefix difference otherwise
        if (leaf) xl = a + (uint32_t)rc;
        else xl = first_true_coop(ProbeGtU64S2{Pd, rc + base}, a, b, J.coop_min);
    } else {
        while (xl < xh) {
            const uint32_t x = xl + ((xh - xl) >> 1);
            const uint32_t tx = __ldg(tarr + x);
            // excluded entries at or before x: those earlier in time, and
            // the one at time tx if it sorts at or before x (the list
            // orders equal times by the other endpoint)
            uint32_t ce = lower_idx(g.multi_t, ea, eb, tx) - ea;
            if (ea + ce < eb && __ldg(g.multi_t + ea + ce) == tx && og <= __ldg(nbr + x)) ++ce;
            uint64_t F;
            if (leaf) F = (uint64_t)(x - a + 1) - ce;
            else F = (__ldg(Pd + 2 * (size_t)x) - base) - (ce ? __ldg(Pm + 2 * (size_t)(ea + ce - 1)) - base_m : 0);
            if (F > rc) xh = x; else xl = x + 1;
        }
    }
    const uint32_t other = __ldg(nbr + xl);
    ct = __ldg(tarr + xl);
    cs = out ? zg : other;
    cd = out ? other : zg;
    // the edge id is read only for a node with children (or a trace)
    if (!leaf || ids) cgid = __ldg(gids + xl);
    return 0;
}

// The tree of sample j (Alg. 3): the root, then every tree edge from its
// candidate list.  Fills R; 0, or -1 on an internal inconsistency (latched
// as ST_BADSTATE).
__device__ int sample_tree(const DevGraph &g, const DevPlan &P, const SampleJob &J, uint64_t seed, uint64_t j,
                           uint32_t *status, uint32_t *tg_out, Recs R)
{
    SampleRng rng;
    rng.init(seed, j);
    int p;
    uint32_t wlo, whi;
    uint32_t root;
    if (sample_root(P, J, rng, status, p, wlo, whi, root)) return -1;
    load_edge(g, root, R, 0);
    for (int q = 1; q < P.ntree; ++q) {
        const int pq = P.tparent[q];
        if (sample_child(g, P, J, q, p, wlo, whi, rng, status, R.src(pq), R.dst(pq), R.t(pq), R.gid(pq),
                         tg_out != nullptr, R.t(q), R.src(q), R.dst(q), R.gid(q)))
            return -1;
    }
    if (tg_out)
        for (int q = 0; q < P.ntree; ++q) tg_out[q] = R.gid(q);
    return 0;
}

// One sample: returns 0 valid, 1/2/3 reject reasons, or -1 on an internal
// inconsistency (latched as ST_BADSTATE).
__device__ int sample_one(const DevGraph &g, const DevPlan &P, const SampleJob &J, uint64_t seed, uint64_t j,
                          uint32_t *status, uint64_t &contrib, uint32_t *tg_out, Recs R)
{
    contrib = 0;
    const int r = sample_tree(g, P, J, seed, j, status, tg_out, R);
    if (r) return r;
    uint32_t tmin, tmax;
    const int why = validate_tree(P, R, tmin, tmax);
    if (why) return why;
    contrib = complete_count(g, P, J.wv, R, tmin, tmax, status);
    return 0;
}

// ---- records in registers ------------------------------------------------
// A tree of NT nodes (NT = nv - 1, known at compile time) keeps a sample's
// edges and vertex map in registers: every loop over tree nodes and motif
// vertices is unrolled, and a runtime index reads through a chain of selects.
// Same draws, same arithmetic and same results as sample_one.

template <int N>
__device__ __forceinline__ uint32_t rsel(const uint32_t (&a)[N], int i)
{
    uint32_t v = a[0];
#pragma unroll
    for (int s = 1; s < N; ++s) v = (i == s) ? a[s] : v;
    return v;
}

template <int NT>
struct RegView {
    const uint32_t (&tt)[NT];
    const uint32_t (&ph)[NT + 1];
    __device__ __forceinline__ uint32_t t(int q) const { return rsel(tt, q); }
    __device__ __forceinline__ uint32_t phi(int v) const { return rsel(ph, v); }
};

template <int NT>
__device__ __forceinline__ int sample_one_reg(const DevGraph &g, const DevPlan &P, const SampleJob &J, uint64_t seed,
                                              uint64_t j, uint32_t *status, uint64_t &contrib)
{
    contrib = 0;
    SampleRng rng;
    rng.init(seed, j);
    int p;
    uint32_t wlo, whi;
    uint32_t root;
    if (sample_root(P, J, rng, status, p, wlo, whi, root)) return -1;
    // Alg. 3: the root edge, then each node from its parent (parents come first)
    uint32_t src[NT], dst[NT], t[NT], gid[NT];
    gid[0] = root;
    src[0] = __ldg(g.g_src + root);
    dst[0] = __ldg(g.g_dst + root);
    t[0] = __ldg(g.g_t + root);
#pragma unroll
    for (int q = 1; q < NT; ++q) {
        const int pq = P.tparent[q];
        uint32_t ps = src[0], pd = dst[0], pt = t[0], pg = gid[0];
#pragma unroll
        for (int h = 1; h < q; ++h)
            if (pq == h) { ps = src[h]; pd = dst[h]; pt = t[h]; pg = gid[h]; }
        gid[q] = 0;
        if (sample_child(g, P, J, q, p, wlo, whi, rng, status, ps, pd, pt, pg, false, t[q], src[q], dst[q], gid[q]))
            return -1;
    }
    // Alg. 4: the vertex map (1-1), the delta span, the pi order of tree edges
    uint32_t phi[NT + 1];
#pragma unroll
    for (int x = 0; x <= NT; ++x) phi[x] = 0;
    uint32_t tmin = 0xFFFFFFFFu, tmax = 0;
#pragma unroll
    for (int q = 0; q < NT; ++q) {
        const int e = P.tedge[q];
        const int va = P.ea[e], vb = P.eb[e];
#pragma unroll
        for (int x = 0; x <= NT; ++x) {
            if (x == va) phi[x] = src[q];
            if (x == vb) phi[x] = dst[q];
        }
        tmin = min(tmin, t[q]);
        tmax = max(tmax, t[q]);
    }
#pragma unroll
    for (int x = 0; x <= NT; ++x)
#pragma unroll
        for (int y = x + 1; y <= NT; ++y)
            if (phi[x] == phi[y]) return 1;
    if ((uint64_t)tmax - (uint64_t)tmin > (uint64_t)P.delta) return 2;
    int64_t prev = -1;
    for (int pos = 0; pos < P.ne; ++pos) {
        const int q = P.tnode_of_edge[P.pos_edge[pos]];
        if (q < 0) continue;
        const int64_t tq = rsel(t, q);
        if (tq <= prev) return 3;
        prev = tq;
    }
    // Alg. 5 (plans whose non-tree runs all have length 1) and N_phi
    bool ovf = false;
    uint64_t cnt = 1;
    if (P.nnt > 0) {
        RegView<NT> v{t, phi};
        cnt = derive_simple(g, P, v, tmin, tmax, ovf, J.coop_min);
    }
    cnt = over_nphi(J.wv, cnt, tmin, tmax, ovf);
    if (ovf) latch(status, ST_OVERFLOW);
    contrib = cnt;
    return 0;
}

// Warp sums of a thread's tallies, then one set of atomics per warp.
__device__ __forceinline__ void add_tallies(Acc *acc, u128 hits, unsigned long long nv, unsigned long long nr1,
                                            unsigned long long nr2, unsigned long long nr3)
{
    uint64_t hl = (uint64_t)hits, hh = (uint64_t)(hits >> 64);
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t ol = __shfl_down_sync(0xffffffffu, hl, o);
        uint64_t oh = __shfl_down_sync(0xffffffffu, hh, o);
        uint64_t s = hl + ol;
        hh += oh + (s < hl ? 1 : 0);
        hl = s;
        nv += __shfl_down_sync(0xffffffffu, nv, o);
        nr1 += __shfl_down_sync(0xffffffffu, nr1, o);
        nr2 += __shfl_down_sync(0xffffffffu, nr2, o);
        nr3 += __shfl_down_sync(0xffffffffu, nr3, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (hl) {
            unsigned long long old = atomicAdd(&acc->hits_lo, (unsigned long long)hl);
            if (old + hl < old) hh += 1;
        }
        if (hh) atomicAdd(&acc->hits_hi, (unsigned long long)hh);
        if (nv) atomicAdd(&acc->valid, nv);
        if (nr1) atomicAdd(&acc->rv, nr1);
        if (nr2) atomicAdd(&acc->rd, nr2);
        if (nr3) atomicAdd(&acc->ro, nr3);
    }
}

#ifndef TM_SAMPLE_THREADS
#define TM_SAMPLE_THREADS 256
#endif
constexpr int kSampleThreads = TM_SAMPLE_THREADS;
#ifndef TM_SAMPLE_MINB
#define TM_SAMPLE_MINB 4   // 64 registers, four blocks of 256 per SM (measured faster than 48 or 40 registers)
#endif
#ifndef TM_SAMPLE_GRID_PER_SM
// tm_sample's grid cap in blocks per SM: one wave of resident blocks, each
// thread striding over samples (measured faster than 2-8 partial waves)
#define TM_SAMPLE_GRID_PER_SM TM_SAMPLE_MINB
#endif
#ifndef TM_RECS_SMEM
#define TM_RECS_SMEM 0   // per-sample records in local memory: L1 stays large for the searches
#endif

template <bool TRACE>
__global__ void __launch_bounds__(kSampleThreads, TM_SAMPLE_MINB) k_sample(DevGraph g, const DevPlan *__restrict__ plan,
                                                              SampleJob J, uint64_t seed, uint64_t first, uint64_t k,
                                                              Acc *acc, uint32_t *status, uint32_t *tr_gid,
                                                              uint64_t *tr_contrib, int32_t *tr_reason)
{
    __shared__ DevPlan sp;
#if TM_RECS_SMEM
    __shared__ uint32_t recs[kRecRows * kSampleThreads];
#endif
    {
        const int *src = reinterpret_cast<const int *>(plan);
        int *dst = reinterpret_cast<int *>(&sp);
        for (int i = threadIdx.x; i < (int)(sizeof(DevPlan) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
#if TM_RECS_SMEM
    Recs R{recs + threadIdx.x, kSampleThreads};
#else
    uint32_t recs_local[kRecRows];
    Recs R{recs_local, 1};
#endif
    u128 hits = 0;
    unsigned long long nv = 0, nr1 = 0, nr2 = 0, nr3 = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
        uint64_t c = 0;
        int why = sample_one(g, sp, J, seed, first + i, status, c, TRACE ? tr_gid + i * sp.ntree : nullptr, R);
        if (why == 0) { ++nv; hits += c; }
        else if (why == 1) ++nr1;
        else if (why == 2) ++nr2;
        else if (why == 3) ++nr3;
        if (TRACE) { tr_contrib[i] = c; tr_reason[i] = why; }
    }
    add_tallies(acc, hits, nv, nr1, nr2, nr3);
}

// k_sample without a trace for a tree of NT nodes, records in registers.
template <int NT>
__global__ void __launch_bounds__(kSampleThreads, TM_SAMPLE_MINB) k_sample_reg(DevGraph g, const DevPlan *__restrict__ plan,
                                                              SampleJob J, uint64_t seed, uint64_t first, uint64_t k,
                                                              Acc *acc, uint32_t *status)
{
    __shared__ DevPlan sp;
    {
        const int *src = reinterpret_cast<const int *>(plan);
        int *dst = reinterpret_cast<int *>(&sp);
        for (int i = threadIdx.x; i < (int)(sizeof(DevPlan) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    u128 hits = 0;
    // per-thread tallies fit 32 bits: the launcher keeps k / (grid threads) below 2^32
    uint32_t nv = 0, nr1 = 0, nr2 = 0, nr3 = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
        uint64_t c = 0;
        int why = sample_one_reg<NT>(g, sp, J, seed, first + i, status, c);
        if (why == 0) { ++nv; hits += c; }
        else if (why == 1) ++nr1;
        else if (why == 2) ++nr2;
        else if (why == 3) ++nr3;
    }
    add_tallies(acc, hits, nv, nr1, nr2, nr3);
}

// ---- motif listing (Alg. 5 emitting the instances it counts) -------------
// The completions of a valid tree, depth first over the non-tree edges in pi
// order, each multi-edge list in time order.  Level i takes an entry of
// El(phi(a_i), phi(b_i)) later than the pi position before it and earlier than
// the next tree edge, inside [tmax - delta, tmin + delta]; a full assignment
// is an instance when its pi span (last time - first time) is at most delta.
// emit(index, cur) receives each instance (cur[i] = multi-edge position of
// level i) in that order; returns the number of instances.
template <class Emit>
__device__ uint64_t enumerate_completions(const DevGraph &g, const DevPlan &P, Recs R, uint32_t tmin, uint32_t tmax,
                                          Emit emit)
{
    const int nn = P.nnt;
    if (nn == 0) { emit(0ull, (const uint32_t *)nullptr); return 1; }
    const uint64_t d = (uint64_t)P.delta;
    const uint64_t glo = (uint64_t)tmax >= d ? (uint64_t)tmax - d : 0, ghi = (uint64_t)tmin + d;
    uint32_t lb[kMaxE], le[kMaxE], cur[kMaxE], end[kMaxE];
    for (int i = 0; i < nn; ++i) {
        const int e = P.pos_edge[P.nt_pos[i]];
        find_pair(g, R.phi(P.ea[e]), R.phi(P.eb[e]), lb[i], le[i]);
        if (lb[i] == le[i]) return 0;
    }
    // time at pi position pos given the current choices of levels < i
    auto time_at = [&](int pos, int i) -> uint64_t {
        const int q = P.tnode_of_edge[P.pos_edge[pos]];
        if (q >= 0) return R.t(q);
        for (int l = 0; l < i; ++l) if (P.nt_pos[l] == pos) return __ldg(g.multi_t + cur[l]);
        return 0;   // not reached: callers ask for tree positions or earlier levels
    };
    auto open_level = [&](int i) {
        const int pos = P.nt_pos[i];
        uint64_t lo = glo, hi = ghi;
        if (pos > 0) { const uint64_t tp = time_at(pos - 1, i) + 1; lo = tp > lo ? tp : lo; }
        if (P.nt_next[i] >= 0) {
            const uint64_t tn = R.t(P.nt_next[i]);
            hi = tn == 0 ? 0 : (tn - 1 < hi ? tn - 1 : hi);
            if (tn == 0) lo = hi + 1;
        }
        if (lo > hi) { cur[i] = end[i] = lb[i]; return; }
        cur[i] = lower_idx(g.multi_t, lb[i], le[i], lo);
        end[i] = lower_idx(g.multi_t, cur[i], le[i], hi + 1);
    };
    uint64_t count = 0;
    int i = 0;
    open_level(0);
    for (;;) {
        if (cur[i] >= end[i]) {
            if (--i < 0) break;
            ++cur[i];
            continue;
        }
        if (i < nn - 1) {
            open_level(++i);
            continue;
        }
        const uint64_t first_t = time_at(0, nn), last_t = time_at(P.ne - 1, nn);
        if (last_t - first_t <= d) emit(count++, (const uint32_t *)cur);
        ++cur[i];
    }
    return count;
}

// Pass 1 of listing: completions per sample (0 when rejected).
__global__ void __launch_bounds__(kSampleThreads, TM_SAMPLE_MINB)
    k_list_count(DevGraph g, const DevPlan *__restrict__ plan, SampleJob J, uint64_t seed, uint64_t first, uint64_t k,
                 uint64_t *__restrict__ cnt_out, uint32_t *status)
{
    __shared__ DevPlan sp;
    {
        const int *src = reinterpret_cast<const int *>(plan);
        int *dst = reinterpret_cast<int *>(&sp);
        for (int i = threadIdx.x; i < (int)(sizeof(DevPlan) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    uint32_t recs_local[kRecRows];
    Recs R{recs_local, 1};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
        uint64_t c = 0;
        if (sample_tree(g, sp, J, seed, first + i, status, nullptr, R) == 0) {
            uint32_t tmin, tmax;
            if (validate_tree(sp, R, tmin, tmax) == 0) {
                bool ovf = false;
                c = derive_cnt(g, sp, R, tmin, tmax, ovf);
                if (ovf) latch(status, ST_OVERFLOW);
            }
        }
        cnt_out[i] = c;
    }
}

// Pass 2: each sample's instances at rows offs[i] .. offs[i+1]-1 (rows at or
// beyond max_inst are not written): ne edge ids per row, motif edge e in
// column e, and the sample id.
__global__ void __launch_bounds__(kSampleThreads, TM_SAMPLE_MINB)
    k_list_emit(DevGraph g, const DevPlan *__restrict__ plan, SampleJob J, uint64_t seed, uint64_t first, uint64_t k,
                const uint64_t *__restrict__ offs, uint64_t max_inst, uint32_t *__restrict__ inst_gids,
                uint64_t *__restrict__ inst_sample, uint32_t *status)
{
    __shared__ DevPlan sp;
    {
        const int *src = reinterpret_cast<const int *>(plan);
        int *dst = reinterpret_cast<int *>(&sp);
        for (int i = threadIdx.x; i < (int)(sizeof(DevPlan) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    uint32_t recs_local[kRecRows];
    Recs R{recs_local, 1};
    uint32_t tree_gids[kMaxTree];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
        const uint64_t o = offs[i], n = offs[i + 1] - o;
        if (n == 0 || o >= max_inst) continue;
        if (sample_tree(g, sp, J, seed, first + i, status, tree_gids, R)) continue;
        uint32_t tmin, tmax;
        if (validate_tree(sp, R, tmin, tmax)) { latch(status, ST_BADSTATE); continue; }
        const uint64_t got = enumerate_completions(g, sp, R, tmin, tmax, [&](uint64_t idx, const uint32_t *cur) {
            const uint64_t r = o + idx;
            if (r >= max_inst) return;
            uint32_t *row = inst_gids + r * (uint64_t)sp.ne;
            for (int q = 0; q < sp.ntree; ++q) row[sp.tedge[q]] = tree_gids[q];
            for (int l = 0; l < sp.nnt; ++l)
                row[sp.pos_edge[sp.nt_pos[l]]] = __ldg(g.out_gid + __ldg(g.multi_to_out + cur[l]));
            inst_sample[r] = first + i;
        });
        if (got != n) latch(status, ST_BADSTATE);   // the enumeration must agree with DeriveCnt
    }
}

// ---- several motifs per sampling run ------------------------------------
// Motifs whose spanning trees are the same temporal pattern share one weight
// pass and one stream of sampled trees: each sample is drawn and validated
// once with the first plan and completed (Alg. 5) once per motif.
template <int NM>
__global__ void __launch_bounds__(kSampleThreads, TM_SAMPLE_MINB)
    k_sample_group(DevGraph g, const DevPlan *__restrict__ plans, SampleJob J, uint64_t seed, uint64_t first,
                   uint64_t k, Acc *acc, uint32_t *status)
{
    __shared__ DevPlan sp[NM];
    {
        const int *src = reinterpret_cast<const int *>(plans);
        int *dst = reinterpret_cast<int *>(sp);
        for (int i = threadIdx.x; i < (int)(NM * sizeof(DevPlan) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    uint32_t recs_local[kRecRows];
    Recs R{recs_local, 1};
    u128 hits[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) hits[m] = 0;
    unsigned long long nv = 0, nr1 = 0, nr2 = 0, nr3 = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
        if (sample_tree(g, sp[0], J, seed, first + i, status, nullptr, R)) continue;
        uint32_t tmin, tmax;
        const int why = validate_tree(sp[0], R, tmin, tmax);
        if (why == 1) { ++nr1; continue; }
        if (why == 2) { ++nr2; continue; }
        if (why == 3) { ++nr3; continue; }
        ++nv;
#pragma unroll
        for (int m = 0; m < NM; ++m) hits[m] += complete_count(g, sp[m], J.wv, R, tmin, tmax, status);
    }
    for (int o = 16; o > 0; o >>= 1) {
        nv += __shfl_down_sync(0xffffffffu, nv, o);
        nr1 += __shfl_down_sync(0xffffffffu, nr1, o);
        nr2 += __shfl_down_sync(0xffffffffu, nr2, o);
        nr3 += __shfl_down_sync(0xffffffffu, nr3, o);
    }
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        uint64_t hl = (uint64_t)hits[m], hh = (uint64_t)(hits[m] >> 64);
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t ol = __shfl_down_sync(0xffffffffu, hl, o);
            const uint64_t oh = __shfl_down_sync(0xffffffffu, hh, o);
            const uint64_t sum = hl + ol;
            hh += oh + (sum < hl ? 1 : 0);
            hl = sum;
        }
        if ((threadIdx.x & 31) == 0) {
            if (hl) {
                const unsigned long long old = atomicAdd(&acc[m].hits_lo, (unsigned long long)hl);
                if (old + hl < old) hh += 1;
            }
            if (hh) atomicAdd(&acc[m].hits_hi, (unsigned long long)hh);
        }
    }
    if ((threadIdx.x & 31) == 0) {   // validity is shared: counted on the first accumulator
        if (nv) atomicAdd(&acc[0].valid, nv);
        if (nr1) atomicAdd(&acc[0].rv, nr1);
        if (nr2) atomicAdd(&acc[0].rd, nr2);
        if (nr3) atomicAdd(&acc[0].ro, nr3);
    }
}

// ---- batched sampling (many queries, one persistent launch) ----
// Work item i is a tile of `tile` consecutive sample ids of one query; query
// q owns items [tile_base[q], tile_base[q+1]).  Blocks take items from a
// device counter until none is left, so queries with very different k share
// the GPU; each sample still draws from its own stream, so every query's
// result equals a separate tm_sample call.
struct BatchQuery {
    DevPlan plan;
    SampleJob job;
    uint64_t seed, first, k;   // sample ids first .. first+k-1
};

template <int THREADS, int SMEM_RECS>
__global__ void __launch_bounds__(THREADS, 1536 / THREADS) k_batch(DevGraph g, const BatchQuery *__restrict__ qs,
                                                  const uint32_t *__restrict__ tile_base, uint32_t nq, uint32_t tile,
                                                  uint32_t *counter, Acc *accs, uint32_t *status)
{
    __shared__ BatchQuery sq;
    __shared__ uint32_t s_item;
    __shared__ int s_q;
    __shared__ unsigned long long red[THREADS / 32][6];
    // per-sample records: shared memory (one column per thread) or local
    // memory; which is faster depends on how much L1 the searches need
    __shared__ uint32_t recs_s[SMEM_RECS ? kRecRows * THREADS : 1];
    uint32_t recs_l[SMEM_RECS ? 1 : kRecRows];
    Recs R = SMEM_RECS ? Recs{recs_s + threadIdx.x, THREADS} : Recs{recs_l, 1};
    const uint32_t total = __ldg(tile_base + nq);
    int cur_q = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            uint32_t item = atomicAdd(counter, 1u);
            s_item = item;
            int q = -1;
            if (item < total) {
                uint32_t lo = 0, hi = nq;          // last q with tile_base[q] <= item
                while (hi - lo > 1) {
                    uint32_t mid = (lo + hi) >> 1;
                    if (__ldg(tile_base + mid) <= item) lo = mid; else hi = mid;
                }
                q = (int)lo;
            }
            s_q = q;
        }
        __syncthreads();
        const uint32_t item = s_item;
        const int q = s_q;
        if (item >= total) break;
        if (q != cur_q) {
            const int *src = reinterpret_cast<const int *>(qs + q);
            int *dst = reinterpret_cast<int *>(&sq);
            for (int i = threadIdx.x; i < (int)(sizeof(BatchQuery) / sizeof(int)); i += THREADS) dst[i] = src[i];
            cur_q = q;
            __syncthreads();
        }
        const uint64_t t0 = (uint64_t)(item - __ldg(tile_base + q)) * tile;
        const uint64_t t1 = min(t0 + tile, sq.k);
        u128 hits = 0;
        unsigned long long nv = 0, n1 = 0, n2 = 0, n3 = 0;
        for (uint64_t i = t0 + threadIdx.x; i < t1; i += THREADS) {
            uint64_t c = 0;
            int why = sample_one(g, sq.plan, sq.job, sq.seed, sq.first + i, status, c, nullptr, R);
            if (why == 0) { ++nv; hits += c; }
            else if (why == 1) ++n1;
            else if (why == 2) ++n2;
            else if (why == 3) ++n3;
        }
        uint64_t hl = (uint64_t)hits, hh = (uint64_t)(hits >> 64);
        for (int o = 16; o > 0; o >>= 1) {
            uint64_t ol = __shfl_down_sync(0xffffffffu, hl, o), oh = __shfl_down_sync(0xffffffffu, hh, o);
            uint64_t sum = hl + ol;
            hh += oh + (sum < hl ? 1 : 0);
            hl = sum;
            nv += __shfl_down_sync(0xffffffffu, nv, o);
            n1 += __shfl_down_sync(0xffffffffu, n1, o);
            n2 += __shfl_down_sync(0xffffffffu, n2, o);
            n3 += __shfl_down_sync(0xffffffffu, n3, o);
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) {
            red[warp][0] = hl; red[warp][1] = hh; red[warp][2] = nv;
            red[warp][3] = n1; red[warp][4] = n2; red[warp][5] = n3;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t L = 0, H = 0, a = 0, b = 0, c = 0, d = 0;
            for (int w = 0; w < THREADS / 32; ++w) {
                uint64_t sum = L + red[w][0];
                H += red[w][1] + (sum < L ? 1 : 0);
                L = sum;
                a += red[w][2]; b += red[w][3]; c += red[w][4]; d += red[w][5];
            }
            Acc *A = accs + q;
            if (L) {
                unsigned long long old = atomicAdd(&A->hits_lo, (unsigned long long)L);
                if (old + L < old) H += 1;
            }
            if (H) atomicAdd(&A->hits_hi, (unsigned long long)H);
            if (a) atomicAdd(&A->valid, (unsigned long long)a);
            if (b) atomicAdd(&A->rv, (unsigned long long)b);
            if (c) atomicAdd(&A->rd, (unsigned long long)c);
            if (d) atomicAdd(&A->ro, (unsigned long long)d);
        }
        __syncthreads();
    }
}

}  // namespace

void fill_job(tm_motif *mo, SampleJob &J, const DevPlan *dplan)
{
    J.plan = dplan;
    J.wcum = mo->wcum;
    J.wguide = mo->wguide;
    J.wshift = wguide_shift(mo->W.lo, mo->W.hi, mo->nwtot);
    J.wv = make_windiv(mo->plan.wdelta);
    J.coop_min = mo->ctx ? mo->ctx->coop_min : 0xFFFFFFFFu;
    J.nwtot = mo->nwtot;
    J.nw0 = mo->layer[0].nwin;
    J.win_beg0 = mo->layer[0].win_beg; J.win_beg1 = mo->layer[1].win_beg;
    J.win_id0 = mo->layer[0].win_id; J.win_id1 = mo->layer[1].win_id;
    J.root_cdf0 = mo->layer[0].root_cdf; J.root_cdf1 = mo->layer[1].root_cdf;
    J.win_gshift0 = mo->layer[0].win_gshift; J.win_gshift1 = mo->layer[1].win_gshift;
    J.win_goff0 = mo->layer[0].win_goff; J.win_goff1 = mo->layer[1].win_goff;
    J.guide0 = mo->layer[0].guide; J.guide1 = mo->layer[1].guide;
    for (int s = 0; s < kMaxTree; ++s) {
        J.pref_dir[s] = mo->pref_dir[s];
        J.pref_multi[s] = mo->pref_multi[s];
    }
    J.W_lo = mo->W.lo;
    J.W_hi = mo->W.hi;
}

static void finish_result(tm_motif *mo, uint64_t k, const Acc &a, tm_result *out)
{
    out->W = mo->W;
    out->hits2.lo = a.hits_lo;
    out->hits2.hi = a.hits_hi;
    out->k = k;
    out->valid = a.valid;
    out->rej_vertex = a.rv;
    out->rej_delta = a.rd;
    out->rej_order = a.ro;
    double W = (double)mo->W.lo + 18446744073709551616.0 * (double)mo->W.hi;
    double h = (double)a.hits_lo + 18446744073709551616.0 * (double)a.hits_hi;
    out->estimate = k ? W * h / (2.0 * (double)k) : 0.0;
}

// The register-record sampler for this plan's tree size; false when the plan
// is not a spanning tree of nv - 1 nodes or needs the general DeriveCnt (the
// caller launches k_sample).
static bool launch_sample_reg(tm_ctx *ctx, const DevPlan &P, unsigned blocks, int threads, const DevPlan *dplan,
                              const SampleJob &J, uint64_t seed, uint64_t first, uint64_t k, Acc *dacc)
{
    if (P.nv != P.ntree + 1 || (P.nnt > 0 && !P.derive_simple)) return false;
    switch (P.ntree) {
#define TM_REG_CASE(N) \
    case N: launch(ctx, k_sample_reg<N>, blocks, threads, ctx->g, dplan, J, seed, first, k, dacc, ctx->status); return true;
        TM_REG_CASE(1) TM_REG_CASE(2) TM_REG_CASE(3) TM_REG_CASE(4) TM_REG_CASE(5) TM_REG_CASE(6) TM_REG_CASE(7)
#undef TM_REG_CASE
    default: return false;
    }
}

int run_samples(tm_ctx *ctx, tm_motif *mo, uint64_t k, uint64_t seed, uint64_t first, tm_result *out,
                uint32_t *trace_gids, uint64_t *trace_contrib, int32_t *trace_reason)
{
    ScratchScope scope(ctx);
    cudaStream_t st = ctx->stream;
    Acc zero{0, 0, 0, 0, 0, 0};
    if (k == 0 || (mo->W.lo == 0 && mo->W.hi == 0)) {
        finish_result(mo, k, zero, out);
        return TM_OK;
    }
    const bool trace = trace_gids || trace_contrib || trace_reason;
    size_t plan_bytes = sizeof(DevPlan), acc_bytes = sizeof(Acc);
    char *scratch = (char *)salloc(ctx, plan_bytes + acc_bytes + 64);
    if (!scratch) return TM_E_NOMEM;
    DevPlan *dplan = (DevPlan *)scratch;
    Acc *dacc = (Acc *)(scratch + ((plan_bytes + 15) / 16) * 16);
    copy_h2d(ctx, dplan, &mo->plan, plan_bytes);
    cudaMemsetAsync(dacc, 0, acc_bytes, st);
    cudaMemsetAsync(ctx->status, 0, 4, st);
    SampleJob J;
    fill_job(mo, J, dplan);
    const int threads = kSampleThreads;
    uint64_t want = (k + threads - 1) / threads;
    uint64_t cap = (uint64_t)ctx->num_sms * TM_SAMPLE_GRID_PER_SM;
    unsigned blocks = (unsigned)std::max<uint64_t>(1, std::min(want, cap));
    if (k / ((uint64_t)blocks * threads) >= 0xFFFFFFFFull)
        return set_err(ctx, TM_E_LIMIT, "too many samples in one call (split the range with first_index)");
    uint32_t *dg = nullptr; uint64_t *dc = nullptr; int32_t *dr = nullptr;
    size_t gbytes = 0;
    int rc;
    {
        PhaseScope ph(ctx, TM_PH_SAMPLE);
        if (trace) {
            gbytes = (size_t)k * (4 * mo->plan.ntree + 8 + 4);
            char *t = (char *)salloc(ctx, gbytes);
            if (!t) return TM_E_NOMEM;
            dc = (uint64_t *)t;
            dr = (int32_t *)(t + (size_t)k * 8);
            dg = (uint32_t *)(t + (size_t)k * 12);
            launch(ctx, k_sample<true>, blocks, threads, ctx->g, dplan, J, seed, first, k, dacc, ctx->status, dg, dc, dr);
        } else if (!launch_sample_reg(ctx, mo->plan, blocks, threads, dplan, J, seed, first, k, dacc)) {
            launch(ctx, k_sample<false>, blocks, threads, ctx->g, dplan, J, seed, first, k, dacc, ctx->status, nullptr,
                                                        nullptr, nullptr);
        }
        rc = check_cuda(ctx, cudaGetLastError(), "sampler launch");
    }
    Acc h{};
    copy_d2h(ctx, &h, dacc, acc_bytes);
    if (trace && rc == TM_OK) {
        if (trace_gids) copy_d2h(ctx, trace_gids, dg, (size_t)k * 4 * mo->plan.ntree);
        if (trace_contrib) copy_d2h(ctx, trace_contrib, dc, (size_t)k * 8);
        if (trace_reason) copy_d2h(ctx, trace_reason, dr, (size_t)k * 4);
    }
    uint32_t bits = 0;
    int rc2 = read_status(ctx, &bits);
    if (rc) return rc;
    if (rc2) return rc2;
    finish_result(mo, k, h, out);
    if (bits & ST_OVERFLOW) return set_err(ctx, TM_E_OVERFLOW, "a completion count exceeds 2^64");
    if (bits) return set_err(ctx, TM_E_CUDA, "sampler reached an inconsistent state (status " + std::to_string(bits) + ")");
    return TM_OK;
}


void finish_result_acc(tm_motif *mo, uint64_t k, const SampleAcc &a, tm_result *out) { finish_result(mo, k, a, out); }

int run_list(tm_ctx *ctx, tm_motif *mo, uint64_t k, uint64_t seed, uint64_t first, uint64_t max_inst,
             uint32_t *inst_gids, uint64_t *inst_sample, uint64_t *n_inst)
{
    ScratchScope scope(ctx);
    cudaStream_t st = ctx->stream;
    *n_inst = 0;
    if (k == 0 || (mo->W.lo == 0 && mo->W.hi == 0)) return TM_OK;
    DevPlan *dplan = (DevPlan *)salloc(ctx, sizeof(DevPlan));
    uint64_t *dcnt = (uint64_t *)salloc(ctx, (size_t)(k + 1) * 8);
    if (!dplan || !dcnt) return TM_E_NOMEM;
    copy_h2d(ctx, dplan, &mo->plan, sizeof(DevPlan));
    cudaMemsetAsync(ctx->status, 0, 4, st);
    SampleJob J;
    fill_job(mo, J, dplan);
    const uint64_t want = (k + kSampleThreads - 1) / kSampleThreads;
    const unsigned blocks = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)ctx->num_sms * 16));
    {
        PhaseScope ph(ctx, TM_PH_SAMPLE);
        launch(ctx, k_list_count, blocks, kSampleThreads, ctx->g, (const DevPlan *)dplan, J, seed, first, k, dcnt,
               ctx->status);
    }
    int rc = check_cuda(ctx, cudaGetLastError(), "listing count");
    if (rc) return rc;
    // row offsets of every sample (exclusive prefix of the counts, on the host)
    std::vector<uint64_t> offs((size_t)k + 1);
    copy_d2h(ctx, offs.data() + 1, dcnt, (size_t)k * 8);
    rc = check_cuda(ctx, cudaStreamSynchronize(st), "listing count copy");
    if (rc) return rc;
    uint32_t bits = 0;
    rc = read_status(ctx, &bits);
    if (rc) return rc;
    if (bits & ST_OVERFLOW) return set_err(ctx, TM_E_OVERFLOW, "a completion count exceeds 2^64");
    if (bits) return set_err(ctx, TM_E_CUDA, "listing reached an inconsistent state");
    offs[0] = 0;
    for (uint64_t i = 1; i <= k; ++i) {
        if (offs[i] > ~0ull - offs[i - 1]) return set_err(ctx, TM_E_OVERFLOW, "instance count exceeds 2^64");
        offs[i] += offs[i - 1];
    }
    *n_inst = offs[k];
    const uint64_t rows = std::min(max_inst, offs[k]);
    if (rows == 0 || !inst_gids || !inst_sample) return TM_OK;
    const size_t ne = mo->ne;
    uint64_t *doffs = dcnt;   // reuse: k + 1 entries
    uint32_t *dg = (uint32_t *)salloc(ctx, (size_t)rows * ne * 4);
    uint64_t *ds = (uint64_t *)salloc(ctx, (size_t)rows * 8);
    if (!dg || !ds) return TM_E_NOMEM;
    copy_h2d(ctx, doffs, offs.data(), (size_t)(k + 1) * 8);
    cudaMemsetAsync(ctx->status, 0, 4, st);
    {
        PhaseScope ph(ctx, TM_PH_SAMPLE);
        launch(ctx, k_list_emit, blocks, kSampleThreads, ctx->g, (const DevPlan *)dplan, J, seed, first, k,
               (const uint64_t *)doffs, rows, dg, ds, ctx->status);
    }
    rc = check_cuda(ctx, cudaGetLastError(), "listing emit");
    if (rc) return rc;
    copy_d2h(ctx, inst_gids, dg, (size_t)rows * ne * 4);
    copy_d2h(ctx, inst_sample, ds, (size_t)rows * 8);
    rc = read_status(ctx, &bits);
    if (rc) return rc;
    if (bits) return set_err(ctx, TM_E_CUDA, "listing disagreed with DeriveCnt (status " + std::to_string(bits) + ")");
    return TM_OK;
}

// Same temporal pattern of the spanning tree: same vertices and delta, and
// per tree node the same endpoints, parent, meeting side, direction, leaf
// flag and pi relation to the parent, in the same pi order.  Then weights,
// sampled trees and validation are identical; only DeriveCnt differs.
static bool same_tree_pattern(const DevPlan &A, const DevPlan &B)
{
    if (A.nv != B.nv || A.ntree != B.ntree || A.delta != B.delta || A.wdelta != B.wdelta || A.c2 != B.c2) return false;
    for (int q = 0; q < A.ntree; ++q) {
        if (A.ea[A.tedge[q]] != B.ea[B.tedge[q]] || A.eb[A.tedge[q]] != B.eb[B.tedge[q]]) return false;
        if (A.tparent[q] != B.tparent[q] || A.tleaf[q] != B.tleaf[q] || A.tzside[q] != B.tzside[q] ||
            A.tout[q] != B.tout[q] || A.tlater[q] != B.tlater[q])
            return false;
    }
    int sa[kMaxE], sb[kMaxE], na = 0, nb = 0;
    for (int pos = 0; pos < A.ne; ++pos) if (A.tnode_of_edge[A.pos_edge[pos]] >= 0) sa[na++] = A.tnode_of_edge[A.pos_edge[pos]];
    for (int pos = 0; pos < B.ne; ++pos) if (B.tnode_of_edge[B.pos_edge[pos]] >= 0) sb[nb++] = B.tnode_of_edge[B.pos_edge[pos]];
    if (na != nb) return false;
    for (int i = 0; i < na; ++i) if (sa[i] != sb[i]) return false;
    return true;
}

template <int NM>
static void launch_group(tm_ctx *ctx, unsigned blocks, const DevPlan *dplans, const SampleJob &J, uint64_t seed,
                         uint64_t first, uint64_t k, Acc *dacc)
{
    launch(ctx, k_sample_group<NM>, blocks, kSampleThreads, ctx->g, dplans, J, seed, first, k, dacc, ctx->status);
}

int run_group(tm_ctx *ctx, tm_motif *const *motifs, uint32_t nm, uint64_t k, uint64_t seed, uint64_t first,
              tm_result *out)
{
    tm_motif *m0 = motifs[0];
    for (uint32_t i = 1; i < nm; ++i)
        if (!same_tree_pattern(m0->plan, motifs[i]->plan))
            return set_err(ctx, TM_E_MOTIF, "motif " + std::to_string(i) + "'s spanning tree differs from motif 0's");
    ScratchScope scope(ctx);
    cudaStream_t st = ctx->stream;
    std::vector<Acc> h(nm, Acc{0, 0, 0, 0, 0, 0});
    if (k == 0 || (m0->W.lo == 0 && m0->W.hi == 0)) {
        for (uint32_t i = 0; i < nm; ++i) finish_result(m0, k, h[i], &out[i]);
        return TM_OK;
    }
    const size_t plan_bytes = sizeof(DevPlan) * nm, acc_bytes = sizeof(Acc) * nm;
    char *scratch = (char *)salloc(ctx, plan_bytes + acc_bytes + 64);
    if (!scratch) return TM_E_NOMEM;
    DevPlan *dplans = (DevPlan *)scratch;
    Acc *dacc = (Acc *)(scratch + ((plan_bytes + 15) / 16) * 16);
    std::vector<DevPlan> hp(nm);
    for (uint32_t i = 0; i < nm; ++i) hp[i] = motifs[i]->plan;
    copy_h2d(ctx, dplans, hp.data(), plan_bytes);
    cudaMemsetAsync(dacc, 0, acc_bytes, st);
    cudaMemsetAsync(ctx->status, 0, 4, st);
    SampleJob J;
    fill_job(m0, J, dplans);
    const uint64_t want = (k + kSampleThreads - 1) / kSampleThreads;
    const unsigned blocks = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)ctx->num_sms * 16));
    {
        PhaseScope ph(ctx, TM_PH_SAMPLE);
        switch (nm) {
        case 1: launch_group<1>(ctx, blocks, dplans, J, seed, first, k, dacc); break;
        case 2: launch_group<2>(ctx, blocks, dplans, J, seed, first, k, dacc); break;
        case 3: launch_group<3>(ctx, blocks, dplans, J, seed, first, k, dacc); break;
        case 4: launch_group<4>(ctx, blocks, dplans, J, seed, first, k, dacc); break;
        case 5: launch_group<5>(ctx, blocks, dplans, J, seed, first, k, dacc); break;
        case 6: launch_group<6>(ctx, blocks, dplans, J, seed, first, k, dacc); break;
        case 7: launch_group<7>(ctx, blocks, dplans, J, seed, first, k, dacc); break;
        default: launch_group<8>(ctx, blocks, dplans, J, seed, first, k, dacc); break;
        }
    }
    int rc = check_cuda(ctx, cudaGetLastError(), "group sampler launch");
    copy_d2h(ctx, h.data(), dacc, acc_bytes);
    uint32_t bits = 0;
    const int rc2 = read_status(ctx, &bits);
    if (rc) return rc;
    if (rc2) return rc2;
    for (uint32_t i = 0; i < nm; ++i) {
        Acc a = h[i];
        a.valid = h[0].valid; a.rv = h[0].rv; a.rd = h[0].rd; a.ro = h[0].ro;
        finish_result(m0, k, a, &out[i]);
    }
    if (bits & ST_OVERFLOW) return set_err(ctx, TM_E_OVERFLOW, "a completion count exceeds 2^64");
    if (bits) return set_err(ctx, TM_E_CUDA, "sampler reached an inconsistent state (status " + std::to_string(bits) + ")");
    return TM_OK;
}


// The batched kernel in one of its shapes: 128 or 256 threads per block,
// per-sample records in local or shared memory.  Persistent: as many blocks
// as fit on the device at once, capped by the number of work items.
template <int T, int S>
static int launch_batch_t(tm_ctx *ctx, uint64_t total, BatchQuery *dq, uint32_t *dbase, uint32_t n, uint32_t tile,
                          uint32_t *dcounter, Acc *dacc)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<T, S>, T, 0);
    uint64_t blocks = (uint64_t)std::max(1, per_sm) * (uint64_t)ctx->num_sms;
    blocks = std::min<uint64_t>(blocks, std::max<uint64_t>(total, 1));
    launch(ctx, k_batch<T, S>, (unsigned)blocks, T, ctx->g, (const BatchQuery *)dq, (const uint32_t *)dbase, n, tile,
           dcounter, dacc, ctx->status);
    return check_cuda(ctx, cudaGetLastError(), "batch launch");
}

static int launch_batch_kernel(tm_ctx *ctx, int threads, int smem_recs, uint64_t total, BatchQuery *dq,
                               uint32_t *dbase, uint32_t n, uint32_t tile, uint32_t *dcounter, Acc *dacc)
{
    if (threads == 128)
        return smem_recs ? launch_batch_t<128, 1>(ctx, total, dq, dbase, n, tile, dcounter, dacc)
                         : launch_batch_t<128, 0>(ctx, total, dq, dbase, n, tile, dcounter, dacc);
    return smem_recs ? launch_batch_t<256, 1>(ctx, total, dq, dbase, n, tile, dcounter, dacc)
                     : launch_batch_t<256, 0>(ctx, total, dq, dbase, n, tile, dcounter, dacc);
}

// One persistent launch over every item's sample tiles (spec batching).
int run_batch_items(tm_ctx *ctx, const BatchItem *items, uint32_t n, uint32_t tile, SampleAcc *acc, int wait_ms)
{
    ScratchScope scope(ctx);
    cudaStream_t st = ctx->stream;
    for (uint32_t i = 0; i < n; ++i) acc[i] = SampleAcc{0, 0, 0, 0, 0, 0};
    if (n == 0) return TM_OK;
    if (tile == 0) tile = 2048;
    std::vector<BatchQuery> hq(n);
    std::vector<uint32_t> base(n + 1, 0);
    uint64_t total = 0;
    for (uint32_t q = 0; q < n; ++q) {
        tm_motif *mo = items[q].mo;
        bool empty = (mo->W.lo == 0 && mo->W.hi == 0);
        uint64_t cnt = empty ? 0 : items[q].count;
        base[q] = (uint32_t)total;
        total += cnt / tile + (cnt % tile != 0 ? 1 : 0);   // no wrap for k near 2^64
        if (total >= 0xFFFFFFF0ull) return set_err(ctx, TM_E_LIMIT, "too many sample tiles in one batch");
        hq[q].plan = mo->plan;
        hq[q].seed = items[q].seed;
        hq[q].first = items[q].first;
        hq[q].k = cnt;
    }
    base[n] = (uint32_t)total;
    if (total == 0) return TM_OK;
    size_t qbytes = sizeof(BatchQuery) * n, bbytes = 4 * (size_t)(n + 1), abytes = sizeof(Acc) * n;
    // sums land in a pinned staging buffer of the context: after a timed-out
    // wait the copy still completes later, into memory that stays valid.
    // Growing it synchronizes, so it happens before anything is launched.
    if (ctx->pinned_acc_bytes < abytes) {
        cudaStreamSynchronize(st);
        if (ctx->pinned_acc) cudaFreeHost(ctx->pinned_acc);
        ctx->pinned_acc = nullptr;
        ctx->pinned_acc_bytes = 0;
        size_t want = std::max<size_t>(abytes, 4096 * sizeof(Acc));
        if (cudaMallocHost(&ctx->pinned_acc, want) != cudaSuccess) {
            cudaGetLastError();
            ctx->pinned_acc = nullptr;
            return set_err(ctx, TM_E_NOMEM, "pinned staging buffer");
        }
        ctx->pinned_acc_bytes = want;
    }
    char *buf = (char *)salloc(ctx, qbytes + bbytes + abytes + 1024);
    if (!buf) return TM_E_NOMEM;
    BatchQuery *dq = (BatchQuery *)buf;
    uint32_t *dbase = (uint32_t *)(buf + ((qbytes + 255) / 256) * 256);
    Acc *dacc = (Acc *)((char *)dbase + ((bbytes + 255) / 256) * 256);
    uint32_t *dcounter = (uint32_t *)((char *)dacc + ((abytes + 255) / 256) * 256);
    for (uint32_t q = 0; q < n; ++q) fill_job(items[q].mo, hq[q].job, &dq[q].plan);
    copy_h2d(ctx, dq, hq.data(), qbytes);
    copy_h2d(ctx, dbase, base.data(), bbytes);
    cudaMemsetAsync(dacc, 0, abytes, st);
    cudaMemsetAsync(dcounter, 0, 4, st);
    cudaMemsetAsync(ctx->status, 0, 4, st);
    int rc;
    {
        PhaseScope ph(ctx, TM_PH_BATCH);
        rc = launch_batch_kernel(ctx, ctx->batch_threads, ctx->batch_smem_recs, total, dq, dbase, n, tile, dcounter,
                                 dacc);
    }
    copy_d2h(ctx, ctx->pinned_acc, dacc, abytes);
    copy_d2h(ctx, ctx->status_host, ctx->status, 4);
    if (rc) { cudaStreamSynchronize(st); return rc; }
    if (wait_ms > 0) {
        // bounded wait: poll the stream until it drains or the limit passes
        cudaEvent_t ev = nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return check_cuda(ctx, cudaGetLastError(), "event");
        cudaEventRecord(ev, st);
        auto t0 = std::chrono::steady_clock::now();
        cudaError_t q;
        while ((q = cudaEventQuery(ev)) == cudaErrorNotReady) {
            if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(wait_ms)) {
                cudaEventDestroy(ev);
                return set_err(ctx, TM_E_TIMEOUT, "batched sampler did not finish within the wait limit");
            }
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
        cudaEventDestroy(ev);
        if (q != cudaSuccess) return check_cuda(ctx, q, "batched sampler");
    } else {
        rc = check_cuda(ctx, cudaStreamSynchronize(st), "batched sampler");
        if (rc) return rc;
    }
    prof_collect(ctx);
    memcpy(acc, ctx->pinned_acc, abytes);
    uint32_t bits = *ctx->status_host;
    if (bits & ST_OVERFLOW) return set_err(ctx, TM_E_OVERFLOW, "a completion count exceeds 2^64");
    if (bits) return set_err(ctx, TM_E_CUDA, "batched sampler reached an inconsistent state");
    return TM_OK;
}

int run_batch(tm_ctx *ctx, uint32_t nq, tm_motif *const *motifs, const uint64_t *k, const uint64_t *seed,
              tm_result *out)
{
    std::vector<BatchItem> items(nq);
    std::vector<SampleAcc> acc(nq);
    for (uint32_t q = 0; q < nq; ++q) items[q] = BatchItem{motifs[q], seed[q], 0, k[q]};
    uint32_t tile = ctx->cfg.sample_tile > 0 ? (uint32_t)ctx->cfg.sample_tile : 2048;
    int rc = run_batch_items(ctx, items.data(), nq, tile, acc.data(), 0);
    if (rc) return rc;
    for (uint32_t q = 0; q < nq; ++q) finish_result(motifs[q], k[q], acc[q], &out[q]);
    return TM_OK;
}

}  // namespace timest

// ---------------------------------------------------------------------------
// Allocation-free sampling.
//
// Some callers cannot allocate device memory while they sample: a serving
// loop that has handed the whole memory pool to resident weights, a host
// framework that owns the allocator and forbids allocations from plug-ins,
// or a latency-bound loop that cannot afford an allocator call (which may
// synchronise the device).  tm_sample_noalloc runs the same sampling kernel
// as tm_sample, but its scratch -- the device copy of the motif plan and the
// result accumulators -- lives in the fixed array below instead of memory
// obtained from the allocator.
// ---------------------------------------------------------------------------
namespace timest {
namespace {

constexpr size_t kNoAllocScratchBytes = 4096;   // plan copy + accumulators
constexpr int kNoAllocMaxDevices = 64;

// One array per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_sample_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
void *g_scratch_addr[kNoAllocMaxDevices] = {};

// Device address of g_sample_scratch on the current device (ctx->device);
// looked up once per device.  The symbol's name in host code is only a
// host-side stand-in, so the kernel must be given this address instead.
int scratch_address(tm_ctx *ctx, unsigned char **out)
{
    if (ctx->device < 0 || ctx->device >= kNoAllocMaxDevices)
        return set_err(ctx, TM_E_LIMIT, "tm_sample_noalloc supports device ordinals below 64");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[ctx->device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_sample_scratch);
        if (e != cudaSuccess) return check_cuda(ctx, e, "cudaGetSymbolAddress(sample scratch)");
        g_scratch_addr[ctx->device] = p;
    }
    *out = (unsigned char *)g_scratch_addr[ctx->device];
    return TM_OK;
}

}  // namespace
}  // namespace timest

extern "C" int tm_sample_noalloc(tm_ctx *ctx, tm_motif *mo, uint64_t k, uint64_t seed, uint64_t first_index,
                                 tm_result *out)
{
    using namespace timest;
    if (!ctx || !mo || mo->ctx != ctx || !out) return TM_E_ARG;
    if (!mo->have_weights || mo->graph_epoch != ctx->epoch || !ctx->preprocessed)
        return set_err(ctx, TM_E_STATE, "weights not computed for the current graph");
    const size_t plan_bytes = ((sizeof(DevPlan) + 15) / 16) * 16;
    const size_t need = plan_bytes + sizeof(Acc);
    if (need > kNoAllocScratchBytes)
        return set_err(ctx, TM_E_LIMIT, "motif plan (" + std::to_string(need) + " bytes) exceeds the " +
                                            std::to_string(kNoAllocScratchBytes) + "-byte allocation-free scratch");
    int rc = check_cuda(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    if (rc) return rc;
    unsigned char *scratch = nullptr;
    rc = scratch_address(ctx, &scratch);
    if (rc) return rc;
    Acc zero{0, 0, 0, 0, 0, 0};
    if (k == 0 || (mo->W.lo == 0 && mo->W.hi == 0)) {
        finish_result(mo, k, zero, out);
        return TM_OK;
    }
    DevPlan *dplan = (DevPlan *)scratch;
    Acc *dacc = (Acc *)(scratch + plan_bytes);
    cudaStream_t st = ctx->stream;
    copy_h2d(ctx, dplan, &mo->plan, sizeof(DevPlan));
    cudaMemsetAsync(dacc, 0, sizeof(Acc), st);   // the array keeps the previous call's sums
    cudaMemsetAsync(ctx->status, 0, 4, st);
    SampleJob J;
    fill_job(mo, J, dplan);
    const int threads = kSampleThreads;
    uint64_t want = (k + threads - 1) / threads;
    uint64_t cap = (uint64_t)ctx->num_sms * 16;
    unsigned blocks = (unsigned)std::max<uint64_t>(1, std::min(want, cap));
    launch(ctx, k_sample<false>, blocks, threads, ctx->g, dplan, J, seed, first_index, k, dacc, ctx->status, nullptr,
           nullptr, nullptr);
    rc = check_cuda(ctx, cudaGetLastError(), "sampler launch");
    Acc h{};
    copy_d2h(ctx, &h, dacc, sizeof(Acc));
    uint32_t bits = 0;
    int rc2 = read_status(ctx, &bits);
    if (rc) return rc;
    if (rc2) return rc2;
    finish_result(mo, k, h, out);
    if (bits & ST_OVERFLOW) return set_err(ctx, TM_E_OVERFLOW, "a completion count exceeds 2^64");
    if (bits) return set_err(ctx, TM_E_CUDA, "sampler reached an inconsistent state (status " + std::to_string(bits) + ")");
    return TM_OK;
}
