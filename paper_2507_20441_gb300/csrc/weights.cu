// Weight pass of TIMEST (Sec. 3.1): windows (Constraint 3, Alg. 1), the
// per-edge dynamic program over the rooted spanning tree (Claims 3.1-3.2,
// Alg. 2), segmented prefix sums of child weights, and the root CDF whose
// window totals give W (Claim 3.4).
//
// Windows [i*delta, (i+2)*delta) with the same parity of i are disjoint, so
// each edge has at most one window per parity ("layer" p = i mod 2) and one
// weight per (tree edge, layer).  The weight of tree node q for edge e in
// layer p is the product over q's children c of
//     sum of w_c over Lambda_z(time range of c) - sum over El(z, o)(same range)
// (the candidate list of Claim 3.1), where both ranges are clipped to e's
// window and the sums are differences of segmented prefix sums.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "scan.cuh"
#include "tm_device.cuh"
#include "tm_internal.h"

namespace timest {

namespace {

constexpr int TB = 256;
inline unsigned blocks_for(uint64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

struct ChildPrefix {
    const uint64_t *pd[2][kMaxTree];   // [layer][slot] prefix in the out/in order
    const uint64_t *pm[2][kMaxTree];   // [layer][slot] prefix in the multi-edge order
};

// Candidate ranges up to this many entries are scanned for the excluded
// neighbour; longer ones search the excluded multi-edge list instead.
constexpr uint32_t kScanLimit = 48;

// One side of tree node q (Claim 3.2): the product of the factors of q's
// children that meet q at its tail (side 0) or head (side 1), for every edge
// matched to q and both layers.  Threads walk the meeting vertex's own list
// (out-list order for side 0, in-list order for side 1), so the lanes of a
// warp share the vertex, its candidate lists and nearby positions in them.
// Each child's range [a, b) is galloped to from the parent edge's position
// in that list (or its cross rank into the vertex's other list).  The
// excluded entries of Claim 3.1 are exactly the entries of [a, b) whose other
// endpoint is the parent's other endpoint: short ranges are scanned for them
// in place; long ones search the excluded multi-edge list.
// Results are written in this list order.  A root with children at both ends
// runs side 0 (first) then side 1 (last), which reads side 0's partial
// product and pending-overflow bit through the out->in position map.
// Overflow rule: a factor >= 2^64, or an exact product >= 2^64 with no zero
// factor.
#ifndef TM_DP_MINB
#define TM_DP_MINB 6   // 40 registers: six blocks of 256 per SM (measured fastest)
#endif
__global__ void __launch_bounds__(256, TM_DP_MINB) k_dp(DevGraph g, DevPlan P, int q, int side, int first, int last,
                                            ChildPrefix cp, ulonglong2 *__restrict__ wout,
                                            const ulonglong2 *__restrict__ in, const uint8_t *__restrict__ pin,
                                            uint8_t *__restrict__ pout, uint32_t *status)
{
    const uint32_t pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= g.m) return;
    const uint32_t t = __ldg((side ? g.in_t : g.out_t) + pos);
    const uint32_t z = __ldg((side ? g.in_dst : g.out_src) + pos);
    // the parent's other endpoint; without Constraint 2 nothing is excluded
    const uint32_t o = P.c2 ? __ldg((side ? g.in_nbr : g.out_nbr) + pos) : kNone;
    const uint32_t pr = __ldg((side ? g.in_pair : g.out_pair) + pos);
    const int64_t d = P.delta, wd = P.wdelta;
    uint64_t wlo[2], whi[2], prod[2] = {1, 1};
    bool zero[2], ovf[2] = {false, false};
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int64_t wi = layer_window(t, p, wd);
        zero[p] = wi < 0;
        wlo[p] = zero[p] ? 0 : (uint64_t)(wi * wd);
        whi[p] = zero[p] ? 0 : (uint64_t)((wi + 2) * wd - 1);
    }
    if (!first) {
        const uint32_t xp = __ldg(g.in_to_out + pos);   // side 1 reads side 0's partial (both layers)
        const ulonglong2 pv = __ldg(in + xp);
        const uint32_t pb = pin[xp];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            if (zero[p]) continue;
            prod[p] = p ? pv.y : pv.x;
            ovf[p] = (pb >> p) & 1u;
            if (prod[p] == 0) zero[p] = true;
        }
    }
    for (int ci = 0; ci < P.nchild[q] && !(zero[0] && zero[1]); ++ci) {
        const int c = P.child[q][ci];
        if (P.tzside[c] != side) continue;
        const bool out = P.tout[c] != 0, later = P.tlater[c] != 0, leaf = P.tleaf[c] != 0;
        if (!later && t == 0) { zero[0] = zero[1] = true; break; }
        const uint32_t *off = out ? g.out_off : g.in_off;
        const uint32_t *tarr = out ? g.out_t : g.in_t;
        const uint32_t *nbr = out ? g.out_nbr : g.in_nbr;
        const uint32_t beg = __ldg(off + z), end = __ldg(off + z + 1);
        const uint32_t base = ((side == 0) == out) ? gallop_back(tarr, beg, pos, t)
                                                   : __ldg((side == 0 ? g.out_xrank : g.in_xrank) + pos);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            if (zero[p]) continue;
            uint64_t lo, hi;
            if (later) { lo = (uint64_t)t + 1; hi = (uint64_t)t + (uint64_t)d; }
            else { lo = (uint64_t)t >= (uint64_t)d ? (uint64_t)t - (uint64_t)d : 0; hi = (uint64_t)t - 1; }
            lo = lo < wlo[p] ? wlo[p] : lo;
            hi = hi > whi[p] ? whi[p] : hi;
            if (lo > hi) { zero[p] = true; continue; }
            uint32_t a, b;
            if (later) { a = gallop_idx(tarr, base, end, lo); b = gallop_idx(tarr, a, end, hi + 1); }
            else { b = base; a = gallop_back(tarr, beg, base, lo); }
            const uint64_t *Pd = leaf ? nullptr : cp.pd[p][P.tslot[c]];
            uint64_t pbase = 0, sum;
            if (!leaf && b > a) pbase = (a > beg && (uint64_t)__ldg(tarr + a - 1) >= wlo[p]) ? __ldg(Pd + a - 1) : 0;
            uint64_t excl = 0;
            if (b - a <= kScanLimit) {
                uint64_t prev = pbase;
                for (uint32_t x = a; x < b; ++x) {
                    uint64_t wx = 1;
                    if (!leaf) { const uint64_t px = __ldg(Pd + x); wx = px - prev; prev = px; }
                    if (__ldg(nbr + x) == o) excl += wx;
                }
            } else {
                const uint32_t pe = !P.c2 ? kNone : (out == (side == 0)) ? pr : __ldg(g.rev_pair + pr);
                if (pe != kNone) {
                    const uint32_t xb = __ldg(g.pair_off + pe), xe = __ldg(g.pair_off + pe + 1);
                    const uint32_t ea = lower_idx(g.multi_t, xb, xe, lo);
                    const uint32_t eb = gallop_idx(g.multi_t, ea, xe, hi + 1);
                    if (eb > ea) {
                        if (leaf) excl = eb - ea;
                        else {
                            const uint64_t *Pm = cp.pm[p][P.tslot[c]];
                            const uint64_t bs = (ea > xb && (uint64_t)__ldg(g.multi_t + ea - 1) >= wlo[p]) ? __ldg(Pm + ea - 1) : 0;
                            excl = __ldg(Pm + eb - 1) - bs;
                        }
                    }
                }
            }
            if (leaf) sum = (uint64_t)(b - a) - excl;
            else sum = (b > a ? __ldg(Pd + b - 1) - pbase : 0) - excl;
            if (sum == 0) zero[p] = true;
            else prod[p] = mul_chk(prod[p], sum, ovf[p]);
        }
    }
    wout[pos] = make_ulonglong2(zero[0] ? 0 : prod[0], zero[1] ? 0 : prod[1]);   // both layers, one store
    if (!last) pout[pos] = (uint8_t)(((!zero[0] && ovf[0]) ? 1u : 0u) | ((!zero[1] && ovf[1]) ? 2u : 0u));
    if (last && ((!zero[0] && ovf[0]) || (!zero[1] && ovf[1]))) latch(status, ST_OVERFLOW);
}

// ---- scans over the three orders ----------------------------------------
// segment = (owner, window of layer p); owner boundaries come from a bit set.
// Segment heads of one layer (exports rebuild weights from prefix sums).
struct DirHead {
    const uint32_t *tarr;       // position -> t'
    const uint32_t *ownbits;    // bit set: position starts a new owner
    int p;
    int64_t d;
    __device__ bool head(uint64_t i) const
    {
        if (i == 0) return true;
        if ((__ldg(ownbits + (i >> 5)) >> (i & 31)) & 1u) return true;
        return layer_window(__ldg(tarr + i), p, d) != layer_window(__ldg(tarr + i - 1), p, d);
    }
};

struct RootHead {
    const uint32_t *tarr;       // g_t
    int p;
    int64_t d;
    __device__ bool head(uint64_t i) const
    {
        if (i == 0) return true;
        return layer_window(__ldg(tarr + i), p, d) != layer_window(__ldg(tarr + i - 1), p, d);
    }
};

// Both layers at once (two-lane scans): the pair of weights of a position is
// one 16-byte gather; heads are per layer (bit p).
struct DirScan2 {
    static constexpr bool kGathered = true;
    const ulonglong2 *w;        // (layer 0, layer 1) weights in the order the DP wrote them
    const uint32_t *perm;       // scan position -> weight position (null: same order)
    const uint32_t *tarr;       // position -> t'
    const uint32_t *ownbits;    // bit set: position starts a new owner
    int64_t d;
    __device__ ulonglong2 value2(uint64_t i) const { return __ldg(w + (perm ? __ldg(perm + i) : i)); }
    __device__ uint32_t head2(uint64_t i) const
    {
        if (i == 0 || ((__ldg(ownbits + (i >> 5)) >> (i & 31)) & 1u)) return 3u;
        const uint32_t a = __ldg(tarr + i), b = __ldg(tarr + i - 1);
        return (layer_window(a, 0, d) != layer_window(b, 0, d) ? 1u : 0u) |
               (layer_window(a, 1, d) != layer_window(b, 1, d) ? 2u : 0u);
    }
};

struct RootScan2 {
    static constexpr bool kGathered = true;
    const ulonglong2 *w;        // root weight pairs in list order
    const uint32_t *tarr;       // g_t
    int64_t d;
    const uint32_t *perm;       // gid -> weight position
    __device__ ulonglong2 value2(uint64_t i) const { return __ldg(w + (perm ? __ldg(perm + i) : i)); }
    __device__ uint32_t head2(uint64_t i) const
    {
        if (i == 0) return 3u;
        const uint32_t a = __ldg(tarr + i), b = __ldg(tarr + i - 1);
        return (layer_window(a, 0, d) != layer_window(b, 0, d) ? 1u : 0u) |
               (layer_window(a, 1, d) != layer_window(b, 1, d) ? 2u : 0u);
    }
};

// Window heads of layer p in GLOBAL order.
// Window heads of both layers (layer p = blockIdx.y) into flag[p*m + i].
__global__ void k_window_heads(const uint32_t *__restrict__ t, uint32_t m, int64_t d, uint32_t *__restrict__ flag)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (i >= m) return;
    const int64_t w = layer_window(t[i], p, d);
    flag[(size_t)p * m + i] = (w >= 0 && (i == 0 || layer_window(t[i - 1], p, d) != w)) ? 1u : 0u;
}

// The exclusive scan ran over both layers' flags back to back: layer 0 has
// pos[m] windows, layer 1 the rest of the total.
__global__ void k_window_counts(const uint32_t *__restrict__ pos, uint32_t m, uint32_t *__restrict__ counts)
{
    const uint32_t c0 = pos[m];
    counts[1] -= c0;
    counts[0] = c0;
}

struct WinOut {
    uint32_t *beg[2], *id[2];
    uint32_t nwin[2];
};

// Both layers (p = blockIdx.y): window starts and indices; layer 1's scanned
// positions start at layer 0's count (base).  Also the end sentinels.
__global__ void k_window_fill(const uint32_t *__restrict__ t, const uint32_t *__restrict__ flag,
                              const uint32_t *__restrict__ pos, uint32_t m, int64_t d, uint32_t base1, WinOut W)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    uint32_t *beg = p ? W.beg[1] : W.beg[0], *wid = p ? W.id[1] : W.id[0];
    if (i == 0) beg[p ? W.nwin[1] : W.nwin[0]] = m;
    if (i >= m || !flag[(size_t)p * m + i]) return;
    const uint32_t k = pos[(size_t)p * m + i] - (p ? base1 : 0);
    beg[k] = i;
    wid[k] = (uint32_t)layer_window(t[i], p, d);
}

// Window totals W_i (last root-CDF entry of each window) and their 128-bit
// running sum over (layer 0 windows, layer 1 windows).  One block; each
// thread scans a contiguous chunk.
__global__ void k_window_cum(const uint64_t *__restrict__ cdf0, const uint32_t *__restrict__ beg0, uint32_t nw0,
                             const uint64_t *__restrict__ cdf1, const uint32_t *__restrict__ beg1, uint32_t nw1,
                             uint64_t *__restrict__ wcum)
{
    __shared__ u128 warp_tot[32];
    const uint32_t n = nw0 + nw1;
    const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
    uint32_t lo = threadIdx.x * per, hi = min(n, lo + per);
    if (lo > n) lo = n;
    auto total = [&](uint32_t k) -> uint64_t {
        if (k < nw0) return cdf0[beg0[k + 1] - 1];
        k -= nw0;
        return cdf1[beg1[k + 1] - 1];
    };
    u128 s = 0;
    for (uint32_t k = lo; k < hi; ++k) s += total(k);
    // exclusive scan of the chunk sums (128-bit) across the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u128 incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t yl = __shfl_up_sync(0xffffffffu, (uint64_t)incl, o);
        uint64_t yh = __shfl_up_sync(0xffffffffu, (uint64_t)(incl >> 64), o);
        if (lane >= o) incl += (u128)yl | ((u128)yh << 64);
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        u128 run = 0;
        const int nw = (blockDim.x + 31) / 32;
        for (int w = 0; w < nw; ++w) { u128 c = warp_tot[w]; warp_tot[w] = run; run += c; }
        wcum[2 * (size_t)n] = (uint64_t)run;
        wcum[2 * (size_t)n + 1] = (uint64_t)(run >> 64);
    }
    __syncthreads();
    u128 run = warp_tot[warp] + incl - s;
    for (uint32_t k = lo; k < hi; ++k) {
        wcum[2 * (size_t)k] = (uint64_t)run;
        wcum[2 * (size_t)k + 1] = (uint64_t)(run >> 64);
        run += total(k);
    }
}

// ---- guide table of the root search --------------------------------------
// Window kk of a layer gets about n/4 buckets of width 2^s over its draws
// [0, W_kk); the table holds, per bucket j, the first edge whose in-window
// CDF exceeds j 2^s, then the window's last edge.  count[kk] = buckets + 1.
__device__ __forceinline__ uint64_t ceil_shift(uint64_t c, uint32_t s) { return (c >> s) + ((c & ((1ull << s) - 1)) != 0); }

struct GuideLayer {
    const uint64_t *cdf;
    const uint32_t *win_beg, *flag, *pos;
    uint32_t pbase;             // first scanned position of this layer's windows
    uint32_t nwin;
    uint32_t *gshift, *goff, *guide;
};
struct GuideArgs {
    GuideLayer L[2];
};

// One block per layer: each thread sizes a contiguous run of windows, then
// the block turns the counts into the windows' table offsets.
__global__ void __launch_bounds__(1024) k_guide_setup(GuideArgs A)
{
    __shared__ uint32_t warp_tot[32];
    const GuideLayer &L = blockIdx.x ? A.L[1] : A.L[0];
    const uint32_t nw = L.nwin, per = (nw + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = min(nw, threadIdx.x * per), hi = min(nw, lo + per);
    uint32_t sum = 0;
    for (uint32_t kk = lo; kk < hi; ++kk) {
        const uint32_t n = L.win_beg[kk + 1] - L.win_beg[kk];
        const uint64_t W = L.cdf[L.win_beg[kk + 1] - 1];
        const uint64_t target = n >> 2 ? n >> 2 : 1;
        uint32_t sh = 0;
        while (sh < 63 && W && ((W - 1) >> sh) + 1 > target) ++sh;
        L.gshift[kk] = sh;
        const uint32_t c = (uint32_t)(W ? ((W - 1) >> sh) + 1 : 0) + 1;
        L.goff[kk] = c;   // count for now, offset below
        sum += c;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) { const uint32_t c = warp_tot[w]; warp_tot[w] = run; run += c; }
    }
    __syncthreads();
    uint32_t run = warp_tot[warp] + incl - sum;
    for (uint32_t kk = lo; kk < hi; ++kk) {
        const uint32_t c = L.goff[kk];
        L.goff[kk] = run;
        run += c;
    }
}

// one thread per edge and layer (blockIdx.y): the buckets whose lower bound
// falls in [cdf[x-1], cdf[x]) start at x
__global__ void k_guide_fill(GuideArgs A, const uint32_t *__restrict__ t, uint32_t m, int64_t d)
{
    const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (x >= m || layer_window(t[x], p, d) < 0) return;
    const GuideLayer &L = p ? A.L[1] : A.L[0];
    const uint32_t kk = L.pos[x] + L.flag[x] - 1 - L.pbase;
    const uint32_t wbeg = L.win_beg[kk], wend = L.win_beg[kk + 1];
    const uint32_t sh = L.gshift[kk];
    uint32_t *G = L.guide + L.goff[kk];
    const uint64_t c1 = L.cdf[x], c0 = x > wbeg ? L.cdf[x - 1] : 0;
    const uint64_t j1 = ceil_shift(c1, sh);
    for (uint64_t j = ceil_shift(c0, sh); j < j1; ++j) G[j] = x;
    if (x == wend - 1) G[j1] = x;
}

// Reconstruct w for one order from its segmented prefix (exports).
template <class F>
__global__ void k_unprefix(F f, const uint64_t *__restrict__ pref, const uint32_t *__restrict__ perm, uint32_t m,
                           uint64_t *__restrict__ out)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    uint64_t w = pref[i] - (f.head(i) ? 0 : pref[i - 1]);
    out[perm ? perm[i] : i] = w;
}

__global__ void k_leaf_weights(const uint32_t *__restrict__ t, uint32_t m, int p, int64_t d, uint64_t *__restrict__ out)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) out[i] = layer_window(t[i], p, d) >= 0 ? 1 : 0;
}

}  // namespace

static void *malloc_motif(tm_ctx *ctx, tm_motif *mo, size_t bytes)
{
    void *p = dalloc(ctx, bytes ? bytes : 8);
    if (p) { mo->bufs.push_back({p, bytes ? bytes : 8}); mo->bytes += bytes; }
    return p;
}

static void free_motif_weights(tm_ctx *ctx, tm_motif *mo)
{
    for (auto &b : mo->bufs) dfree(ctx, b.first, b.second);
    mo->bufs.clear();
    mo->bytes = 0;
    for (int p = 0; p < 2; ++p) mo->layer[p] = LayerData();
    mo->wcum = nullptr;
    mo->have_weights = false;
}

// Owner bit sets of the out-, in- and multi-edge orders (built with the graph).
struct OwnerBits { const uint32_t *out, *in, *multi; };

int compute_weights(tm_ctx *ctx, tm_motif *mo)
{
    ScratchScope scope(ctx);
    free_motif_weights(ctx, mo);
    const DevGraph &g = ctx->g;
    const DevPlan &P = mo->plan;
    cudaStream_t st = ctx->stream;
    const uint32_t m = g.m;
    const int64_t d = P.wdelta;   // window unit (delta, or one window without Constraint 3)
    int rc = TM_OK;
    cudaMemsetAsync(ctx->status, 0, 4, st);
    // ---- windows of each layer (K2): count both layers, then one block for
    // everything the motif keeps (windows, root CDF, prefix arrays, totals)
    // both layers' flags and scanned positions back to back: [p*m, (p+1)*m)
    uint32_t *flag_all, *pos_all, *flag[2], *pos[2], *dcount;
    uint32_t nwh[2] = {0, 0};
    {
        PhaseScope ph(ctx, TM_PH_WINDOWS);
        dcount = (uint32_t *)salloc(ctx, 8);
        flag_all = (uint32_t *)salloc(ctx, (size_t)(m ? m : 1) * 8);
        pos_all = (uint32_t *)salloc(ctx, ((size_t)m + 1) * 8);
        if (!dcount || !flag_all || !pos_all) return TM_E_NOMEM;
        for (int p = 0; p < 2; ++p) { flag[p] = flag_all + (size_t)p * m; pos[p] = pos_all + (size_t)p * m; }
        cudaMemsetAsync(dcount, 0, 8, st);
        if (m) {
            launch(ctx, k_window_heads, dim3(blocks_for(m, TB), 2), TB, g.g_t, m, d, flag_all);
            rc = exclusive_scan_u32(ctx, flag_all, pos_all, 2 * (uint64_t)m, dcount + 1);
            if (rc) return rc;
            launch(ctx, k_window_counts, 1, 1, (const uint32_t *)pos_all, m, dcount);
        }
        copy_d2h(ctx, nwh, dcount, 8);
        rc = check_cuda(ctx, cudaStreamSynchronize(st), "window count");
        if (rc) return rc;
    }
    {
        auto al = [](size_t b) { return (b + 255) / 256 * 256; };
        const size_t mm = (size_t)(m ? m : 1);
        auto guide_n = [&](uint32_t nw) { return (size_t)m / 4 + 3 * (size_t)nw + 1; };
        size_t total = al(((size_t)nwh[0] + 1) * 4) * 4 + al(((size_t)nwh[1] + 1) * 4) * 4 + 2 * al(mm * 8) +
                       (size_t)P.nslots * 4 * al(mm * 8) + al(((size_t)nwh[0] + nwh[1] + 1) * 16) +
                       al(guide_n(nwh[0]) * 4) + al(guide_n(nwh[1]) * 4);
        char *blk = (char *)malloc_motif(ctx, mo, total);
        if (!blk) return TM_E_NOMEM;
        size_t off = 0;
        auto take = [&](size_t bytes) { char *q = blk + off; off += al(bytes); return (void *)q; };
        for (int p = 0; p < 2; ++p) {
            LayerData &L = mo->layer[p];
            L.nwin = nwh[p];
            L.win_beg = (uint32_t *)take(((size_t)nwh[p] + 1) * 4);
            L.win_id = (uint32_t *)take(((size_t)nwh[p] + 1) * 4);
            L.root_cdf = (uint64_t *)take(mm * 8);
            L.win_gshift = (uint32_t *)take(((size_t)nwh[p] + 1) * 4);
            L.win_goff = (uint32_t *)take(((size_t)nwh[p] + 1) * 4);
            L.guide = (uint32_t *)take(guide_n(nwh[p]) * 4);
            for (int sl = 0; sl < P.nslots; ++sl) {
                L.pref_dir[sl] = (uint64_t *)take(mm * 8);
                L.pref_multi[sl] = (uint64_t *)take(mm * 8);
            }
        }
        mo->wcum = (uint64_t *)take(((size_t)nwh[0] + nwh[1] + 1) * 16);
    }
    {
        PhaseScope ph(ctx, TM_PH_WINDOWS);
        WinOut wo{{mo->layer[0].win_beg, mo->layer[1].win_beg}, {mo->layer[0].win_id, mo->layer[1].win_id},
                  {nwh[0], nwh[1]}};
        launch(ctx, k_window_fill, dim3(blocks_for(m ? m : 1, TB), 2), TB, g.g_t, (const uint32_t *)flag_all,
               (const uint32_t *)pos_all, m, d, nwh[0], wo);
    }
    // ---- DP over tree nodes in increasing height (K3) + prefixes (K4)
    const OwnerBits ob{g.own_out, g.own_in, g.own_multi};
    ulonglong2 *w = nullptr, *pw = nullptr;   // (layer 0, layer 1) weight pairs
    uint8_t *pend = nullptr;                  // bit p: pending overflow of layer p's partial
    w = (ulonglong2 *)salloc(ctx, (size_t)(m ? m : 1) * 16);
    if (!w) return TM_E_NOMEM;
    ChildPrefix cp{};
    int maxh = 0;
    for (int q = 0; q < P.ntree; ++q) maxh = std::max(maxh, (int)P.height[q]);
    std::vector<int> order;
    for (int h = 1; h <= maxh; ++h)
        for (int q = P.ntree - 1; q >= 0; --q)
            if (P.height[q] == h) order.push_back(q);
    if (P.tleaf[0]) order.push_back(0);   // single-edge motif: the root is a leaf
    for (int q : order) {
        // sides of q that children meet; the weights come out in the order of
        // the last side run (out-list order for side 0, in-list for side 1)
        bool has[2] = {false, false};
        for (int ci = 0; ci < P.nchild[q]; ++ci) has[P.tzside[P.child[q][ci]]] = true;
        const bool in_order = has[1];
        {
            PhaseScope ph(ctx, TM_PH_DP);
            if (has[0] && has[1] && !pw) {
                pw = (ulonglong2 *)salloc(ctx, (size_t)(m ? m : 1) * 16);
                pend = (uint8_t *)salloc(ctx, (size_t)(m ? m : 1));
                if (!pw || !pend) return TM_E_NOMEM;
            }
            if (m) {
                if (has[0] && has[1]) {
                    launch(ctx, k_dp, blocks_for(m, TB), TB, g, P, q, 0, 1, 0, cp, pw, (const ulonglong2 *)nullptr,
                           (const uint8_t *)nullptr, pend, ctx->status);
                    launch(ctx, k_dp, blocks_for(m, TB), TB, g, P, q, 1, 0, 1, cp, w, (const ulonglong2 *)pw,
                           (const uint8_t *)pend, (uint8_t *)nullptr, ctx->status);
                } else {
                    launch(ctx, k_dp, blocks_for(m, TB), TB, g, P, q, in_order ? 1 : 0, 1, 1, cp, w,
                           (const ulonglong2 *)nullptr, (const uint8_t *)nullptr, (uint8_t *)nullptr, ctx->status);
                }
            }
        }
        rc = check_cuda(ctx, cudaGetLastError(), "weight DP");
        if (rc) return rc;
        if (q == 0) {
            PhaseScope ph(ctx, TM_PH_ROOT);
            GuideArgs ga{};
            RootScan2 f{w, g.g_t, d, in_order ? g.in_pos : g.out_pos};
            rc = segmented_scan2_u64(ctx, f, m, mo->layer[0].root_cdf, mo->layer[1].root_cdf);
            if (rc) return rc;
            for (int p = 0; p < 2; ++p) {
                LayerData &L = mo->layer[p];
                ga.L[p] = GuideLayer{L.root_cdf, L.win_beg, flag[p], pos[p], p ? nwh[0] : 0u, L.nwin, L.win_gshift,
                                     L.win_goff, L.guide};
            }
            // guide tables of the root search, both layers
            if (m) {
                launch(ctx, k_guide_setup, 2, 1024, ga);
                launch(ctx, k_guide_fill, dim3(blocks_for(m, TB), 2), TB, ga, g.g_t, m, d);
            }
        } else {
            PhaseScope ph(ctx, TM_PH_PREFIX);
            int slot = P.tslot[q];
            bool out = P.tout[q] != 0;
            // scan order of the parent's candidate list -> position of the weight
            const uint32_t *dmap = (out == !in_order) ? nullptr : (out ? g.out_to_in : g.in_to_out);
            const uint32_t *mmap = in_order ? g.multi_to_in : g.multi_to_out;
            LayerData &L0 = mo->layer[0], &L1 = mo->layer[1];
            DirScan2 fd{w, dmap, out ? g.out_t : g.in_t, out ? ob.out : ob.in, d};
            rc = segmented_scan2_u64(ctx, fd, m, L0.pref_dir[slot], L1.pref_dir[slot]);
            if (rc) return rc;
            DirScan2 fm{w, mmap, g.multi_t, ob.multi, d};
            rc = segmented_scan2_u64(ctx, fm, m, L0.pref_multi[slot], L1.pref_multi[slot]);
            if (rc) return rc;
            for (int p = 0; p < 2; ++p) {
                cp.pd[p][slot] = mo->layer[p].pref_dir[slot];
                cp.pm[p][slot] = mo->layer[p].pref_multi[slot];
            }
        }
    }
    // ---- window totals and their 128-bit running sum (K5)
    uint32_t nw0 = mo->layer[0].nwin, nw1 = mo->layer[1].nwin;
    mo->nwtot = nw0 + nw1;
    uint64_t Wh[2] = {0, 0};
    {
        PhaseScope ph(ctx, TM_PH_ROOT);
        launch(ctx, k_window_cum, 1, 1024, mo->layer[0].root_cdf, mo->layer[0].win_beg, nw0, mo->layer[1].root_cdf,
                                         mo->layer[1].win_beg, nw1, mo->wcum);
        copy_d2h(ctx, Wh, mo->wcum + 2 * (size_t)mo->nwtot, 16);
    }
    uint32_t bits = 0;
    rc = read_status(ctx, &bits);
    if (rc) return rc;
    if (bits & ST_OVERFLOW) return set_err(ctx, TM_E_OVERFLOW, "a weight, prefix sum or window total exceeds 2^64");
    if (bits) return set_err(ctx, TM_E_CUDA, "device status error in weight pass");
    mo->W.lo = Wh[0];
    mo->W.hi = Wh[1];
    mo->have_weights = true;
    mo->graph_epoch = ctx->epoch;
    return TM_OK;
}

// w_{q,e} by gid for one layer, rebuilt from the stored prefix arrays.
int export_weights(tm_ctx *ctx, tm_motif *mo, int q, int layer, uint64_t *host_out)
{
    ScratchScope scope(ctx);
    const DevGraph &g = ctx->g;
    const DevPlan &P = mo->plan;
    cudaStream_t st = ctx->stream;
    uint32_t m = g.m;
    if (m == 0) return TM_OK;
    uint64_t *out = (uint64_t *)salloc(ctx, (size_t)m * 8);
    if (!out) return TM_E_NOMEM;
    int rc = TM_OK;
    if (P.tleaf[q] && q != 0) {
        launch(ctx, k_leaf_weights, blocks_for(m, TB), TB, g.g_t, m, layer, P.wdelta, out);
    } else if (q == 0) {
        RootHead f{g.g_t, layer, P.wdelta};
        launch(ctx, k_unprefix<RootHead>, blocks_for(m, TB), TB, f, mo->layer[layer].root_cdf, nullptr, m, out);
    } else {
        const OwnerBits ob{g.own_out, g.own_in, g.own_multi};
        bool o = P.tout[q] != 0;
        DirHead f{o ? g.out_t : g.in_t, o ? ob.out : ob.in, layer, P.wdelta};
        launch(ctx, k_unprefix<DirHead>, blocks_for(m, TB), TB, f, mo->layer[layer].pref_dir[P.tslot[q]],
                                                              o ? g.out_gid : g.in_gid, m, out);
        rc = check_cuda(ctx, cudaStreamSynchronize(st), "export");
    }
    copy_d2h(ctx, host_out, out, (size_t)m * 8);
    int rc2 = check_cuda(ctx, cudaStreamSynchronize(st), "export copy");
    return rc ? rc : rc2;
}

void release_weights(tm_ctx *ctx, tm_motif *mo) { free_motif_weights(ctx, mo); }

}  // namespace timest
