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

// Prefix arrays of the child nodes: per position the (layer 0, layer 1)
// prefix pair, so one 16-byte load serves both layers.
struct ChildPrefix {
    const ulonglong2 *pd[kMaxTree];    // [slot] prefix in the out/in order
    const ulonglong2 *pm[kMaxTree];    // [slot] prefix in the multi-edge order
};

__device__ __forceinline__ uint64_t lane_of(const ulonglong2 v, int p) { return p ? v.y : v.x; }

// a[i] for a runtime slot i by a chain of selects: indexing a kernel
// parameter array at a runtime index would copy it to local memory
__device__ __forceinline__ const ulonglong2 *pick_slot(const ulonglong2 *const (&a)[kMaxTree], int i)
{
    const ulonglong2 *v = a[0];
#pragma unroll
    for (int s = 1; s < kMaxTree; ++s) v = (i == s) ? a[s] : v;
    return v;
}

// Candidate ranges up to this many entries are scanned for the excluded
// neighbour; longer ones search the excluded multi-edge list instead.
#ifndef TM_DP_SCAN_LIMIT
#define TM_DP_SCAN_LIMIT 96   // measured: 96 and 128 beat 48, 16 and 8 on the 5e7-edge workload
#endif
constexpr uint32_t kScanLimit = TM_DP_SCAN_LIMIT;

// One side of tree node q (Claim 3.2): the product of the factors of q's
// children that meet q at its tail (side 0) or head (side 1), for every edge
// matched to q and both layers.  Threads walk the meeting vertex's own list
// (out-list order for side 0, in-list order for side 1), so the lanes of a
// warp share the vertex, its candidate lists and nearby positions in them.
// Each child's range is galloped to from the parent edge's position in that
// list (or its cross rank into the vertex's other list).  Both layers share
// the unclipped range: e's windows of the two layers both contain t, so the
// bound on the side of e itself is common and only the far bound is clipped,
// in at most one layer, by a search inside the unclipped range.  The
// excluded entries of Claim 3.1 are exactly the entries of the range whose
// other endpoint is the parent's other endpoint: short ranges are scanned for
// them in place (one pass serves both layers); long ones search the excluded
// multi-edge list.
// Results are written in this list order, or through `scatter` into another
// order (a node whose parent scans the out-list order while its own DP runs
// in in-list order writes through the in -> out map).  A root with children at both ends
// runs side 0 (first) then side 1 (last), which reads side 0's partial
// product through the out->in position map, and its pending-overflow bits
// from two bit sets of m/32 words (one per layer; a warp of side 0 writes
// the word of its 32 positions with a ballot), small enough to stay in L2.
// Overflow rule: a factor >= 2^64, or an exact product >= 2^64 with no zero
// factor.
#ifndef TM_DP_MINB
#define TM_DP_MINB 5   // 48 registers, five blocks of 256 per SM (measured faster than 40 or 64 registers)
#endif
__global__ void __launch_bounds__(256, TM_DP_MINB) k_dp(DevGraph g, DevPlan P, WinDiv wv, int q, int side, int first,
                                                        int last, ChildPrefix cp, ulonglong2 *__restrict__ wout,
                                                        const uint32_t *__restrict__ scatter,
                                                        const ulonglong2 *__restrict__ in,
                                                        const uint32_t *__restrict__ pin, uint32_t *__restrict__ pout,
                                                        uint32_t *status)
{
    const uint32_t pos = blockIdx.x * blockDim.x + threadIdx.x;
    // whole warps stay for the pending-bit ballots of side 0
    if (pos >= g.m && (last || (pos & ~31u) >= g.m)) return;
    const bool live = pos < g.m;
    uint32_t pend_bits = 0;
    if (live) {
        const uint32_t t = __ldg((side ? g.in_t : g.out_t) + pos);
        const uint32_t z = __ldg((side ? g.in_dst : g.out_src) + pos);
        // the parent's other endpoint; without Constraint 2 nothing is excluded
        const uint32_t o = P.c2 ? __ldg((side ? g.in_nbr : g.out_nbr) + pos) : kNone;
        const uint64_t d = (uint64_t)P.delta, wd = (uint64_t)wv.d;
        const uint32_t qt = wv.quot(t);
        // window bounds as 32-bit times: wlo <= t fits, whi is clamped to the
        // largest t' (no time lies beyond it), which leaves every comparison
        // below unchanged and keeps the bounds in half the registers
        uint32_t wlo[2], whi[2];
        uint64_t prod[2] = {1, 1};
        bool zero[2], ovf[2] = {false, false};
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int64_t wi = WinDiv::win_of(qt, p);
            zero[p] = wi < 0;
            const uint64_t whi64 = ((uint64_t)wi + 2) * wd - 1;
            wlo[p] = zero[p] ? 0u : (uint32_t)((uint64_t)wi * wd);
            whi[p] = zero[p] ? 0u : (whi64 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)whi64);
        }
        if (!first) {
            const uint32_t xp = __ldg(g.in_to_out + pos);   // side 1 reads side 0's partial (both layers)
            const ulonglong2 pv = __ldg(in + xp);
            const uint32_t words = (g.m + 31) >> 5;
            const uint32_t pb = ((__ldg(pin + (xp >> 5)) >> (xp & 31)) & 1u) |
                                (((__ldg(pin + words + (xp >> 5)) >> (xp & 31)) & 1u) << 1);
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                if (zero[p]) continue;
                prod[p] = lane_of(pv, p);
                ovf[p] = (pb >> p) & 1u;
                if (prod[p] == 0) zero[p] = true;
            }
        }
        for (int ci = 0; ci < P.nchild[q] && !(zero[0] && zero[1]); ++ci) {
            const int c = P.child[q][ci];
            if (P.tzside[c] != side) continue;
            const bool out = P.tout[c] != 0, later = P.tlater[c] != 0, leaf = P.tleaf[c] != 0;
            // no earlier time than 0, no later one than the largest t'
            if ((!later && t == 0) || (later && t == 0xFFFFFFFFu)) { zero[0] = zero[1] = true; break; }
            const uint32_t *off = out ? g.out_off : g.in_off;
            const uint32_t *tarr = out ? g.out_t : g.in_t;
            const uint32_t *nbr = out ? g.out_nbr : g.in_nbr;
            const uint32_t beg = __ldg(off + z), end = __ldg(off + z + 1);
            const uint32_t base = ((side == 0) == out) ? gallop_back(tarr, beg, pos, t)
                                                       : __ldg((side == 0 ? g.out_xrank : g.in_xrank) + pos);
            // per-layer ranges [a[p], b[p]) with times in [lo[p], hi[p]]
            uint32_t a[2], b[2], lo[2], hi[2];
            if (later) {
                const uint64_t hu64 = (uint64_t)t + d;
                const uint32_t l0 = t + 1, hu = hu64 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)hu64;
                const uint32_t a0 = gallop_idx(tarr, base, end, l0);
                const uint32_t bu = gallop_idx(tarr, a0, end, (uint64_t)hu + 1);
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    lo[p] = l0;
                    hi[p] = hu < whi[p] ? hu : whi[p];
                    a[p] = a0;
                    b[p] = (zero[p] || hi[p] == hu) ? bu : lower_idx(tarr, a0, bu, (uint64_t)hi[p] + 1);
                    if (lo[p] > hi[p]) zero[p] = true;
                }
            } else {
                const uint32_t h0 = t - 1, lu = (uint64_t)t >= d ? (uint32_t)((uint64_t)t - d) : 0u;
                const uint32_t au = gallop_back(tarr, beg, base, lu);
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    hi[p] = h0;
                    lo[p] = lu > wlo[p] ? lu : wlo[p];
                    b[p] = base;
                    a[p] = (zero[p] || lo[p] == lu) ? au : lower_idx(tarr, au, base, lo[p]);
                    if (lo[p] > hi[p]) zero[p] = true;
                }
            }
            if (zero[0] && zero[1]) break;
            const ulonglong2 *Pd = leaf ? nullptr : pick_slot(cp.pd, P.tslot[c]);
            uint64_t excl[2] = {0, 0};
            // the union of the live layers' ranges
            uint32_t ua = 0xFFFFFFFFu, ub = 0;
#pragma unroll
            for (int p = 0; p < 2; ++p)
                if (!zero[p]) { ua = min(ua, a[p]); ub = max(ub, b[p]); }
            // an excluded entry x (other endpoint o) of the range: its weight,
            // in each layer whose range holds it
            auto add_excl = [&](uint32_t x) {
                ulonglong2 wx2 = make_ulonglong2(1, 1);
                if (!leaf) {
                    // the entry's weight: its prefix minus the previous entry's in
                    // the same (vertex, window) segment
                    const ulonglong2 px = __ldg(Pd + x);
                    const ulonglong2 pp = x > beg ? __ldg(Pd + x - 1) : make_ulonglong2(0, 0);
                    const uint32_t tp = x > beg ? __ldg(tarr + x - 1) : 0;
                    wx2.x = px.x - ((x > beg && tp >= wlo[0]) ? pp.x : 0);
                    wx2.y = px.y - ((x > beg && tp >= wlo[1]) ? pp.y : 0);
                }
#pragma unroll
                for (int p = 0; p < 2; ++p)
                    if (!zero[p] && x >= a[p] && x < b[p]) excl[p] += lane_of(wx2, p);
            };
            if (!P.c2) {
                // without Constraint 2 nothing is excluded
            } else if (ub <= ua || ub - ua <= kScanLimit) {
                // (reading four neighbours per 16-byte load measured no faster)
                for (uint32_t x = ua; x < ub; ++x)
                    if (__ldg(nbr + x) == o) add_excl(x);
            } else {
                // the excluded multi-edge list: z -> o for a child leaving z, o -> z
                // for one entering it
                const uint32_t pe = !P.c2 ? kNone : out ? pair_of(g, z, o) : pair_of(g, o, z);
                if (pe != kNone) {
                    const uint32_t xb = __ldg(g.pair_off + pe), xe = __ldg(g.pair_off + pe + 1);
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        if (zero[p]) continue;
                        const uint32_t ea = lower_idx(g.multi_t, xb, xe, lo[p]);
                        const uint32_t eb = gallop_idx(g.multi_t, ea, xe, (uint64_t)hi[p] + 1);
                        if (eb <= ea) continue;
                        if (leaf) {
                            excl[p] = eb - ea;
                        } else {
                            const ulonglong2 *Pm = pick_slot(cp.pm, P.tslot[c]);
                            const uint64_t bs = (ea > xb && __ldg(g.multi_t + ea - 1) >= wlo[p])
                                                    ? lane_of(__ldg(Pm + ea - 1), p) : 0;
                            excl[p] = lane_of(__ldg(Pm + eb - 1), p) - bs;
                        }
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                if (zero[p]) continue;
                uint64_t sum;
                if (leaf) {
                    sum = (uint64_t)(b[p] - a[p]) - excl[p];
                } else if (b[p] > a[p]) {
                    const uint64_t top = lane_of(__ldg(Pd + b[p] - 1), p);
                    const uint64_t pbase = (a[p] > beg && __ldg(tarr + a[p] - 1) >= wlo[p])
                                               ? lane_of(__ldg(Pd + a[p] - 1), p) : 0;
                    sum = top - pbase - excl[p];
                } else {
                    sum = 0;
                }
                if (sum == 0) zero[p] = true;
                else prod[p] = mul_chk(prod[p], sum, ovf[p]);
            }
        }
        // both layers, one store; at the position scatter[pos] when a map is given
        wout[scatter ? __ldg(scatter + pos) : pos] = make_ulonglong2(zero[0] ? 0 : prod[0], zero[1] ? 0 : prod[1]);
        pend_bits = ((!zero[0] && ovf[0]) ? 1u : 0u) | ((!zero[1] && ovf[1]) ? 2u : 0u);
        if (last && pend_bits) latch(status, ST_OVERFLOW);
    }
    if (!last) {   // side 0: the warp's pending bits, one word per layer
        const uint32_t b0 = __ballot_sync(0xffffffffu, pend_bits & 1u);
        const uint32_t b1 = __ballot_sync(0xffffffffu, (pend_bits >> 1) & 1u);
        if ((threadIdx.x & 31) == 0) {
            const uint32_t words = (g.m + 31) >> 5;
            pout[pos >> 5] = b0;
            pout[words + (pos >> 5)] = b1;
        }
    }
}

// ---- scans over the three orders ----------------------------------------
// segment = (owner, window of layer p); owner boundaries come from a bit set.
// Whether the windows of layer p differ between two times.
__device__ __forceinline__ uint32_t win_change(const WinDiv &wv, uint32_t ta, uint32_t tb)
{
    const uint32_t qa = wv.quot(ta), qb = wv.quot(tb);
    return (WinDiv::win_of(qa, 0) != WinDiv::win_of(qb, 0) ? 1u : 0u) |
           (WinDiv::win_of(qa, 1) != WinDiv::win_of(qb, 1) ? 2u : 0u);
}

// Segment heads of one layer (exports rebuild weights from prefix sums).
struct DirHead {
    const uint32_t *tarr;       // position -> t'
    const uint32_t *ownbits;    // bit set: position starts a new owner
    int p;
    WinDiv wv;
    __device__ bool head(uint64_t i) const
    {
        if (i == 0) return true;
        if ((__ldg(ownbits + (i >> 5)) >> (i & 31)) & 1u) return true;
        return (win_change(wv, __ldg(tarr + i), __ldg(tarr + i - 1)) >> p) & 1u;
    }
};

struct RootHead {
    const uint32_t *tarr;       // g_t
    int p;
    WinDiv wv;
    __device__ bool head(uint64_t i) const
    {
        if (i == 0) return true;
        return (win_change(wv, __ldg(tarr + i), __ldg(tarr + i - 1)) >> p) & 1u;
    }
};

// Both layers at once (two-lane scans): the pair of weights of a position is
// one 16-byte gather; heads are per layer (bit p).
struct DirScan2 {
    static constexpr bool kGathered = true;
    const ulonglong2 *w;        // (layer 0, layer 1) weights
    const uint32_t *perm;       // scan position -> weight position (null: same order)
    const uint32_t *tarr;       // position -> t'
    const uint32_t *ownbits;    // bit set: position starts a new owner
    WinDiv wv;
    __device__ ulonglong2 value2(uint64_t i) const { return __ldg(w + (perm ? __ldg(perm + i) : i)); }
    __device__ uint32_t head2(uint64_t i) const
    {
        if (i == 0 || ((__ldg(ownbits + (i >> 5)) >> (i & 31)) & 1u)) return 3u;
        return win_change(wv, __ldg(tarr + i), __ldg(tarr + i - 1));
    }
};

struct RootScan2 {
    static constexpr bool kGathered = true;
    const ulonglong2 *w;        // root weight pairs in list order
    const uint32_t *tarr;       // g_t
    WinDiv wv;
    const uint32_t *perm;       // gid -> weight position
    __device__ ulonglong2 value2(uint64_t i) const { return __ldg(w + (perm ? __ldg(perm + i) : i)); }
    __device__ uint32_t head2(uint64_t i) const
    {
        if (i == 0) return 3u;
        return win_change(wv, __ldg(tarr + i), __ldg(tarr + i - 1));
    }
};

// ---- windows of both layers (Constraint 3, Alg. 1) ------------------------
// A window of layer p starts at GLOBAL position i when t'_i lies in a window
// of layer p and t'_{i-1} does not lie in the same one.  Each thread takes
// kWinItems consecutive positions; tile = one block's positions.
constexpr int kWinItems = 8;
constexpr int kWinTile = TB * kWinItems;

// Head bits of position i (bit p: a window of layer p starts there) and the
// window indices of both layers.
__device__ __forceinline__ uint32_t win_heads_at(const uint32_t *__restrict__ t, uint32_t i, const WinDiv &wv,
                                                 int64_t &w0, int64_t &w1)
{
    const uint32_t q = wv.quot(__ldg(t + i));
    w0 = WinDiv::win_of(q, 0);
    w1 = WinDiv::win_of(q, 1);
    uint32_t h = (w0 >= 0 ? 1u : 0u) | (w1 >= 0 ? 2u : 0u);
    if (i > 0) h &= win_change(wv, __ldg(t + i), __ldg(t + i - 1));
    return h;
}

// Per tile: the number of window starts of each layer (counts[tile] for
// layer 0, counts[ntile + tile] for layer 1).
__global__ void __launch_bounds__(TB) k_win_count(const uint32_t *__restrict__ t, uint32_t m, WinDiv wv, uint32_t ntile,
                                                  uint32_t *__restrict__ counts)
{
    __shared__ uint32_t s0[TB / 32], s1[TB / 32];
    const uint32_t base = blockIdx.x * (uint32_t)kWinTile + threadIdx.x * kWinItems;
    uint32_t c0 = 0, c1 = 0;
#pragma unroll
    for (int j = 0; j < kWinItems; ++j) {
        const uint32_t i = base + j;
        if (i >= m) break;
        int64_t w0, w1;
        const uint32_t h = win_heads_at(t, i, wv, w0, w1);
        c0 += h & 1u;
        c1 += h >> 1;
    }
    for (int o = 16; o > 0; o >>= 1) {
        c0 += __shfl_down_sync(0xffffffffu, c0, o);
        c1 += __shfl_down_sync(0xffffffffu, c1, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { s0[warp] = c0; s1[warp] = c1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t a = 0, b = 0;
        for (int w = 0; w < TB / 32; ++w) { a += s0[w]; b += s1[w]; }
        counts[blockIdx.x] = a;
        counts[ntile + blockIdx.x] = b;
    }
}

struct WinOut {
    uint32_t *beg[2], *id[2];
    uint32_t nwin[2];
};

// The windows' first positions and indices, written at the tile's scanned
// offsets (offs[tile] for layer 0, offs[ntile + tile] - nw0 for layer 1),
// plus the end sentinels beg[nwin] = m.
__global__ void __launch_bounds__(TB) k_win_fill(const uint32_t *__restrict__ t, uint32_t m, WinDiv wv, uint32_t ntile,
                                                 const uint32_t *__restrict__ offs, WinOut W)
{
    __shared__ uint32_t s0[TB / 32], s1[TB / 32];
    const uint32_t base = blockIdx.x * (uint32_t)kWinTile + threadIdx.x * kWinItems;
    uint32_t hb = 0, c0 = 0, c1 = 0;
#pragma unroll
    for (int j = 0; j < kWinItems; ++j) {
        const uint32_t i = base + j;
        if (i >= m) break;
        int64_t w0, w1;
        const uint32_t h = win_heads_at(t, i, wv, w0, w1);
        hb |= h << (2 * j);
        c0 += h & 1u;
        c1 += h >> 1;
    }
    // exclusive ranks of this thread's starts inside the tile, per layer
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t i0 = c0, i1 = c1;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y0 = __shfl_up_sync(0xffffffffu, i0, o), y1 = __shfl_up_sync(0xffffffffu, i1, o);
        if (lane >= o) { i0 += y0; i1 += y1; }
    }
    if (lane == 31) { s0[warp] = i0; s1[warp] = i1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t r0 = 0, r1 = 0;
        for (int w = 0; w < TB / 32; ++w) {
            const uint32_t a = s0[w], b = s1[w];
            s0[w] = r0; s1[w] = r1;
            r0 += a; r1 += b;
        }
    }
    __syncthreads();
    uint32_t k0 = offs[blockIdx.x] + s0[warp] + i0 - c0;
    uint32_t k1 = offs[ntile + blockIdx.x] - W.nwin[0] + s1[warp] + i1 - c1;
#pragma unroll
    for (int j = 0; j < kWinItems; ++j) {
        const uint32_t h = (hb >> (2 * j)) & 3u;
        if (!h) continue;
        const uint32_t i = base + j;
        const uint32_t q = wv.quot(__ldg(t + i));
        if (h & 1u) { W.beg[0][k0] = i; W.id[0][k0] = (uint32_t)WinDiv::win_of(q, 0); ++k0; }
        if (h & 2u) { W.beg[1][k1] = i; W.id[1][k1] = (uint32_t)WinDiv::win_of(q, 1); ++k1; }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        W.beg[0][W.nwin[0]] = m;
        W.beg[1][W.nwin[1]] = m;
    }
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

// Guide table of the window pick: entry j is the window holding draw j 2^s
// (the last k with wcum[k] <= j 2^s), for the ceil(W / 2^s) buckets, then a
// sentinel (the last window).  One thread per bucket, a binary search each;
// W is read on the device (the last cumulative entry).
__global__ void k_wguide(const uint64_t *__restrict__ wcum, uint32_t nw, uint32_t *__restrict__ guide)
{
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    const u128 W = (u128)wcum[2 * (size_t)nw] | ((u128)wcum[2 * (size_t)nw + 1] << 64);
    if (W == 0) return;
    const uint32_t s = wguide_shift((uint64_t)W, (uint64_t)(W >> 64), nw);
    const uint64_t nb = (uint64_t)((W + ((u128)1 << s) - 1) >> s);
    if (j > nb) return;
    if (j == nb) { guide[j] = nw - 1; return; }
    const u128 x = (u128)j << s;
    uint32_t lo = 0, hi = nw;   // wcum[0] = 0 <= x; find the last k with wcum[k] <= x
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        const u128 c = (u128)wcum[2 * (size_t)mid] | ((u128)wcum[2 * (size_t)mid + 1] << 64);
        if (c <= x) lo = mid; else hi = mid;
    }
    guide[j] = lo;
}

// ---- guide table of the root search --------------------------------------
// Window kk of a layer gets about n/4 buckets of width 2^s over its draws
// [0, W_kk); the table holds, per bucket j, the first edge whose in-window
// CDF exceeds j 2^s, then the window's last edge.  count[kk] = buckets + 1.
__device__ __forceinline__ uint64_t ceil_shift(uint64_t c, uint32_t s) { return (c >> s) + ((c & ((1ull << s) - 1)) != 0); }

struct GuideLayer {
    const uint64_t *cdf;
    const uint32_t *win_beg;
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

// Edges in GLOBAL order, kGuideItems consecutive ones per thread, layer p =
// blockIdx.y: the buckets whose lower bound falls in [cdf[x-1], cdf[x]) start
// at edge x.  A warp takes 32 x kGuideItems consecutive edges, lane l the
// edges l, l + 32, ... of them (coalesced CDF reads); the warp finds the
// window of its first edge by a binary search over the window starts, and a
// lane steps to the next window as its edges cross one, so a window of any
// size is spread over many threads.
#ifndef TM_GUIDE_ITEMS
#define TM_GUIDE_ITEMS 32   // measured: 32 edges per lane beat 8 (1.77 against 1.81 ms for the root phase) and 2
#endif
constexpr int kGuideItems = TM_GUIDE_ITEMS;
__global__ void __launch_bounds__(TB) k_guide_fill(GuideArgs A, uint32_t m)
{
    const int p = blockIdx.y;
    const GuideLayer &L = p ? A.L[1] : A.L[0];
    const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t xs = (gt >> 5) * (32u * kGuideItems) + (gt & 31u);
    if (xs >= m || L.nwin == 0) return;
    // kk = the last window starting at or before the warp's first edge x0
    // (none: x0 precedes every window); the same search in every lane, so
    // each probe is one broadcast load
    const uint32_t x0 = (uint32_t)(xs - (gt & 31u));
    uint32_t lo = 0, hi = L.nwin;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (L.win_beg[mid] <= x0) lo = mid + 1; else hi = mid;
    }
    int64_t kk = (int64_t)lo - 1;
    const uint64_t xe = min((uint64_t)m, (uint64_t)(xs + 32u * kGuideItems));
    // kGuideBatch edges' CDF pairs loaded before any is used (independent
    // loads in flight), then the edges in order
    constexpr int kGuideBatch = 4;
    for (uint64_t xb = xs; xb < xe; xb += 32u * kGuideBatch) {
        uint64_t c1v[kGuideBatch], c0v[kGuideBatch];
#pragma unroll
        for (int u = 0; u < kGuideBatch; ++u) {
            const uint64_t xx = xb + 32u * u;
            c1v[u] = xx < xe ? L.cdf[xx] : 0;
            c0v[u] = (xx < xe && xx > 0) ? L.cdf[xx - 1] : 0;
        }
#pragma unroll
        for (int u = 0; u < kGuideBatch; ++u) {
            const uint64_t xx = xb + 32u * u;
            if (xx >= xe) break;
            const uint32_t x = (uint32_t)xx;
            while (kk + 1 < (int64_t)L.nwin && L.win_beg[kk + 1] <= x) ++kk;
            if (kk < 0) continue;   // before the layer's first window
            const uint32_t wbeg = L.win_beg[kk], wend = L.win_beg[kk + 1];
            const uint32_t sh = L.gshift[kk];
            uint32_t *G = L.guide + L.goff[kk];
            const uint64_t c1 = c1v[u], c0 = x > wbeg ? c0v[u] : 0;
            const uint64_t j1 = ceil_shift(c1, sh);
            for (uint64_t j = ceil_shift(c0, sh); j < j1; ++j) G[j] = x;
            if (x == wend - 1) G[j1] = x;
        }
    }
}

// Reconstruct w for one order from its segmented prefix (exports); the
// prefix of position i is pref[i * stride].
template <class F>
__global__ void k_unprefix(F f, const uint64_t *__restrict__ pref, int stride, const uint32_t *__restrict__ perm,
                           uint32_t m, uint64_t *__restrict__ out)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    uint64_t w = pref[(size_t)i * stride] - (f.head(i) ? 0 : pref[(size_t)(i - 1) * stride]);
    out[perm ? perm[i] : i] = w;
}

__global__ void k_leaf_weights(const uint32_t *__restrict__ t, uint32_t m, int p, WinDiv wv, uint64_t *__restrict__ out)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) out[i] = wv.win(t[i], p) >= 0 ? 1 : 0;
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
    for (int sl = 0; sl < kMaxTree; ++sl) mo->pref_dir[sl] = mo->pref_multi[sl] = nullptr;
    mo->wcum = nullptr;
    mo->wguide = nullptr;
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
    const WinDiv wv = make_windiv(P.wdelta);   // window unit (delta, or one window without Constraint 3)
    int rc = TM_OK;
    cudaMemsetAsync(ctx->status, 0, 4, st);
    // ---- windows of each layer (K2): per tile the window starts of both
    // layers, one scan over the tile counts, then one block for everything
    // the motif keeps (windows, root CDF, prefix arrays, totals)
    const uint32_t ntile = m ? (m + kWinTile - 1) / kWinTile : 0;
    uint32_t *wcount = nullptr, *woffs = nullptr;
    uint32_t nwh[2] = {0, 0};
    {
        PhaseScope ph(ctx, TM_PH_WINDOWS);
        wcount = (uint32_t *)salloc(ctx, ((size_t)2 * ntile + 1) * 4);
        woffs = (uint32_t *)salloc(ctx, ((size_t)2 * ntile + 2) * 4);
        if (!wcount || !woffs) return TM_E_NOMEM;
        if (m) {
            launch(ctx, k_win_count, ntile, TB, g.g_t, m, wv, ntile, wcount);
            rc = exclusive_scan_u32(ctx, wcount, woffs, 2 * (uint64_t)ntile, woffs + 2 * (size_t)ntile);
            if (rc) return rc;
            uint32_t both[2] = {0, 0};
            copy_d2h(ctx, &both[0], woffs + ntile, 4);                  // layer 0's windows
            copy_d2h(ctx, &both[1], woffs + 2 * (size_t)ntile, 4);      // all windows
            rc = check_cuda(ctx, cudaStreamSynchronize(st), "window count");
            if (rc) return rc;
            nwh[0] = both[0];
            nwh[1] = both[1] - both[0];
        }
    }
    {
        auto al = [](size_t b) { return (b + 255) / 256 * 256; };
        const size_t mm = (size_t)(m ? m : 1);
        auto guide_n = [&](uint32_t nw) { return (size_t)m / 4 + 3 * (size_t)nw + 1; };
        size_t total = al(((size_t)nwh[0] + 1) * 4) * 4 + al(((size_t)nwh[1] + 1) * 4) * 4 + 2 * al(mm * 8) +
                       (size_t)P.nslots * 2 * al(mm * 16) + al(((size_t)nwh[0] + nwh[1] + 1) * 16) +
                       al(guide_n(nwh[0]) * 4) + al(guide_n(nwh[1]) * 4) + al((4 * ((size_t)nwh[0] + nwh[1]) + 2) * 4);
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
        }
        for (int sl = 0; sl < P.nslots; ++sl) {
            mo->pref_dir[sl] = (ulonglong2 *)take(mm * 16);
            mo->pref_multi[sl] = (ulonglong2 *)take(mm * 16);
        }
        mo->wcum = (uint64_t *)take(((size_t)nwh[0] + nwh[1] + 1) * 16);
        mo->wguide = (uint32_t *)take((4 * ((size_t)nwh[0] + nwh[1]) + 2) * 4);
    }
    {
        PhaseScope ph(ctx, TM_PH_WINDOWS);
        WinOut wo{{mo->layer[0].win_beg, mo->layer[1].win_beg}, {mo->layer[0].win_id, mo->layer[1].win_id},
                  {nwh[0], nwh[1]}};
        if (m) launch(ctx, k_win_fill, ntile, TB, g.g_t, m, wv, ntile, (const uint32_t *)woffs, wo);
        else {
            cudaMemsetAsync(mo->layer[0].win_beg, 0, 4, st);
            cudaMemsetAsync(mo->layer[1].win_beg, 0, 4, st);
        }
    }
    // ---- DP over tree nodes in increasing height (K3) + prefixes (K4)
    const OwnerBits ob{g.own_out, g.own_in, g.own_multi};
    ulonglong2 *w = nullptr, *pw = nullptr;   // (layer 0, layer 1) weight pairs
    uint32_t *pend = nullptr;                 // per layer a bit set: pending overflow of a side-0 partial
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
                pend = (uint32_t *)salloc(ctx, ((size_t)m / 32 + 1) * 8);
                if (!pw || !pend) return TM_E_NOMEM;
            }
            if (m) {
                if (has[0] && has[1]) {
                    launch(ctx, k_dp, blocks_for(m, TB), TB, g, P, wv, q, 0, 1, 0, cp, pw, (const uint32_t *)nullptr,
                           (const ulonglong2 *)nullptr, (const uint32_t *)nullptr, pend, ctx->status);
                    launch(ctx, k_dp, blocks_for(m, TB), TB, g, P, wv, q, 1, 0, 1, cp, w, (const uint32_t *)nullptr,
                           (const ulonglong2 *)pw, (const uint32_t *)pend, (uint32_t *)nullptr, ctx->status);
                } else {
                    // a non-root node leaving its parent's meeting vertex runs in
                    // in-list order and is scanned by its parent in out-list
                    // order: it writes through the in -> out map
                    const bool to_out = q != 0 && P.tout[q] != 0 && in_order;
                    launch(ctx, k_dp, blocks_for(m, TB), TB, g, P, wv, q, in_order ? 1 : 0, 1, 1, cp, w,
                           to_out ? (const uint32_t *)g.in_to_out : (const uint32_t *)nullptr,
                           (const ulonglong2 *)nullptr, (const uint32_t *)nullptr, (uint32_t *)nullptr, ctx->status);
                }
            }
        }
        rc = check_cuda(ctx, cudaGetLastError(), "weight DP");
        if (rc) return rc;
        if (q == 0) {
            PhaseScope ph(ctx, TM_PH_ROOT);
            GuideArgs ga{};
            RootScan2 f{w, g.g_t, wv, in_order ? g.in_pos : g.out_pos};
            rc = segmented_scan2_u64(ctx, f, m, mo->layer[0].root_cdf, mo->layer[1].root_cdf);
            if (rc) return rc;
            for (int p = 0; p < 2; ++p) {
                LayerData &L = mo->layer[p];
                ga.L[p] = GuideLayer{L.root_cdf, L.win_beg, L.nwin, L.win_gshift, L.win_goff, L.guide};
            }
            // guide tables of the root search, both layers (edge-parallel)
            if (m && nwh[0] + nwh[1]) {
                launch(ctx, k_guide_setup, 2, 1024, ga);
                const uint64_t gwarps = ((uint64_t)m + 32 * kGuideItems - 1) / (32 * kGuideItems);
                launch(ctx, k_guide_fill, dim3(blocks_for(gwarps * 32, TB), 2), TB, ga, m);
            }
        } else {
            PhaseScope ph(ctx, TM_PH_PREFIX);
            const int slot = P.tslot[q];
            const bool out = P.tout[q] != 0;
            // A non-root node's DP runs in the list order of its far endpoint,
            // never in the order its parent scans (out-list order when the node
            // leaves the meeting vertex, in-list order when it enters it).  A
            // node leaving it wrote its weights through the in -> out map, so
            // they are in out-list order already; for a node entering it the
            // in-list order is one gather through the same map.  Multi-edge
            // lists are grouped by source like the out-lists, so the multi-edge
            // prefix gathers, within each source's run, from the weights in
            // out-list order (w in both cases).
            DirScan2 fd{w, out ? nullptr : g.in_to_out, out ? g.out_t : g.in_t, out ? ob.out : ob.in, wv};
            rc = segmented_scan2_u64(ctx, fd, m, nullptr, nullptr, mo->pref_dir[slot]);
            if (rc) return rc;
            DirScan2 fm{w, g.multi_to_out, g.multi_t, ob.multi, wv};
            rc = segmented_scan2_u64(ctx, fm, m, nullptr, nullptr, mo->pref_multi[slot]);
            if (rc) return rc;
            cp.pd[slot] = mo->pref_dir[slot];
            cp.pm[slot] = mo->pref_multi[slot];
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
        if (mo->nwtot)
            launch(ctx, k_wguide, blocks_for(4 * (uint64_t)mo->nwtot + 1, TB), TB, (const uint64_t *)mo->wcum,
                   mo->nwtot, mo->wguide);
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
    const WinDiv wv = make_windiv(P.wdelta);
    int rc = TM_OK;
    if (P.tleaf[q] && q != 0) {
        launch(ctx, k_leaf_weights, blocks_for(m, TB), TB, g.g_t, m, layer, wv, out);
    } else if (q == 0) {
        RootHead f{g.g_t, layer, wv};
        launch(ctx, k_unprefix<RootHead>, blocks_for(m, TB), TB, f, (const uint64_t *)mo->layer[layer].root_cdf, 1,
               (const uint32_t *)nullptr, m, out);
    } else {
        const OwnerBits ob{g.own_out, g.own_in, g.own_multi};
        bool o = P.tout[q] != 0;
        DirHead f{o ? g.out_t : g.in_t, o ? ob.out : ob.in, layer, wv};
        launch(ctx, k_unprefix<DirHead>, blocks_for(m, TB), TB, f,
               (const uint64_t *)mo->pref_dir[P.tslot[q]] + layer, 2, (const uint32_t *)(o ? g.out_gid : g.in_gid),
               m, out);
        rc = check_cuda(ctx, cudaStreamSynchronize(st), "export");
    }
    copy_d2h(ctx, host_out, out, (size_t)m * 8);
    int rc2 = check_cuda(ctx, cudaStreamSynchronize(st), "export copy");
    return rc ? rc : rc2;
}

void release_weights(tm_ctx *ctx, tm_motif *mo) { free_motif_weights(ctx, mo); }

}  // namespace timest
