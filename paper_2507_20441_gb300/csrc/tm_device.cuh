// Device helpers: counter-based random numbers, bounded binary searches,
// 128-bit arithmetic and the status word.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tm_internal.h"

namespace timest {

typedef unsigned __int128 u128;

__device__ __forceinline__ void latch(uint32_t *status, uint32_t bits)
{
    atomicOr(status, bits);
}

// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): each round
// multiplies counter words 0 and 2 by the two round multipliers, feeds the
// high halves (xored with words 1/3 and the key) and the low halves forward;
// the key advances by the golden-ratio Weyl increments between rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t hi0 = __umulhi(m0, c.x), lo0 = m0 * c.x;
        uint32_t hi1 = __umulhi(m1, c.z), lo1 = m1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Per-sample stream: key = seed, counter = (sample id, draw number, 0).
struct SampleRng {
    uint32_t k0, k1, j0, j1, d;
    __device__ void init(uint64_t seed, uint64_t j)
    {
        k0 = (uint32_t)seed; k1 = (uint32_t)(seed >> 32);
        j0 = (uint32_t)j; j1 = (uint32_t)(j >> 32); d = 0;
    }
    __device__ __forceinline__ uint4 block() { return philox10(make_uint4(j0, j1, d++, 0u), k0, k1); }

    // U[0,n) by masked rejection; n <= 1 consumes no draw.
    __device__ uint64_t below(uint64_t n, uint32_t *status)
    {
        if (n <= 1) return 0;
        int b = 64 - __clzll((long long)(n - 1));
        uint64_t mask = (b >= 64) ? ~0ull : ((1ull << b) - 1);
        for (int it = 0; it < 512; ++it) {
            uint4 x = block();
            uint64_t v = ((uint64_t)x.x | ((uint64_t)x.y << 32)) & mask;
            if (v < n) return v;
        }
        latch(status, ST_BADSTATE);
        return 0;
    }
    __device__ u128 below128(u128 n, uint32_t *status)
    {
        if (n <= 1) return 0;
        u128 nm1 = n - 1;
        uint64_t hi = (uint64_t)(nm1 >> 64);
        int b = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)(uint64_t)nm1);
        u128 mask = (b >= 128) ? ~(u128)0 : ((((u128)1) << b) - 1);
        for (int it = 0; it < 512; ++it) {
            uint4 x = block();
            u128 v = (u128)x.x | ((u128)x.y << 32) | ((u128)x.z << 64) | ((u128)x.w << 96);
            v &= mask;
            if (v < n) return v;
        }
        latch(status, ST_BADSTATE);
        return 0;
    }
};

// First index in [lo, hi) with a[i] >= x (a sorted ascending); hi if none.
__device__ __forceinline__ uint32_t lower_idx(const uint32_t *__restrict__ a, uint32_t lo, uint32_t hi, uint64_t x)
{
    uint32_t n = hi - lo;
    while (n > 0) {
        uint32_t half = n >> 1;
        uint32_t mid = lo + half;
        if ((uint64_t)__ldg(a + mid) < x) { lo = mid + 1; n -= half + 1; }
        else n = half;
    }
    return lo;
}

// Same result as lower_idx, searching outward from lo first (1, 2, 4, ...
// entries ahead): cheaper when the answer is close to lo.
__device__ __forceinline__ uint32_t gallop_idx(const uint32_t *__restrict__ a, uint32_t lo, uint32_t hi, uint64_t x)
{
    // invariant: every index below `lo` holds a value < x
    uint32_t step = 1;
    uint32_t probe = lo;
    while (probe < hi && (uint64_t)__ldg(a + probe) < x) {
        lo = probe + 1;
        probe = (hi - probe > step) ? probe + step : hi;
        step = step < 0x40000000u ? step << 1 : step;
    }
    // the answer lies in [lo, probe]: probe == hi or a[probe] >= x
    return lower_idx(a, lo, probe, x);
}

// First index in [beg, base] with a[i] >= x, when every index >= base is
// known to hold a value >= x: searches backward from base (1, 2, 4, ...).
__device__ __forceinline__ uint32_t gallop_back(const uint32_t *__restrict__ a, uint32_t beg, uint32_t base, uint64_t x)
{
    uint32_t hi = base, step = 1;
    while (hi > beg) {
        const uint32_t probe = (hi - beg > step) ? hi - step : beg;
        if ((uint64_t)__ldg(a + probe) < x) return lower_idx(a, probe + 1, hi, x);
        hi = probe;
        step = step < 0x40000000u ? step << 1 : step;
    }
    return beg;
}

// Candidate range [a, b) of a child edge at vertex z (Claim 3.1): the entries
// of z's out-list (out_c) or in-list with times in [lo, hi], found from the
// parent edge's own position `pos` in z's out-list (side 0) or in-list
// (side 1) and its time t.  The first entry with time >= t is reached from
// `pos` (same list) or from the precomputed cross rank (other list); the
// bounds are then galloped to from there.  A later child has lo > t, an
// earlier one hi = t - 1.
__device__ __forceinline__ void child_range(const DevGraph &g, int side, bool out_c, uint32_t z, uint32_t pos,
                                            uint32_t t, bool later, uint64_t lo, uint64_t hi, uint32_t &a,
                                            uint32_t &b, uint32_t &beg, const uint32_t *&tarr)
{
    const uint32_t *off = out_c ? g.out_off : g.in_off;
    tarr = out_c ? g.out_t : g.in_t;
    beg = __ldg(off + z);
    const uint32_t end = __ldg(off + z + 1);
    uint32_t base;
    if ((side == 0) == out_c) base = gallop_back(tarr, beg, pos, t);
    else base = __ldg((side == 0 ? g.out_xrank : g.in_xrank) + pos);
    if (later) {
        a = gallop_idx(tarr, base, end, lo);
        b = gallop_idx(tarr, a, end, hi + 1);
    } else {
        b = base;
        a = gallop_back(tarr, beg, base, lo);
    }
}

// The pair (multi-edge list) id of (u, v), or kNone when no edge u -> v exists:
// a search of u's pairs, which are sorted by destination.
__device__ __forceinline__ uint32_t pair_of(const DevGraph &g, uint32_t u, uint32_t v)
{
    const uint32_t lo = __ldg(g.vpair_off + u), hi = __ldg(g.vpair_off + u + 1);
    const uint32_t p = lower_idx(g.pair_dst, lo, hi, v);
    return (p < hi && __ldg(g.pair_dst + p) == v) ? p : kNone;
}

// ---- warp-cooperative search ----------------------------------------------
// A lane whose search range holds at least coop_min entries is served by all
// active lanes of its warp together: with n lanes, each step probes n evenly
// spaced positions at once and a ballot keeps the bracket between the last
// false and the first true probe, so the range shrinks (n + 1)-fold per step
// instead of 2-fold.  Lanes with long ranges are served one after the other;
// the others search alone.  Probe(x) must be monotone (false ... true) on
// the range; the result is the first x in [lo, hi) with Probe(x), else hi.
struct ProbeGtU64S2 {            // v[2x] > key (a lane of interleaved prefix pairs)
    const uint64_t *v;
    uint64_t key;
    __device__ __forceinline__ bool operator()(uint32_t x) const { return __ldg(v + 2 * (size_t)x) > key; }
    __device__ __forceinline__ ProbeGtU64S2 bcast(unsigned mask, int src) const
    {
        return ProbeGtU64S2{(const uint64_t *)__shfl_sync(mask, (unsigned long long)v, src),
                            __shfl_sync(mask, (unsigned long long)key, src)};
    }
};
struct ProbeGeU32 {              // a[x] >= key
    const uint32_t *a;
    uint32_t key;
    __device__ __forceinline__ bool operator()(uint32_t x) const { return __ldg(a + x) >= key; }
    __device__ __forceinline__ ProbeGeU32 bcast(unsigned mask, int src) const
    {
        return ProbeGeU32{(const uint32_t *)__shfl_sync(mask, (unsigned long long)a, src), __shfl_sync(mask, key, src)};
    }
};

template <class Probe>
__device__ __forceinline__ uint32_t first_true_serial(const Probe &pr, uint32_t lo, uint32_t hi)
{
    uint32_t n = hi - lo;
    while (n > 0) {
        const uint32_t half = n >> 1, mid = lo + half;
        if (!pr(mid)) { lo = mid + 1; n -= half + 1; }
        else n = half;
    }
    return lo;
}

template <class Probe>
__device__ uint32_t first_true_coop(const Probe &pr, uint32_t lo, uint32_t hi, uint32_t coop_min)
{
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    const bool mine = hi - lo >= coop_min;
    unsigned todo = __ballot_sync(act, mine);
    uint32_t res = hi;
    if (todo) {
        const uint32_t n = (uint32_t)__popc(act);
        const uint32_t rank = (uint32_t)__popc(act & ((1u << lane) - 1u));
        const int last = 31 - __clz((int)act);
        while (todo) {
            const int leader = __ffs((int)todo) - 1;
            todo &= todo - 1u;
            const Probe q = pr.bcast(act, leader);
            uint32_t l = __shfl_sync(act, lo, leader), h = __shfl_sync(act, hi, leader);
            // invariant: Probe false below l, true from h on (h = the range end if none)
            while (h - l > n) {
                const uint32_t pp = l + (uint32_t)(((uint64_t)(rank + 1u) * (h - l)) / (uint64_t)(n + 1u));
                const unsigned b = __ballot_sync(act, q(pp));
                if (b) {
                    const int fl = __ffs((int)b) - 1;
                    const unsigned below = act & ((1u << fl) - 1u);
                    const int pl = below ? 31 - __clz((int)below) : fl;
                    const uint32_t pf = __shfl_sync(act, pp, fl), pb = __shfl_sync(act, pp, pl);
                    h = pf;
                    if (below) l = pb + 1u;
                } else {
                    l = __shfl_sync(act, pp, last) + 1u;
                }
            }
            const uint32_t x = l + rank;   // at most n candidates left: one probe each
            const unsigned b = __ballot_sync(act, x < h && q(x));
            const uint32_t a = b ? l + (uint32_t)__popc(act & ((1u << (__ffs((int)b) - 1)) - 1u)) : h;
            if (lane == leader) res = a;
        }
    }
    if (!mine) res = first_true_serial(pr, lo, hi);
    return res;
}

// First index in [lo, hi) with v[i] > x (v non-decreasing).
__device__ __forceinline__ uint32_t upper_idx64(const uint64_t *__restrict__ v, uint32_t lo, uint32_t hi, uint64_t x)
{
    uint32_t n = hi - lo;
    while (n > 0) {
        uint32_t half = n >> 1;
        uint32_t mid = lo + half;
        if (__ldg(v + mid) <= x) { lo = mid + 1; n -= half + 1; }
        else n = half;
    }
    return lo;
}

// Checked u64 add / multiply.
__device__ __forceinline__ uint64_t add_chk(uint64_t a, uint64_t b, bool &ovf)
{
    uint64_t s = a + b;
    ovf |= (s < a);
    return s;
}
__device__ __forceinline__ uint64_t mul_chk(uint64_t a, uint64_t b, bool &ovf)
{
    ovf |= (__umul64hi(a, b) != 0);
    return a * b;
}

// Window of layer p holding t' (windows [i*d, (i+2)*d), i = p mod 2), or -1.
__device__ __forceinline__ int64_t layer_window(uint32_t t, int p, int64_t d)
{
    int64_t tt = (int64_t)t;
    if (tt < p * d) return -1;
    return p + 2 * ((tt - p * d) / (2 * d));
}

}  // namespace timest
