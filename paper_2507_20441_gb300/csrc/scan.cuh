// Device-wide scans used by the CSR builder and the weight pass.
//
// * exclusive_scan_u32: reduce-then-scan over u32 counts (recursive over the
//   tile totals), for radix-sort offsets and compaction.
// * segmented_scan_u64: inclusive prefix sums that restart at segment heads,
//   with every 64-bit addition inside a segment checked for wrap-around.  It
//   is a three-phase reduce / scan-of-tile-aggregates / rescan, so no block
//   ever waits on another block.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tm_device.cuh"
#include "tm_internal.h"

namespace timest {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// ---------------------------------------------------------------- u32 ----
__global__ void k_tile_sum_u32(const uint32_t *__restrict__ in, uint64_t n, uint32_t *__restrict__ tile_sum)
{
    __shared__ uint32_t warp_sum[SCAN_THREADS / 32];
    uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        uint64_t i = base + (uint64_t)j * SCAN_THREADS + threadIdx.x;
        if (i < n) s += in[i];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t v = threadIdx.x < SCAN_THREADS / 32 ? warp_sum[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) tile_sum[blockIdx.x] = v;
    }
}

// Exclusive scan of one tile with a carry-in taken from carry[blockIdx.x]
// (or 0 when carry is null); blocked layout (each thread SCAN_ITEMS
// consecutive values).  Writes the grand total to *total when it is the last
// tile and total is non-null.
// With tile_sums non-null the carry-in is instead the sum of the unscanned
// tile totals tile_sums[0 .. blockIdx.x), added up by the block itself.
__global__ void k_tile_scan_u32(const uint32_t *__restrict__ in, uint64_t n, const uint32_t *__restrict__ carry,
                                uint32_t *__restrict__ out, uint32_t *__restrict__ total,
                                const uint32_t *__restrict__ tile_sums = nullptr)
{
    __shared__ uint32_t warp_tot[SCAN_THREADS / 32];
    __shared__ uint32_t s_carry;
    if (tile_sums) {
        uint32_t c = 0;
        for (uint32_t i = threadIdx.x; i < blockIdx.x; i += SCAN_THREADS) c += tile_sums[i];
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w = 0; w < SCAN_THREADS / 32; ++w) t += warp_tot[w];
            s_carry = t;
        }
        __syncthreads();
    }
    uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        uint64_t i = base + j;
        v[j] = (i < n) ? in[i] : 0;
        s += v[j];
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < SCAN_THREADS / 32 ? warp_tot[lane] : 0;
        uint32_t wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = wi - w;
    }
    __syncthreads();
    uint32_t run = (tile_sums ? s_carry : carry ? carry[blockIdx.x] : 0) + warp_tot[warp] + incl - s;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        uint64_t i = base + j;
        if (i < n) out[i] = run;
        run += v[j];
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) *total = run;
}

// Exclusive scan of n u32 values (in may equal out).  If total is non-null
// the grand total is written there (device pointer).
inline int exclusive_scan_u32(tm_ctx *ctx, const uint32_t *in, uint32_t *out, uint64_t n, uint32_t *total)
{
    if (n == 0) {
        if (total) cudaMemsetAsync(total, 0, sizeof(uint32_t), ctx->stream);
        return TM_OK;
    }
    uint64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 1) {
        launch(ctx, k_tile_scan_u32, 1, SCAN_THREADS, in, n, (const uint32_t *)nullptr, out, total,
               (const uint32_t *)nullptr);
        return check_cuda(ctx, cudaGetLastError(), "scan");
    }
    ScratchScope scope(ctx);
    uint32_t *ts = (uint32_t *)salloc(ctx, tiles * sizeof(uint32_t));
    if (!ts) return TM_E_NOMEM;
    launch(ctx, k_tile_sum_u32, (unsigned)tiles, SCAN_THREADS, in, n, ts);
    if (tiles <= 4096) {   // each block adds up the totals before it: two launches in all
        launch(ctx, k_tile_scan_u32, (unsigned)tiles, SCAN_THREADS, in, n, (const uint32_t *)nullptr, out, total,
               (const uint32_t *)ts);
        return check_cuda(ctx, cudaGetLastError(), "scan");
    }
    int rc = exclusive_scan_u32(ctx, ts, ts, tiles, nullptr);
    if (rc == TM_OK) {
        launch(ctx, k_tile_scan_u32, (unsigned)tiles, SCAN_THREADS, in, n, (const uint32_t *)ts, out, total,
               (const uint32_t *)nullptr);
        rc = check_cuda(ctx, cudaGetLastError(), "scan");
    }
    return rc;
}

// ------------------------------------------ segmented u64, two layers ----
// Inclusive prefix sums that restart at segment heads, with every 64-bit
// addition inside a segment checked for wrap-around, over pairs (layer 0,
// layer 1) that share their positions (one gather of a 16-byte pair serves
// both layers).  Heads may differ per layer (bit p of head2()).  Functor
// interface: value2(pos) -> ulonglong2, head2(pos) -> bits, and
// kGathered (value2 is a gather).
struct SegAgg2 {
    uint64_t v0, v1;
    uint32_t f;     // bit p: the range contains a head of layer p
    uint32_t pad;
};

__device__ __forceinline__ SegAgg2 seg_combine2(SegAgg2 a, SegAgg2 b, bool &ovf)
{
    SegAgg2 r;
    r.f = a.f | b.f;
    r.v0 = (b.f & 1u) ? b.v0 : add_chk(a.v0, b.v0, ovf);
    r.v1 = (b.f & 2u) ? b.v1 : add_chk(a.v1, b.v1, ovf);
    r.pad = 0;
    return r;
}

__device__ __forceinline__ SegAgg2 seg_shfl_up2(SegAgg2 a, int o)
{
    SegAgg2 y;
    y.v0 = __shfl_up_sync(0xffffffffu, a.v0, o);
    y.v1 = __shfl_up_sync(0xffffffffu, a.v1, o);
    y.f = __shfl_up_sync(0xffffffffu, a.f, o);
    y.pad = 0;
    return y;
}

template <class F>
__global__ void k_segscan2_reduce(F f, uint64_t n, SegAgg2 *__restrict__ aggs, ulonglong2 *__restrict__ stash,
                                  uint32_t *status)
{
    __shared__ SegAgg2 warp_agg[SCAN_THREADS / 32];
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
    bool ovf = false;
    SegAgg2 a{0, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        const uint64_t i = base + j;
        if (i < n) {
            const ulonglong2 v = f.value2(i);
            if (stash) stash[i] = v;          // gathered once; the rescan reads it back in order
            SegAgg2 x{v.x, v.y, f.head2(i), 0};
            a = seg_combine2(a, x, ovf);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const SegAgg2 y = seg_shfl_up2(a, o);
        if (lane >= o) a = seg_combine2(y, a, ovf);
    }
    if (lane == 31) warp_agg[warp] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        SegAgg2 t = warp_agg[0];
        for (int w = 1; w < SCAN_THREADS / 32; ++w) t = seg_combine2(t, warp_agg[w], ovf);
        aggs[blockIdx.x] = t;
    }
    if (ovf) latch(status, ST_OVERFLOW);
}

__global__ void k_segscan2_carries(SegAgg2 *__restrict__ aggs, uint64_t ntiles, uint32_t *status)
{
    __shared__ SegAgg2 warp_tot[32];
    bool ovf = false;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t per = (ntiles + blockDim.x - 1) / blockDim.x;
    uint64_t lo = (uint64_t)threadIdx.x * per, hi = lo + per;
    if (hi > ntiles) hi = ntiles;
    if (lo > ntiles) lo = ntiles;
    SegAgg2 a{0, 0, 0, 0};
    for (uint64_t i = lo; i < hi; ++i) a = seg_combine2(a, aggs[i], ovf);
    SegAgg2 incl = a;
    for (int o = 1; o < 32; o <<= 1) {
        const SegAgg2 y = seg_shfl_up2(incl, o);
        if (lane >= o) incl = seg_combine2(y, incl, ovf);
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) / 32;
        const SegAgg2 w = lane < nw ? warp_tot[lane] : SegAgg2{0, 0, 0, 0};
        SegAgg2 wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const SegAgg2 y = seg_shfl_up2(wi, o);
            if (lane >= o) wi = seg_combine2(y, wi, ovf);
        }
        SegAgg2 ex = seg_shfl_up2(wi, 1);
        if (lane == 0) ex = SegAgg2{0, 0, 0, 0};
        if (lane < nw) warp_tot[lane] = ex;
    }
    __syncthreads();
    const SegAgg2 ex_lane = seg_shfl_up2(incl, 1);
    SegAgg2 run = warp_tot[warp];
    if (lane > 0) run = seg_combine2(run, ex_lane, ovf);
    for (uint64_t i = lo; i < hi; ++i) {
        const SegAgg2 c = aggs[i];
        aggs[i] = run;
        run = seg_combine2(run, c, ovf);
    }
    if (ovf) latch(status, ST_OVERFLOW);
}

#ifndef TM_SCAN2_MINB
#define TM_SCAN2_MINB 4   // four blocks of 256 per SM (measured faster than two)
#endif
template <class F>
__global__ void __launch_bounds__(SCAN_THREADS, TM_SCAN2_MINB) k_segscan2_final(F f, uint64_t n, const SegAgg2 *__restrict__ carries,
                                 const ulonglong2 *__restrict__ stash, uint64_t *__restrict__ out0,
                                 uint64_t *__restrict__ out1, ulonglong2 *__restrict__ outp, uint32_t *status)
{
    __shared__ SegAgg2 warp_agg[SCAN_THREADS / 32];
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
    bool ovf = false;
    ulonglong2 v[SCAN_ITEMS];
    uint32_t hbits = 0;
    SegAgg2 a{0, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        const uint64_t i = base + j;
        v[j] = make_ulonglong2(0, 0);
        if (i < n) {
            v[j] = stash ? stash[i] : f.value2(i);
            const uint32_t h = f.head2(i);
            hbits |= h << (2 * j);
            SegAgg2 x{v[j].x, v[j].y, h, 0};
            a = seg_combine2(a, x, ovf);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    SegAgg2 incl = a;
    for (int o = 1; o < 32; o <<= 1) {
        const SegAgg2 y = seg_shfl_up2(incl, o);
        if (lane >= o) incl = seg_combine2(y, incl, ovf);
    }
    if (lane == 31) warp_agg[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        SegAgg2 run = carries[blockIdx.x];
        for (int w = 0; w < SCAN_THREADS / 32; ++w) {
            const SegAgg2 c = warp_agg[w];
            warp_agg[w] = run;
            run = seg_combine2(run, c, ovf);
        }
    }
    __syncthreads();
    const SegAgg2 excl_lane = seg_shfl_up2(incl, 1);
    SegAgg2 pre = warp_agg[warp];
    if (lane > 0) pre = seg_combine2(pre, excl_lane, ovf);
    uint64_t r0 = pre.v0, r1 = pre.v1;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        const uint64_t i = base + j;
        if (i < n) {
            const uint32_t h = (hbits >> (2 * j)) & 3u;
            r0 = (h & 1u) ? v[j].x : add_chk(r0, v[j].x, ovf);
            r1 = (h & 2u) ? v[j].y : add_chk(r1, v[j].y, ovf);
            if (outp) {
                outp[i] = make_ulonglong2(r0, r1);
            } else {
                out0[i] = r0;
                out1[i] = r1;
            }
        }
    }
    if (ovf) latch(status, ST_OVERFLOW);
}

// ---- one pass with decoupled look-back -------------------------------
// Each block takes the next tile from a counter (so every tile before it has
// been started), scans it, publishes its aggregate, then its first warp walks
// back over the tiles before it, 32 at a time, combining their aggregates
// until it meets a published inclusive prefix or both layers have met a
// segment head (a head cuts the sums off), and publishes its own inclusive
// prefix.  Waits are bounded: a tile that does not publish within the limit
// latches ST_TIMEOUT.
struct SegTile {
    unsigned long long a0, a1, p0, p1;   // aggregate and inclusive prefix of both layers
    uint32_t af, pf;                     // their head bits
    uint32_t status;                     // 0 none, 1 aggregate, 2 inclusive prefix
    uint32_t pad;
};

constexpr int kLookbackPolls = 1 << 22;   // with a 64 ns sleep each: a limit of at least a quarter second

__device__ __forceinline__ void seg_publish(SegTile *t, const SegAgg2 &v, uint32_t st)
{
    volatile SegTile *vt = t;
    if (st == 1) { vt->a0 = v.v0; vt->a1 = v.v1; vt->af = v.f; }
    else { vt->p0 = v.v0; vt->p1 = v.v1; vt->pf = v.f; }
    __threadfence();
    vt->status = st;
}

// (Staging each tile through shared memory so that the global loads and
// stores are striped across lanes measured slower: 1.82 against 1.51 ms for
// the two list-order scans on 5e7 edges.)
#ifndef TM_SCAN_MINB
#define TM_SCAN_MINB 4   // 64 registers, four blocks per SM: measured 1.50 against 1.71 ms uncapped (76 registers)
#endif
template <class F>
__global__ void __launch_bounds__(SCAN_THREADS, TM_SCAN_MINB) k_segscan2_onepass(F f, uint64_t n, SegTile *__restrict__ tiles,
                                                                   uint32_t *__restrict__ counter,
                                                                   ulonglong2 *__restrict__ keep,
                                                                   uint64_t *__restrict__ out0,
                                                                   uint64_t *__restrict__ out1,
                                                                   ulonglong2 *__restrict__ outp, uint32_t *status)
{
    __shared__ SegAgg2 warp_agg[SCAN_THREADS / 32];
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t base = (uint64_t)tile * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
    bool ovf = false;
    ulonglong2 v[SCAN_ITEMS];
    uint32_t hbits = 0;
    SegAgg2 a{0, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        const uint64_t i = base + j;
        v[j] = make_ulonglong2(0, 0);
        if (i < n) {
            v[j] = f.value2(i);
            if (keep) keep[i] = v[j];
            const uint32_t h = f.head2(i);
            hbits |= h << (2 * j);
            SegAgg2 x{v[j].x, v[j].y, h, 0};
            a = seg_combine2(a, x, ovf);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    SegAgg2 incl = a;
    for (int o = 1; o < 32; o <<= 1) {
        const SegAgg2 y = seg_shfl_up2(incl, o);
        if (lane >= o) incl = seg_combine2(y, incl, ovf);
    }
    if (lane == 31) warp_agg[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        // the tile's aggregate (every lane of warp 0 folds the warp totals)
        SegAgg2 T = warp_agg[0];
        for (int w = 1; w < SCAN_THREADS / 32; ++w) T = seg_combine2(T, warp_agg[w], ovf);
        SegAgg2 ex{0, 0, 0, 0};
        if (tile == 0) {
            if (lane == 0) seg_publish(tiles, T, 2);
        } else {
            if (lane == 0) seg_publish(tiles + tile, T, 1);
            // look back 32 tiles at a time, lane i at tile (base - i): a tile
            // ends the walk when it holds an inclusive prefix, when the heads
            // met so far (from the closest tile outward) cover both layers, or
            // before tile 0
            for (int64_t jb = (int64_t)tile - 1;; jb -= 32) {
                const int64_t j = jb - lane;
                SegAgg2 v{0, 0, 0, 0};
                uint32_t st = 2;
                if (j >= 0) {
                    volatile SegTile *pt = tiles + j;
                    st = pt->status;
                    for (int it = 0; st == 0 && it < kLookbackPolls; ++it) {
                        __nanosleep(64);
                        st = pt->status;
                    }
                    if (st == 0) latch(status, ST_TIMEOUT);
                    __threadfence();
                    if (st == 2) v = SegAgg2{pt->p0, pt->p1, pt->pf, 0};
                    else if (st == 1) v = SegAgg2{pt->a0, pt->a1, pt->af, 0};
                }
                // heads met from the closest tile (lane 0) up to this lane
                uint32_t cf = v.f;
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, cf, o);
                    if (lane >= o) cf |= y;
                }
                const bool term = j < 0 || st != 1 || (cf & 3u) == 3u;
                const unsigned tb = __ballot_sync(0xffffffffu, term);
                const int L = tb ? __ffs((int)tb) - 1 : 31;   // the last lane to take
                if (lane > L) v = SegAgg2{0, 0, 0, 0};
                // fold lanes L .. 0 in tile order (earlier tiles first)
                for (int o = 1; o < 32; o <<= 1) {
                    const SegAgg2 y{__shfl_down_sync(0xffffffffu, v.v0, o), __shfl_down_sync(0xffffffffu, v.v1, o),
                                    __shfl_down_sync(0xffffffffu, v.f, o), 0};
                    if (lane + o < 32) v = seg_combine2(y, v, ovf);
                }
                v = SegAgg2{__shfl_sync(0xffffffffu, v.v0, 0), __shfl_sync(0xffffffffu, v.v1, 0),
                            __shfl_sync(0xffffffffu, v.f, 0), 0};
                ex = seg_combine2(v, ex, ovf);
                if (tb) break;
            }
            if (lane == 0) seg_publish(tiles + tile, seg_combine2(ex, T, ovf), 2);
        }
        if (lane == 0) {
            SegAgg2 run = ex;
            for (int w = 0; w < SCAN_THREADS / 32; ++w) {
                const SegAgg2 c = warp_agg[w];
                warp_agg[w] = run;
                run = seg_combine2(run, c, ovf);
            }
        }
    }
    __syncthreads();
    const SegAgg2 excl_lane = seg_shfl_up2(incl, 1);
    SegAgg2 pre = warp_agg[warp];
    if (lane > 0) pre = seg_combine2(pre, excl_lane, ovf);
    uint64_t r0 = pre.v0, r1 = pre.v1;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        const uint64_t i = base + j;
        if (i < n) {
            const uint32_t h = (hbits >> (2 * j)) & 3u;
            r0 = (h & 1u) ? v[j].x : add_chk(r0, v[j].x, ovf);
            r1 = (h & 2u) ? v[j].y : add_chk(r1, v[j].y, ovf);
            if (outp) {
                outp[i] = make_ulonglong2(r0, r1);
            } else {
                out0[i] = r0;
                out1[i] = r1;
            }
        }
    }
    if (ovf) latch(status, ST_OVERFLOW);
}

// Outputs: out0 / out1 (one array per layer), or outp (the (layer 0,
// layer 1) pairs interleaved) when it is non-null.  A gathering functor's
// values are stashed in scan order; with `keep` non-null the stash is that
// caller-owned array (n pairs), which then holds the gathered values.
#ifndef TM_SCAN_ONEPASS
#define TM_SCAN_ONEPASS 1   // 1: one pass with look-back; 0: reduce, carries, rescan
#endif
template <class F>
int segmented_scan2_u64(tm_ctx *ctx, const F &f, uint64_t n, uint64_t *out0, uint64_t *out1,
                        ulonglong2 *outp = nullptr, ulonglong2 *keep = nullptr)
{
    if (n == 0) return TM_OK;
    const uint64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    ScratchScope scope(ctx);
#if TM_SCAN_ONEPASS
    if (tiles >= 0xFFFFFFFFull) return set_err(ctx, TM_E_LIMIT, "scan of more than 2^32 tiles");
    char *st = (char *)salloc(ctx, tiles * sizeof(SegTile) + 256);
    if (!st) return TM_E_NOMEM;
    uint32_t *counter = (uint32_t *)(st + tiles * sizeof(SegTile));
    cudaMemsetAsync(st, 0, tiles * sizeof(SegTile) + 4, ctx->stream);
    launch(ctx, k_segscan2_onepass<F>, (unsigned)tiles, SCAN_THREADS, f, n, (SegTile *)st, counter, keep, out0, out1,
           outp, ctx->status);
    return check_cuda(ctx, cudaGetLastError(), "segmented scan");
#endif
    SegAgg2 *aggs = (SegAgg2 *)salloc(ctx, tiles * sizeof(SegAgg2));
    ulonglong2 *stash = !F::kGathered ? nullptr : keep ? keep : (ulonglong2 *)salloc(ctx, n * sizeof(ulonglong2));
    if (!aggs || (F::kGathered && !stash)) return TM_E_NOMEM;
    launch(ctx, k_segscan2_reduce<F>, (unsigned)tiles, SCAN_THREADS, f, n, aggs, stash, ctx->status);
    launch(ctx, k_segscan2_carries, 1, 1024, aggs, tiles, ctx->status);
    launch(ctx, k_segscan2_final<F>, (unsigned)tiles, SCAN_THREADS, f, n, aggs, (const ulonglong2 *)stash, out0,
           out1, outp, ctx->status);
    return check_cuda(ctx, cudaGetLastError(), "segmented scan");
}

}  // namespace
}  // namespace timest
