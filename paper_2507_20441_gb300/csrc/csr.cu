// Temporal CSR builder (Sec. 3 preamble; Defs. 3.1-3.3).
//
// From m raw tuples (u, v, t) it builds, all on the device:
//   GLOBAL order (t', src, dst)      -> gid, the edge id used everywhere
//   out-lists   (src | t', dst)      -> out_off / out_t / out_nbr / out_gid / out_pos
//   in-lists    (dst | t', src)      -> in_off / in_t / in_nbr / in_gid / in_pos / in_to_out
//   multi-edge  (src, dst | t')      -> pairs, pair_off / pair_dst / multi_t / multi_to_out
// with t' = t - t_min.  The orderings come from a stable LSD radix sort (up to
// 7-bit digits, up to four payload arrays) written here.  The GLOBAL order is
// a sort by t' after which each run of equal t' is put in (src, dst) order in
// place (one thread, one block, or, for a run of more than 4096 edges, the
// full three-key sort).  The OUT and IN orders are stable re-sorts of the
// GLOBAL order by one endpoint that carry gid, t' and the other endpoint as
// payloads, so no list array is gathered; each edge's list position by gid
// (the inverse of the sort's permutation) is then written through buckets of
// consecutive gids.  The IN sort carries each edge's out-list position too
// (read in GLOBAL order), which is the in -> out map, and the multi-edge
// order is a stable re-sort of the IN order by source carrying t', the
// destination and that map (-> multi_to_out).  The random accesses left are
// the cross ranks, found by binary searches in the owner's other list (four
// per thread in lockstep).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <memory>
#include <string>

#include "scan.cuh"
#include "tm_device.cuh"
#include "tm_internal.h"

namespace timest {

namespace {

// ---- radix sort --------------------------------------------------------
// Keys are sorted least significant digit first, with up to 7-bit digits
// (a 21-bit vertex id takes three passes, a 27-bit time four).  A pass is
//   1. per-tile digit counts (4096 keys per tile), stored digit-major;
//   2. an exclusive scan of those counts, which gives, for every (digit,
//      tile), where the tile's run of that digit starts in the output;
//   3. the scatter: each tile ranks its keys stably (per warp, by one ballot
//      per digit bit, or at once when the warp's digits agree; then across
//      warps), reorders them by digit in shared memory and writes each
//      digit's run out contiguously.
// No block waits on another.
#ifndef TM_RS_ITEMS
#define TM_RS_ITEMS 16   // keys per thread (8 and 12 measured slower)
#endif
#ifndef TM_RS_MATCH
#define TM_RS_MATCH 0    // 1: peers of a digit by one match-any instead of a ballot per digit bit
#endif
constexpr int OS_THREADS = 256;
constexpr int OS_ITEMS = TM_RS_ITEMS;
constexpr int OS_TILE = OS_THREADS * OS_ITEMS;     // 4096 keys per tile
constexpr int OS_WARPS = OS_THREADS / 32;
constexpr int OS_WCHUNK = OS_ITEMS * 32;           // keys per warp chunk
#ifndef TM_RS_MAXBITS
#define TM_RS_MAXBITS 7   // measured: 7-bit digits beat 9 (a 27-bit time in four passes instead of three)
#endif
constexpr int OS_MAXBITS = TM_RS_MAXBITS;
constexpr int OS_MAXRADIX = 1 << OS_MAXBITS;
constexpr int OS_SCAN = 512;   // entries of the block scan of the digit totals (two per thread)
static_assert(OS_MAXRADIX <= OS_SCAN && OS_THREADS * 2 == OS_SCAN, "digit scan layout");
constexpr int OS_MAXPASS = (32 + OS_MAXBITS - 1) / OS_MAXBITS;   // any 32-bit key
// dynamic shared memory of a scatter pass with np payload arrays
[[maybe_unused]] constexpr size_t os_smem(int np)
{
    return (size_t)OS_TILE * 4 * (1 + np) + (size_t)OS_TILE * 2 + (size_t)OS_WARPS * OS_MAXRADIX * 2 +
           (size_t)(OS_SCAN + OS_MAXRADIX) * 4;
}

// per-tile digit counts, written to counts[d * ntiles + tile].  Each warp
// counts into its own histogram with shared atomics; a warp whose 32 digits
// agree (sorted or nearly sorted input) adds once.
// Up to two independent arrays of the same length sorted by the same passes:
// blocks [0, ntiles) work on set 0, blocks [ntiles, 2 ntiles) on set 1.  The
// counts of set 1 follow those of set 0, so after one exclusive scan over
// both, set 1's output offsets are shifted by exactly n.
struct RsSet {
    const uint32_t *kin, *p0in, *p1in;
    uint32_t *kout, *p0out, *p1out;
    const uint32_t *p2in = nullptr;
    uint32_t *p2out = nullptr;
    const uint32_t *p3in = nullptr;
    uint32_t *p3out = nullptr;
    uint32_t *inv = nullptr;   // when set: inv[payload 0] = output position (the inverse permutation)
};
struct RsJobs {
    RsSet s[2];
};

__global__ void __launch_bounds__(OS_THREADS, 6) k_rs_count(RsJobs J, uint32_t n, int shift, int bits, uint32_t ntiles,
                                                             uint32_t *__restrict__ counts_all)
{
    const uint32_t job = blockIdx.x >= ntiles ? 1u : 0u, tile = blockIdx.x - job * ntiles;
    const uint32_t *__restrict__ kin = job ? J.s[1].kin : J.s[0].kin;
    uint32_t *__restrict__ counts = counts_all + ((size_t)job * ntiles << bits);
    __shared__ uint32_t h[OS_WARPS][OS_MAXRADIX];
    const uint32_t radix = 1u << bits, dmask = radix - 1u;
    for (uint32_t i = threadIdx.x; i < (uint32_t)(OS_WARPS * OS_MAXRADIX); i += OS_THREADS) (&h[0][0])[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t base = tile * OS_TILE;
    uint32_t kv[OS_ITEMS];
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {   // all loads in flight before any count
        const uint32_t i = base + j * OS_THREADS + threadIdx.x;
        kv[j] = i < n ? __ldg(kin + i) : 0u;
    }
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {
        const uint32_t i = base + j * OS_THREADS + threadIdx.x;
        const bool valid = i < n;
        const uint32_t d = valid ? ((kv[j] >> shift) & dmask) : radix;
        const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
        if (__all_sync(0xffffffffu, d == d0)) {
            if (lane == 0 && d0 < radix) atomicAdd(&h[warp][d0], 32u);
        } else if (valid) {
            atomicAdd(&h[warp][d], 1u);
        }
    }
    __syncthreads();
    for (uint32_t d = threadIdx.x; d < radix; d += OS_THREADS) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < OS_WARPS; ++w) c += h[w][d];
        counts[(size_t)d * ntiles + tile] = c;
    }
}

// block-wide exclusive scan of two values per thread (512 entries)
__device__ __forceinline__ void os_block_scan512(uint32_t *vals /* smem [512] in/out */, uint32_t *warp_tot /* smem [8] */)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    uint32_t a = vals[2 * t], b = vals[2 * t + 1];
    uint32_t s = a + b, incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < OS_WARPS ? warp_tot[lane] : 0, wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < OS_WARPS) warp_tot[lane] = wi - w;
    }
    __syncthreads();
    uint32_t ex = warp_tot[warp] + incl - s;
    vals[2 * t] = ex;
    vals[2 * t + 1] = ex + a;
    __syncthreads();
}

// Keys (and payloads) of one tile are ranked stably per warp chunk: a warp
// whose 32 digits agree takes its ranks directly; otherwise the lanes with
// the same digit are found with one ballot per digit bit.  A null p0in reads
// payload 0 as the key's input index.  With inv set (a final pass), each
// element also writes its output position at inv[payload 0].  Payloads 0-2
// are held in registers from the start; payload 3 is read when the tile is
// placed in shared memory.
template <int NP>
__global__ void __launch_bounds__(OS_THREADS, NP >= 3 ? 2 : NP >= 2 ? 3 : 4)
    k_rs_scatter(RsJobs J, uint32_t n, int shift, int bits, uint32_t ntiles, const uint32_t *__restrict__ offs_all)
{
    const uint32_t job = blockIdx.x >= ntiles ? 1u : 0u, tile = blockIdx.x - job * ntiles;
    // per-field selects keep the parameter block out of local memory
    const uint32_t *__restrict__ kin = job ? J.s[1].kin : J.s[0].kin;
    const uint32_t *__restrict__ p0in = job ? J.s[1].p0in : J.s[0].p0in;
    const uint32_t *__restrict__ p1in = job ? J.s[1].p1in : J.s[0].p1in;
    uint32_t *__restrict__ kout = job ? J.s[1].kout : J.s[0].kout;
    uint32_t *__restrict__ p0out = job ? J.s[1].p0out : J.s[0].p0out;
    uint32_t *__restrict__ p1out = job ? J.s[1].p1out : J.s[0].p1out;
    const uint32_t *__restrict__ p2in = job ? J.s[1].p2in : J.s[0].p2in;
    uint32_t *__restrict__ p2out = job ? J.s[1].p2out : J.s[0].p2out;
    const uint32_t *__restrict__ p3in = job ? J.s[1].p3in : J.s[0].p3in;
    uint32_t *__restrict__ p3out = job ? J.s[1].p3out : J.s[0].p3out;
    uint32_t *__restrict__ inv = job ? J.s[1].inv : J.s[0].inv;
    const uint32_t *__restrict__ offs = offs_all + ((size_t)job * ntiles << bits);
    const uint32_t bias = job * n;   // set 1's scanned offsets start at n
    extern __shared__ __align__(16) unsigned char os_smem_buf[];
    uint32_t *s_key = reinterpret_cast<uint32_t *>(os_smem_buf);
    uint32_t *s_p0 = s_key + OS_TILE;
    uint32_t *s_p1 = s_p0 + (NP >= 1 ? OS_TILE : 0);
    uint32_t *s_p2 = s_p1 + (NP >= 2 ? OS_TILE : 0);
    uint32_t *s_p3 = s_p2 + (NP >= 3 ? OS_TILE : 0);
    uint16_t *s_rank = reinterpret_cast<uint16_t *>(s_p3 + (NP >= 4 ? OS_TILE : 0));
    uint16_t *s_wcnt = s_rank + OS_TILE;                                            // [warp][digit]
    uint32_t *s_tex = reinterpret_cast<uint32_t *>(s_wcnt + OS_WARPS * OS_MAXRADIX);  // digit start in the tile
    uint32_t *s_gpos = s_tex + OS_SCAN;                                             // digit start in the output
    __shared__ uint32_t s_wt[OS_WARPS];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t radix = 1u << bits, dmask = radix - 1u;
    const uint32_t base = tile * OS_TILE;
    for (int i = t; i < OS_WARPS * OS_MAXRADIX; i += OS_THREADS) s_wcnt[i] = 0;
    for (uint32_t d = t; d < (uint32_t)OS_MAXRADIX; d += OS_THREADS)
        s_gpos[d] = d < radix ? __ldg(offs + (size_t)d * ntiles + tile) - bias : 0u;
    const uint32_t lt = (1u << lane) - 1u;
    uint16_t *wc = s_wcnt + warp * OS_MAXRADIX;
    constexpr int NA = NP >= 1 ? OS_ITEMS : 1, NB = NP >= 2 ? OS_ITEMS : 1, NC = NP >= 3 ? OS_ITEMS : 1;
    uint32_t kv[OS_ITEMS], av[NA], bv[NB], cv[NC];
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {   // keys and payloads in flight before any vote
        const uint32_t i = base + warp * OS_WCHUNK + j * 32 + lane;
        kv[j] = i < n ? __ldg(kin + i) : 0u;
        if (NP >= 1) av[j % NA] = i < n ? (p0in ? __ldg(p0in + i) : i) : 0u;
        if (NP >= 2) bv[j % NB] = i < n ? __ldg(p1in + i) : 0u;
        if (NP >= 3) cv[j % NC] = i < n ? __ldg(p2in + i) : 0u;
    }
    __syncthreads();
    // ---- rank inside each warp's chunk (order: warp, item, lane)
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {
        const uint32_t li = warp * OS_WCHUNK + j * 32 + lane;
        const bool valid = base + li < n;
        const uint32_t d = valid ? ((kv[j] >> shift) & dmask) : radix;
        uint32_t peers;
#if TM_RS_MATCH
        peers = __match_any_sync(0xffffffffu, d);   // lanes with the same digit (invalid lanes: digit radix)
#else
        if (__all_sync(0xffffffffu, d == __shfl_sync(0xffffffffu, d, 0))) {
            peers = 0xffffffffu;
        } else {
            peers = __ballot_sync(0xffffffffu, valid);
            if (!valid) peers = ~peers;
            for (int b = 0; b < bits; ++b) {
                const uint32_t bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
                peers &= ((d >> b) & 1u) ? bb : ~bb;
            }
        }
#endif
        uint32_t cur = valid ? wc[d] : 0;
        __syncwarp();
        if (valid) {
            s_rank[li] = (uint16_t)(cur + __popc(peers & lt));
            if ((peers & lt) == 0) wc[d] = (uint16_t)(cur + __popc(peers));
        }
        __syncwarp();
    }
    __syncthreads();
    // ---- per digit: tile total and warp offsets
    for (uint32_t d = t; d < (uint32_t)OS_SCAN; d += OS_THREADS) {   // entries past the radix: 0
        uint32_t run = 0;
        if (d < radix)
            for (int w = 0; w < OS_WARPS; ++w) {
                uint32_t c = s_wcnt[w * OS_MAXRADIX + d];
                s_wcnt[w * OS_MAXRADIX + d] = (uint16_t)run;
                run += c;
            }
        s_tex[d] = run;
    }
    __syncthreads();
    os_block_scan512(s_tex, s_wt);
    // ---- place keys (and payloads) in digit order inside shared memory
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {
        const uint32_t li = warp * OS_WCHUNK + j * 32 + lane;
        if (base + li < n) {
            const uint32_t k = kv[j];
            const uint32_t d = (k >> shift) & dmask;
            const uint32_t pos = s_tex[d] + s_wcnt[warp * OS_MAXRADIX + d] + s_rank[li];
            s_key[pos] = k;
            if (NP >= 1) s_p0[pos] = av[j % NA];
            if (NP >= 2) s_p1[pos] = bv[j % NB];
            if (NP >= 3) s_p2[pos] = cv[j % NC];
            if (NP >= 4) s_p3[pos] = __ldg(p3in + base + li);
        }
    }
    __syncthreads();
    // ---- write the tile's digit runs out
    const uint32_t tile_n = min((uint32_t)OS_TILE, n - base);
    for (uint32_t p = t; p < tile_n; p += OS_THREADS) {
        const uint32_t k = s_key[p];
        const uint32_t d = (k >> shift) & dmask;
        const uint32_t g = s_gpos[d] + (p - s_tex[d]);
        kout[g] = k;
        if (NP >= 1) p0out[g] = s_p0[p];
        if (NP >= 2) p1out[g] = s_p1[p];
        if (NP >= 3) p2out[g] = s_p2[p];
        if (NP >= 4) p3out[g] = s_p3[p];
        if (NP >= 1 && inv) inv[s_p0[p]] = g;
    }
}

// The same pass with the tile staged through one shared array at a time:
// keys first (which also fixes every element's output position), then each
// payload, read from global memory in its own round.  Shared memory stays at
// 52 KB whatever the payload count, so four blocks fit on an SM where the
// all-at-once layout above fits two.
#ifndef TM_RS_STAGED
#define TM_RS_STAGED 1
#endif
#ifndef TM_RS_ST_MINB
#define TM_RS_ST_MINB 4   // blocks per SM the staged pass is compiled for (64 registers)
#endif
[[maybe_unused]] constexpr size_t os_smem_staged()
{
    return (size_t)OS_TILE * 4 * 2 + (size_t)OS_TILE * 2 + (size_t)OS_WARPS * OS_MAXRADIX * 2 +
           (size_t)(OS_SCAN + OS_MAXRADIX) * 4;
}

template <int NP>
__global__ void __launch_bounds__(OS_THREADS, TM_RS_ST_MINB)
    k_rs_scatter_st(RsJobs J, uint32_t n, int shift, int bits, uint32_t ntiles, const uint32_t *__restrict__ offs_all)
{
    const uint32_t job = blockIdx.x >= ntiles ? 1u : 0u, tile = blockIdx.x - job * ntiles;
    const uint32_t *__restrict__ kin = job ? J.s[1].kin : J.s[0].kin;
    uint32_t *__restrict__ kout = job ? J.s[1].kout : J.s[0].kout;
    uint32_t *__restrict__ inv = job ? J.s[1].inv : J.s[0].inv;
    const uint32_t *__restrict__ offs = offs_all + ((size_t)job * ntiles << bits);
    const uint32_t bias = job * n;
    extern __shared__ __align__(16) unsigned char os_smem_buf[];
    uint32_t *s_buf = reinterpret_cast<uint32_t *>(os_smem_buf);                  // one array of the tile
    uint32_t *s_g = s_buf + OS_TILE;                                              // output position by tile slot
    uint16_t *s_rank = reinterpret_cast<uint16_t *>(s_g + OS_TILE);               // rank, then tile slot, by input
    uint16_t *s_wcnt = s_rank + OS_TILE;                                          // [warp][digit]
    uint32_t *s_tex = reinterpret_cast<uint32_t *>(s_wcnt + OS_WARPS * OS_MAXRADIX);   // OS_SCAN entries
    uint32_t *s_gpos = s_tex + OS_SCAN;
    __shared__ uint32_t s_wt[OS_WARPS];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t radix = 1u << bits, dmask = radix - 1u;
    const uint32_t base = tile * OS_TILE;
    const uint32_t tile_n = min((uint32_t)OS_TILE, n - base);
    for (int i = t; i < OS_WARPS * OS_MAXRADIX; i += OS_THREADS) s_wcnt[i] = 0;
    for (uint32_t d = t; d < (uint32_t)OS_MAXRADIX; d += OS_THREADS)
        s_gpos[d] = d < radix ? __ldg(offs + (size_t)d * ntiles + tile) - bias : 0u;
    const uint32_t lt = (1u << lane) - 1u;
    uint16_t *wc = s_wcnt + warp * OS_MAXRADIX;
    uint32_t kv[OS_ITEMS];
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {
        const uint32_t i = base + warp * OS_WCHUNK + j * 32 + lane;
        kv[j] = i < n ? __ldg(kin + i) : 0u;
    }
    __syncthreads();
    // ---- rank inside each warp's chunk (order: warp, item, lane)
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {
        const uint32_t li = warp * OS_WCHUNK + j * 32 + lane;
        const bool valid = base + li < n;
        const uint32_t d = valid ? ((kv[j] >> shift) & dmask) : radix;
        uint32_t peers;
#if TM_RS_MATCH
        peers = __match_any_sync(0xffffffffu, d);
#else
        if (__all_sync(0xffffffffu, d == __shfl_sync(0xffffffffu, d, 0))) {
            peers = 0xffffffffu;
        } else {
            peers = __ballot_sync(0xffffffffu, valid);
            if (!valid) peers = ~peers;
            for (int b = 0; b < bits; ++b) {
                const uint32_t bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
                peers &= ((d >> b) & 1u) ? bb : ~bb;
            }
        }
#endif
        uint32_t cur = valid ? wc[d] : 0;
        __syncwarp();
        if (valid) {
            s_rank[li] = (uint16_t)(cur + __popc(peers & lt));
            if ((peers & lt) == 0) wc[d] = (uint16_t)(cur + __popc(peers));
        }
        __syncwarp();
    }
    __syncthreads();
    for (uint32_t d = t; d < (uint32_t)OS_SCAN; d += OS_THREADS) {   // entries past the radix: 0
        uint32_t run = 0;
        if (d < radix)
            for (int w = 0; w < OS_WARPS; ++w) {
                uint32_t c = s_wcnt[w * OS_MAXRADIX + d];
                s_wcnt[w * OS_MAXRADIX + d] = (uint16_t)run;
                run += c;
            }
        s_tex[d] = run;
    }
    __syncthreads();
    os_block_scan512(s_tex, s_wt);
    // ---- keys into their tile slots; each element keeps its slot (in s_rank,
    // read back only by the thread that wrote it)
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {
        const uint32_t li = warp * OS_WCHUNK + j * 32 + lane;
        if (base + li < n) {
            const uint32_t k = kv[j];
            const uint32_t d = (k >> shift) & dmask;
            const uint32_t pos = s_tex[d] + s_wcnt[warp * OS_MAXRADIX + d] + s_rank[li];
            s_buf[pos] = k;
            s_rank[li] = (uint16_t)pos;
        }
    }
    __syncthreads();
    // ---- keys out; each slot's output position, kept for the payload rounds
    // (slot p is handled by the same thread in every round)
    for (uint32_t p = t; p < tile_n; p += OS_THREADS) {
        const uint32_t k = s_buf[p];
        const uint32_t d = (k >> shift) & dmask;
        const uint32_t g = s_gpos[d] + (p - s_tex[d]);
        s_g[p] = g;
        kout[g] = k;
    }
    // ---- payloads, one round each
#pragma unroll
    for (int a = 0; a < NP; ++a) {
        const uint32_t *__restrict__ pin = a == 0 ? (job ? J.s[1].p0in : J.s[0].p0in)
                                         : a == 1 ? (job ? J.s[1].p1in : J.s[0].p1in)
                                         : a == 2 ? (job ? J.s[1].p2in : J.s[0].p2in)
                                                  : (job ? J.s[1].p3in : J.s[0].p3in);
        uint32_t *__restrict__ pout = a == 0 ? (job ? J.s[1].p0out : J.s[0].p0out)
                                    : a == 1 ? (job ? J.s[1].p1out : J.s[0].p1out)
                                    : a == 2 ? (job ? J.s[1].p2out : J.s[0].p2out)
                                             : (job ? J.s[1].p3out : J.s[0].p3out);
        uint32_t pv[OS_ITEMS];
#pragma unroll
        for (int j = 0; j < OS_ITEMS; ++j) {   // loads in flight before the slots are written
            const uint32_t i = base + warp * OS_WCHUNK + j * 32 + lane;
            pv[j] = i < n ? (pin ? __ldg(pin + i) : i) : 0u;
        }
        __syncthreads();   // the previous round's reads of s_buf are done
#pragma unroll
        for (int j = 0; j < OS_ITEMS; ++j) {
            const uint32_t li = warp * OS_WCHUNK + j * 32 + lane;
            if (base + li < n) s_buf[s_rank[li]] = pv[j];
        }
        __syncthreads();
        for (uint32_t p = t; p < tile_n; p += OS_THREADS) {
            const uint32_t v = s_buf[p], g = s_g[p];
            pout[g] = v;
            if (a == 0 && inv) inv[v] = g;
        }
    }
}

// ---- inverse of a permutation, written through buckets -------------------
// inv[perm[i]] = i as one pass of random 4-byte writes costs a DRAM read and
// write of a whole sector per element once the array is larger than L2.
// Instead the (perm[i], i) pairs are first grouped into buckets of 2^shift
// consecutive values (unstable: the order inside a bucket does not matter),
// then written bucket after bucket, so the writes in flight cover a few
// buckets' worth of inv and every sector is complete before it leaves L2.
constexpr int IB_MAXB = 512;
__global__ void k_inv_cursor(uint32_t *__restrict__ cursor, uint32_t nb, int shift)
{
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) cursor[b] = b << shift;
}

__global__ void __launch_bounds__(OS_THREADS, 4) k_inv_bucket(const uint32_t *__restrict__ perm, uint32_t n, int shift,
                                                               uint32_t nb, uint32_t *__restrict__ cursor,
                                                               uint32_t *__restrict__ tkey, uint32_t *__restrict__ tpos)
{
    __shared__ uint32_t s_cnt[IB_MAXB], s_base[IB_MAXB], s_wt[OS_WARPS];
    __shared__ uint32_t s_key[OS_TILE], s_pos[OS_TILE];
    const int t = threadIdx.x;
    const uint32_t base = blockIdx.x * OS_TILE;
    const uint32_t tile_n = min((uint32_t)OS_TILE, n - base);
    for (int b = t; b < IB_MAXB; b += OS_THREADS) s_cnt[b] = 0;
    uint32_t v[OS_ITEMS];
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {
        const uint32_t i = base + j * OS_THREADS + t;
        v[j] = i < n ? __ldg(perm + i) : 0u;
    }
    __syncthreads();
    uint32_t r[OS_ITEMS];   // rank inside the tile's bucket (shared atomics: any order)
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {
        const uint32_t i = base + j * OS_THREADS + t;
        r[j] = i < n ? atomicAdd(&s_cnt[v[j] >> shift], 1u) : 0u;
    }
    __syncthreads();
    for (uint32_t b = t; b < nb; b += OS_THREADS) {
        const uint32_t c = s_cnt[b];
        s_base[b] = c ? atomicAdd(cursor + b, c) : 0u;
    }
    __syncthreads();
    os_block_scan512(s_cnt, s_wt);   // bucket starts inside the tile
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {
        const uint32_t i = base + j * OS_THREADS + t;
        if (i < n) {
            const uint32_t p = s_cnt[v[j] >> shift] + r[j];
            s_key[p] = v[j];
            s_pos[p] = i;
        }
    }
    __syncthreads();
    for (uint32_t p = t; p < tile_n; p += OS_THREADS) {
        const uint32_t k = s_key[p], b = k >> shift;
        const uint32_t dst = s_base[b] + (p - s_cnt[b]);
        tkey[dst] = k;
        tpos[dst] = s_pos[p];
    }
}

// 4 x TM_INV_VECS pairs per thread: TM_INV_VECS 16-byte loads of each work
// array (256-byte aligned) in flight, at vectors i, i + blockDim, ...
#ifndef TM_INV_VECS
#define TM_INV_VECS 1   // 2 and 4 measured no faster
#endif
__global__ void k_inv_fill(const uint32_t *__restrict__ tkey, const uint32_t *__restrict__ tpos, uint32_t n,
                           uint32_t *__restrict__ inv)
{
    const uint64_t v0 = (uint64_t)blockIdx.x * blockDim.x * TM_INV_VECS + threadIdx.x;
    uint4 k[TM_INV_VECS], p[TM_INV_VECS];
#pragma unroll
    for (int r = 0; r < TM_INV_VECS; ++r) {
        const uint64_t i = (v0 + (uint64_t)r * blockDim.x) * 4;
        if (i + 4 <= n) {
            k[r] = __ldg(reinterpret_cast<const uint4 *>(tkey + i));
            p[r] = __ldg(reinterpret_cast<const uint4 *>(tpos + i));
        }
    }
#pragma unroll
    for (int r = 0; r < TM_INV_VECS; ++r) {
        const uint64_t i = (v0 + (uint64_t)r * blockDim.x) * 4;
        if (i + 4 <= n) {
            inv[k[r].x] = p[r].x; inv[k[r].y] = p[r].y; inv[k[r].z] = p[r].z; inv[k[r].w] = p[r].w;
        } else {
            for (uint64_t j = i; j < n; ++j) inv[__ldg(tkey + j)] = __ldg(tpos + j);
        }
    }
}

int bits_for(uint64_t maxval)
{
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) ++b;
    return b;
}

// Stable LSD sort of (key, p0[, p1]) by the low `bits` bits of key, for one
// or two independent arrays of the same length (same payload count), sorted
// by the same launches; on return the sorted data is in the caller's buffers.
struct RsHost {
    uint32_t *key, *p0, *p1;
};

static int rs_prepare(tm_ctx *ctx, int np)
{
    // per device and cheap: set on every call
#if TM_RS_STAGED
    const int sm = (int)os_smem_staged();
    cudaError_t e = np == 0 ? cudaFuncSetAttribute(k_rs_scatter_st<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)
                  : np == 1 ? cudaFuncSetAttribute(k_rs_scatter_st<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)
                  : np == 2 ? cudaFuncSetAttribute(k_rs_scatter_st<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)
                  : np == 3 ? cudaFuncSetAttribute(k_rs_scatter_st<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)
                            : cudaFuncSetAttribute(k_rs_scatter_st<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
#else
    cudaError_t e = np == 0 ? cudaFuncSetAttribute(k_rs_scatter<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)os_smem(0))
                  : np == 1 ? cudaFuncSetAttribute(k_rs_scatter<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)os_smem(1))
                  : np == 2 ? cudaFuncSetAttribute(k_rs_scatter<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)os_smem(2))
                  : np == 3 ? cudaFuncSetAttribute(k_rs_scatter<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)os_smem(3))
                            : cudaFuncSetAttribute(k_rs_scatter<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)os_smem(4));
#endif
    return check_cuda(ctx, e, "radix pass shared memory");
}

// One LSD pass over digit bits [sh, sh + pb): counts, their scan, the scatter.
static int rs_pass(tm_ctx *ctx, const RsJobs &in, int nsets, int np, uint32_t n, uint32_t ntiles, int sh, int pb,
                   uint32_t *counts)
{
    const unsigned nblk = ntiles * (unsigned)nsets;
    const uint64_t ncount = ((uint64_t)ntiles << pb) * (uint64_t)nsets;
    launch(ctx, k_rs_count, nblk, OS_THREADS, in, n, sh, pb, ntiles, counts);
    int rc = exclusive_scan_u32(ctx, counts, counts, ncount, nullptr);
    if (rc) return rc;
#if TM_RS_STAGED
    const size_t sm = os_smem_staged();
    if (np == 0)
        launch_smem(ctx, k_rs_scatter_st<0>, nblk, OS_THREADS, sm, in, n, sh, pb, ntiles, (const uint32_t *)counts);
    else if (np == 1)
        launch_smem(ctx, k_rs_scatter_st<1>, nblk, OS_THREADS, sm, in, n, sh, pb, ntiles, (const uint32_t *)counts);
    else if (np == 2)
        launch_smem(ctx, k_rs_scatter_st<2>, nblk, OS_THREADS, sm, in, n, sh, pb, ntiles, (const uint32_t *)counts);
    else if (np == 3)
        launch_smem(ctx, k_rs_scatter_st<3>, nblk, OS_THREADS, sm, in, n, sh, pb, ntiles, (const uint32_t *)counts);
    else
        launch_smem(ctx, k_rs_scatter_st<4>, nblk, OS_THREADS, sm, in, n, sh, pb, ntiles, (const uint32_t *)counts);
#else
    if (np == 0)
        launch_smem(ctx, k_rs_scatter<0>, nblk, OS_THREADS, os_smem(0), in, n, sh, pb, ntiles, (const uint32_t *)counts);
    else if (np == 1)
        launch_smem(ctx, k_rs_scatter<1>, nblk, OS_THREADS, os_smem(1), in, n, sh, pb, ntiles, (const uint32_t *)counts);
    else if (np == 2)
        launch_smem(ctx, k_rs_scatter<2>, nblk, OS_THREADS, os_smem(2), in, n, sh, pb, ntiles, (const uint32_t *)counts);
    else if (np == 3)
        launch_smem(ctx, k_rs_scatter<3>, nblk, OS_THREADS, os_smem(3), in, n, sh, pb, ntiles, (const uint32_t *)counts);
    else
        launch_smem(ctx, k_rs_scatter<4>, nblk, OS_THREADS, os_smem(4), in, n, sh, pb, ntiles, (const uint32_t *)counts);
#endif
    return check_cuda(ctx, cudaGetLastError(), "radix pass");
}

int radix_sort_sets(tm_ctx *ctx, const RsHost *sets, int nsets, uint32_t n, int bits)
{
    ScratchScope scope(ctx);
    if (n <= 1 || bits <= 0 || nsets <= 0) return TM_OK;
    if (nsets > 2) return set_err(ctx, TM_E_LIMIT, "at most two arrays per radix sort");
    const int np = sets[0].p1 ? 2 : (sets[0].p0 ? 1 : 0);
    const int npass = (bits + OS_MAXBITS - 1) / OS_MAXBITS;
    if (npass > OS_MAXPASS) return set_err(ctx, TM_E_LIMIT, "radix key wider than 32 bits");
    const uint32_t ntiles = (n + OS_TILE - 1) / OS_TILE;
    uint32_t *counts = (uint32_t *)salloc(ctx, (size_t)nsets * ntiles * OS_MAXRADIX * 4);
    if (!counts) return TM_E_NOMEM;
    RsJobs in{};
    for (int j = 0; j < nsets; ++j) {
        uint32_t *k2 = (uint32_t *)salloc(ctx, (size_t)n * 4);
        uint32_t *a2 = np >= 1 ? (uint32_t *)salloc(ctx, (size_t)n * 4) : nullptr;
        uint32_t *b2 = np >= 2 ? (uint32_t *)salloc(ctx, (size_t)n * 4) : nullptr;
        if (!k2 || (np >= 1 && !a2) || (np >= 2 && !b2)) return TM_E_NOMEM;
        in.s[j] = RsSet{sets[j].key, sets[j].p0, sets[j].p1, k2, a2, b2};
    }
    int rc = rs_prepare(ctx, np);
    if (rc) return rc;
    cudaStream_t st = ctx->stream;
    for (int pass = 0, sh = 0; pass < npass && rc == TM_OK; ++pass) {
        const int left = npass - pass, pb = (bits - sh + left - 1) / left;
        rc = rs_pass(ctx, in, nsets, np, n, ntiles, sh, pb, counts);
        // the outputs of this pass are the inputs of the next
        for (int j = 0; j < nsets; ++j) {
            RsSet &x = in.s[j];
            RsSet y{x.kout, x.p0out, x.p1out, const_cast<uint32_t *>(x.kin), const_cast<uint32_t *>(x.p0in),
                    const_cast<uint32_t *>(x.p1in)};
            x = y;
        }
        sh += pb;
    }
    for (int j = 0; rc == TM_OK && j < nsets; ++j) {
        const RsSet &x = in.s[j];
        if (x.kin == sets[j].key) continue;
        cudaMemcpyAsync(sets[j].key, x.kin, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
        if (np >= 1) cudaMemcpyAsync(sets[j].p0, x.p0in, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
        if (np >= 2) cudaMemcpyAsync(sets[j].p1, x.p1in, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
    }
    return rc;
}


#ifndef TM_RS_INV_BUCKET
#define TM_RS_INV_BUCKET 1   // 0: the last radix pass writes the inverse with one random store per element
#endif

// inv[perm[i]] = i for a permutation perm of [0, n); tkey/tpos are n-entry
// work arrays (allocated here when null).
static int inverse_perm(tm_ctx *ctx, const uint32_t *perm, uint32_t n, uint32_t *inv, uint32_t *tkey, uint32_t *tpos)
{
    ScratchScope scope(ctx);
    if (n == 0) return TM_OK;
    if (!tkey) tkey = (uint32_t *)salloc(ctx, (size_t)n * 4);
    if (!tpos) tpos = (uint32_t *)salloc(ctx, (size_t)n * 4);
    uint32_t *cursor = (uint32_t *)salloc(ctx, IB_MAXB * 4);
    if (!tkey || !tpos || !cursor) return TM_E_NOMEM;
    int shift = 0;
    while (((uint64_t)(n - 1) >> shift) >= (uint64_t)IB_MAXB) ++shift;
    const uint32_t nb = (uint32_t)(((uint64_t)(n - 1) >> shift) + 1);
    launch(ctx, k_inv_cursor, 1, IB_MAXB, cursor, nb, shift);
    launch(ctx, k_inv_bucket, (n + OS_TILE - 1) / OS_TILE, OS_THREADS, perm, n, shift, nb, cursor, tkey, tpos);
    launch(ctx, k_inv_fill, (unsigned)(((uint64_t)n + 1024 * TM_INV_VECS - 1) / (1024 * TM_INV_VECS)), 256,
           (const uint32_t *)tkey, (const uint32_t *)tpos, n, inv);
    return check_cuda(ctx, cudaGetLastError(), "inverse permutation");
}

// The same sort from read-only inputs into separate outputs (no copies): the
// passes alternate between the outputs and scratch so that the last one
// writes the outputs.  A set whose p0_in is null and p0 is not gets payload 0
// = the input index (the sorting permutation).  Outputs must not alias inputs.
struct RsTo {
    const uint32_t *key_in, *p0_in, *p1_in;
    uint32_t *key, *p0, *p1;
    const uint32_t *p2_in = nullptr;
    uint32_t *p2 = nullptr;
    const uint32_t *p3_in = nullptr;
    uint32_t *p3 = nullptr;
    uint32_t *inv = nullptr;   // optional: inv[payload 0] = sorted position, written by the last pass
};

__global__ void k_iota2(uint32_t *__restrict__ a, uint32_t *__restrict__ b, uint32_t m)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) { if (a) a[i] = i; if (b) b[i] = i; }
}

int radix_sort_sets_to(tm_ctx *ctx, const RsTo *sets, int nsets, uint32_t n, int bits)
{
    ScratchScope scope(ctx);
    if (nsets <= 0 || n == 0) return TM_OK;
    if (nsets > 2) return set_err(ctx, TM_E_LIMIT, "at most two arrays per radix sort");
    const int np = sets[0].p3 ? 4 : sets[0].p2 ? 3 : sets[0].p1 ? 2 : (sets[0].p0 ? 1 : 0);
    cudaStream_t st = ctx->stream;
    if (n <= 1 || bits <= 0) {
        for (int j = 0; j < nsets; ++j) {
            const RsTo &x = sets[j];
            cudaMemcpyAsync(x.key, x.key_in, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
            if (np >= 1) {
                if (x.p0_in) cudaMemcpyAsync(x.p0, x.p0_in, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
                else launch(ctx, k_iota2, (n + 255) / 256, 256, x.p0, (uint32_t *)nullptr, n);
            }
            if (np >= 2) cudaMemcpyAsync(x.p1, x.p1_in, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
            if (np >= 3) cudaMemcpyAsync(x.p2, x.p2_in, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
            if (np >= 4) cudaMemcpyAsync(x.p3, x.p3_in, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
            if (x.inv) {   // an identity order (payload 0 is then the input index)
                if (x.p0_in) return set_err(ctx, TM_E_ARG, "internal: inverse of a sort with explicit payload 0");
                launch(ctx, k_iota2, (n + 255) / 256, 256, x.inv, (uint32_t *)nullptr, n);
            }
        }
        return TM_OK;
    }
    const int npass = (bits + OS_MAXBITS - 1) / OS_MAXBITS;
    if (npass > OS_MAXPASS) return set_err(ctx, TM_E_LIMIT, "radix key wider than 32 bits");
    const uint32_t ntiles = (n + OS_TILE - 1) / OS_TILE;
    uint32_t *counts = (uint32_t *)salloc(ctx, (size_t)nsets * ntiles * OS_MAXRADIX * 4);
    if (!counts) return TM_E_NOMEM;
    RsSet scr[2] = {}, dst[2] = {};
    for (int j = 0; j < nsets; ++j) {
        dst[j] = RsSet{nullptr, nullptr, nullptr, sets[j].key, sets[j].p0, sets[j].p1};
        dst[j].p2out = sets[j].p2;
        dst[j].p3out = sets[j].p3;
        if (npass >= 2) {
            uint32_t *k2 = (uint32_t *)salloc(ctx, (size_t)n * 4);
            uint32_t *a2 = np >= 1 ? (uint32_t *)salloc(ctx, (size_t)n * 4) : nullptr;
            uint32_t *b2 = np >= 2 ? (uint32_t *)salloc(ctx, (size_t)n * 4) : nullptr;
            uint32_t *c2 = np >= 3 ? (uint32_t *)salloc(ctx, (size_t)n * 4) : nullptr;
            uint32_t *d2 = np >= 4 ? (uint32_t *)salloc(ctx, (size_t)n * 4) : nullptr;
            if (!k2 || (np >= 1 && !a2) || (np >= 2 && !b2) || (np >= 3 && !c2) || (np >= 4 && !d2)) return TM_E_NOMEM;
            scr[j] = RsSet{nullptr, nullptr, nullptr, k2, a2, b2};
            scr[j].p2out = c2;
            scr[j].p3out = d2;
        }
    }
    int rc = rs_prepare(ctx, np);
    if (rc) return rc;
    RsJobs in{};
    for (int j = 0; j < nsets; ++j) {
        in.s[j] = RsSet{sets[j].key_in, sets[j].p0_in, sets[j].p1_in, nullptr, nullptr, nullptr};
        in.s[j].p2in = sets[j].p2_in;
        in.s[j].p3in = sets[j].p3_in;
    }
    for (int pass = 0, sh = 0; pass < npass && rc == TM_OK; ++pass) {
        const int left = npass - pass, pb = (bits - sh + left - 1) / left;
        // pass i writes the outputs when npass - 1 - i is even, else scratch
        const bool to_dst = ((npass - 1 - pass) & 1) == 0;
        for (int j = 0; j < nsets; ++j) {
            const RsSet &o = to_dst ? dst[j] : scr[j];
            in.s[j].kout = o.kout; in.s[j].p0out = o.p0out; in.s[j].p1out = o.p1out; in.s[j].p2out = o.p2out;
            in.s[j].p3out = o.p3out;
            in.s[j].inv = !TM_RS_INV_BUCKET && pass == npass - 1 ? sets[j].inv : nullptr;
        }
        rc = rs_pass(ctx, in, nsets, np, n, ntiles, sh, pb, counts);
        for (int j = 0; j < nsets; ++j) {
            RsSet nx{in.s[j].kout, in.s[j].p0out, in.s[j].p1out, nullptr, nullptr, nullptr};
            nx.p2in = in.s[j].p2out;
            nx.p3in = in.s[j].p3out;
            in.s[j] = nx;
        }
        sh += pb;
    }
#if TM_RS_INV_BUCKET
    // the inverse permutations, through buckets; the scratch of the passes
    // (free once the last pass has written the outputs) holds the pairs
    for (int j = 0; rc == TM_OK && j < nsets; ++j) {
        if (!sets[j].inv) continue;
        if (sets[j].p0_in) return set_err(ctx, TM_E_ARG, "internal: inverse of a sort with explicit payload 0");
        uint32_t *tk = npass >= 2 ? scr[j].kout : nullptr, *tp = npass >= 2 ? scr[j].p0out : nullptr;
        rc = inverse_perm(ctx, sets[j].p0, n, sets[j].inv, tk, tp);
    }
#endif
    return rc;
}

int radix_sort(tm_ctx *ctx, uint32_t *key, uint32_t *p0, uint32_t *p1, uint32_t n, int bits)
{
    RsHost h{key, p0, p1};
    return radix_sort_sets(ctx, &h, 1, n, bits);
}

// ---- input validation and t' -------------------------------------------
struct Stats {
    long long tmin, tmax;
    unsigned long long nself, nbad;
};

__global__ void k_input_stats(const uint32_t *__restrict__ src, const uint32_t *__restrict__ dst,
                              const int64_t *__restrict__ t, uint64_t m, uint32_t n, Stats *st)
{
    long long lo = LLONG_MAX, hi = LLONG_MIN;
    unsigned long long ns = 0, nb = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u = src[i], v = dst[i];
        if (u >= n || v >= n) { ++nb; continue; }
        if (u == v) { ++ns; continue; }
        long long x = t[i];
        lo = x < lo ? x : lo;
        hi = x > hi ? x : hi;
    }
    // warp, then block reduction: one set of atomics per block
    __shared__ long long s_lo[32], s_hi[32];
    __shared__ unsigned long long s_ns[32], s_nb[32];
    for (int pass = 0; pass < 2; ++pass) {
        for (int o = 16; o > 0; o >>= 1) {
            long long a = __shfl_down_sync(0xffffffffu, lo, o), b = __shfl_down_sync(0xffffffffu, hi, o);
            lo = a < lo ? a : lo; hi = b > hi ? b : hi;
            ns += __shfl_down_sync(0xffffffffu, ns, o);
            nb += __shfl_down_sync(0xffffffffu, nb, o);
        }
        if (pass == 1) break;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
        if (lane == 0) { s_lo[warp] = lo; s_hi[warp] = hi; s_ns[warp] = ns; s_nb[warp] = nb; }
        __syncthreads();
        if (warp != 0) return;
        lo = lane < nw ? s_lo[lane] : LLONG_MAX;
        hi = lane < nw ? s_hi[lane] : LLONG_MIN;
        ns = lane < nw ? s_ns[lane] : 0;
        nb = lane < nw ? s_nb[lane] : 0;
    }
    if (threadIdx.x == 0) {
        if (lo != LLONG_MAX) atomicMin(&st->tmin, lo);
        if (hi != LLONG_MIN) atomicMax(&st->tmax, hi);
        if (ns) atomicAdd(&st->nself, ns);
        if (nb) atomicAdd(&st->nbad, nb);
    }
}

// Elementwise kernels below take kElemItems elements per thread (i, i +
// blockDim, ...): with one element per thread the list offsets kernel
// measured twice as slow.
#ifndef TM_ELEM_ITEMS
#define TM_ELEM_ITEMS 4
#endif
constexpr int kElemItems = TM_ELEM_ITEMS;

// keep flags for self-loop dropping
__global__ void k_keep_nonself(const uint32_t *__restrict__ src, const uint32_t *__restrict__ dst, uint64_t m,
                               uint32_t *__restrict__ keep)
{
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) keep[i] = src[i] != dst[i] ? 1u : 0u;
}

// Compact the kept tuples into (t', src, dst) u32 arrays.
__global__ void k_compact_input(const uint32_t *__restrict__ src, const uint32_t *__restrict__ dst,
                                const int64_t *__restrict__ t, uint64_t m, const uint32_t *__restrict__ keep,
                                const uint32_t *__restrict__ pos, long long tmin, uint32_t *__restrict__ ot,
                                uint32_t *__restrict__ os, uint32_t *__restrict__ od)
{
    const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x * kElemItems + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kElemItems; ++k) {
        const uint64_t i = i0 + (uint64_t)k * blockDim.x;
        if (i >= m) break;
        if (keep && !keep[i]) continue;
        const uint32_t p = pos ? pos[i] : (uint32_t)i;
        ot[p] = (uint32_t)(t[i] - tmin);
        os[p] = src[i];
        od[p] = dst[i];
    }
}

// After the GLOBAL sort: flag tuples equal to their predecessor.
// After a sort by t' alone: order each run of equal t' by (src, dst), and
// count the tuples equal to their predecessor (repeats lie inside a run), so
// the flags above are made only when there are repeats.  Runs
// of up to kRunMax edges are sorted by their head's thread; runs of up to
// kBlockRunMax are listed (start, length) for k_order_long_runs; a longer run
// is flagged and the caller sorts by all three keys instead.
constexpr uint32_t kRunMax = 32;
constexpr uint32_t kBlockRunMax = 4096;
__device__ __forceinline__ void order_run_at(uint32_t i, const uint32_t *__restrict__ t, uint32_t *__restrict__ s,
                                             uint32_t *__restrict__ d, uint32_t m, uint32_t *__restrict__ too_long,
                                             uint2 *__restrict__ long_runs, uint32_t *__restrict__ n_long,
                                             unsigned long long *__restrict__ ndup)
{
    if (i >= m || (i > 0 && t[i - 1] == t[i])) return;   // run heads only
    const uint32_t ti = t[i];
    uint32_t j = i + 1;
    while (j < m && t[j] == ti && j - i < kRunMax) ++j;
    if (j < m && t[j] == ti) {
        while (j < m && t[j] == ti && j - i <= kBlockRunMax) ++j;
        if (j - i > kBlockRunMax) atomicOr(too_long, 1u);
        else long_runs[atomicAdd(n_long, 1u)] = make_uint2(i, j - i);   // at most m / 33 runs
        return;
    }
    const uint32_t len = j - i;
    if (len < 2) return;
    if (len <= 4) {
        // most runs: a 4-key sorting network in registers (missing keys
        // padded with the largest value, which stay at the end)
        uint64_t k0 = ((uint64_t)s[i] << 32) | d[i], k1 = ((uint64_t)s[i + 1] << 32) | d[i + 1];
        uint64_t k2 = len > 2 ? ((uint64_t)s[i + 2] << 32) | d[i + 2] : ~0ull;
        uint64_t k3 = len > 3 ? ((uint64_t)s[i + 3] << 32) | d[i + 3] : ~0ull;
        auto cswap = [](uint64_t &a, uint64_t &b) { const uint64_t lo = a < b ? a : b, hi = a < b ? b : a; a = lo; b = hi; };
        cswap(k0, k1); cswap(k2, k3); cswap(k0, k2); cswap(k1, k3); cswap(k1, k2);
        s[i] = (uint32_t)(k0 >> 32); d[i] = (uint32_t)k0;
        s[i + 1] = (uint32_t)(k1 >> 32); d[i + 1] = (uint32_t)k1;
        if (len > 2) { s[i + 2] = (uint32_t)(k2 >> 32); d[i + 2] = (uint32_t)k2; }
        if (len > 3) { s[i + 3] = (uint32_t)(k3 >> 32); d[i + 3] = (uint32_t)k3; }
        const uint32_t dups = (k0 == k1) + (len > 2 && k1 == k2) + (len > 3 && k2 == k3);
        if (dups) atomicAdd(ndup, (unsigned long long)dups);
        return;
    }
    uint64_t key[kRunMax];
    for (uint32_t k = 0; k < len; ++k) key[k] = ((uint64_t)s[i + k] << 32) | d[i + k];
    for (uint32_t k = 1; k < len; ++k) {   // insertion sort
        const uint64_t x = key[k];
        uint32_t q = k;
        while (q > 0 && key[q - 1] > x) { key[q] = key[q - 1]; --q; }
        key[q] = x;
    }
    uint32_t dups = 0;
    for (uint32_t k = 0; k < len; ++k) {
        s[i + k] = (uint32_t)(key[k] >> 32); d[i + k] = (uint32_t)key[k];
        dups += k > 0 && key[k] == key[k - 1];
    }
    if (dups) atomicAdd(ndup, (unsigned long long)dups);
}

__global__ void k_order_runs(const uint32_t *__restrict__ t, uint32_t *__restrict__ s, uint32_t *__restrict__ d,
                             uint32_t m, uint32_t *__restrict__ too_long, uint2 *__restrict__ long_runs,
                             uint32_t *__restrict__ n_long, unsigned long long *__restrict__ ndup)
{
    const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x * kElemItems + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kElemItems; ++k) {
        const uint64_t i = i0 + (uint64_t)k * blockDim.x;
        if (i >= m) break;
        order_run_at((uint32_t)i, t, s, d, m, too_long, long_runs, n_long, ndup);
    }
}

// One block per listed run (33 .. kBlockRunMax edges): bitonic sort of the
// (src, dst) keys in shared memory.  Blocks stride over the list, whose
// length is read on the device.
__global__ void __launch_bounds__(256) k_order_long_runs(uint32_t *__restrict__ s, uint32_t *__restrict__ d,
                                                         const uint2 *__restrict__ long_runs,
                                                         const uint32_t *__restrict__ n_long,
                                                         unsigned long long *__restrict__ ndup)
{
    __shared__ uint64_t key[kBlockRunMax];
    const uint32_t nl = *n_long;
    for (uint32_t r = blockIdx.x; r < nl; r += gridDim.x) {
        const uint2 run = long_runs[r];
        uint32_t P = 64;
        while (P < run.y) P <<= 1;
        for (uint32_t k = threadIdx.x; k < P; k += blockDim.x)
            key[k] = k < run.y ? (((uint64_t)s[run.x + k] << 32) | d[run.x + k]) : ~0ull;
        __syncthreads();
        for (uint32_t size = 2; size <= P; size <<= 1)
            for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
                for (uint32_t k = threadIdx.x; k < P; k += blockDim.x) {
                    const uint32_t l = k ^ stride;
                    if (l > k) {
                        const bool up = (k & size) == 0;
                        const uint64_t a = key[k], b = key[l];
                        if ((a > b) == up) { key[k] = b; key[l] = a; }
                    }
                }
                __syncthreads();
            }
        uint32_t dups = 0;
        for (uint32_t k = threadIdx.x; k < run.y; k += blockDim.x) {
            s[run.x + k] = (uint32_t)(key[k] >> 32);
            d[run.x + k] = (uint32_t)key[k];
            dups += k > 0 && key[k] == key[k - 1];
        }
        if (dups) atomicAdd(ndup, (unsigned long long)dups);
        __syncthreads();
    }
}

__global__ void k_flag_unique(const uint32_t *__restrict__ t, const uint32_t *__restrict__ s,
                              const uint32_t *__restrict__ d, uint32_t m, uint32_t *__restrict__ keep,
                              unsigned long long *ndup)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    bool dup = i > 0 && t[i] == t[i - 1] && s[i] == s[i - 1] && d[i] == d[i - 1];
    keep[i] = dup ? 0u : 1u;
    if (dup) atomicAdd(ndup, 1ull);
}

__global__ void k_compact3(const uint32_t *__restrict__ a, const uint32_t *__restrict__ b,
                           const uint32_t *__restrict__ c, uint32_t m, const uint32_t *__restrict__ keep,
                           const uint32_t *__restrict__ pos, uint32_t *__restrict__ oa, uint32_t *__restrict__ ob,
                           uint32_t *__restrict__ oc)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || !keep[i]) return;
    uint32_t p = pos[i];
    oa[p] = a[i]; ob[p] = b[i]; oc[p] = c[i];
}


// Owner-start bit sets of the out-, in- and multi-edge orders: position x
// starts a new owner when its source (out-lists) or destination (in-lists)
// differs from position x-1's, or when it heads a pair (multi-edge lists,
// from the pair-head flags).  One thread per position; each warp's ballots
// are one word of each set.
__global__ void k_owner_bits(const uint32_t *__restrict__ out_src, const uint32_t *__restrict__ in_dst,
                             const uint32_t *__restrict__ pair_head, uint32_t m, uint32_t words,
                             uint32_t *__restrict__ own_out, uint32_t *__restrict__ own_in,
                             uint32_t *__restrict__ own_multi)
{
    const uint64_t x0 = (uint64_t)blockIdx.x * blockDim.x * kElemItems + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kElemItems; ++k) {
        // a warp's 32 positions are consecutive and start at a multiple of 32,
        // and words * 32 is a multiple of 32: whole warps leave together
        const uint64_t x = x0 + (uint64_t)k * blockDim.x;
        if (x >= (uint64_t)words * 32) break;
        const bool in = x < m, first = x == 0;
        const bool bo = in && (first || out_src[x] != out_src[x - 1]);
        const bool bi = in && (first || in_dst[x] != in_dst[x - 1]);
        const bool bm = in && pair_head[x] != 0;
        const uint32_t wo = __ballot_sync(0xffffffffu, bo), wi = __ballot_sync(0xffffffffu, bi),
                       wm = __ballot_sync(0xffffffffu, bm);
        if ((threadIdx.x & 31) == 0) {
            own_out[x >> 5] = wo;
            own_in[x >> 5] = wi;
            own_multi[x >> 5] = wm;
        }
    }
}

// off[v] = first position whose sorted key is >= v, for v in [0, n].  With
// m_dev set, the key count is min(m, *m_dev) (a count known only on the
// device; m bounds the grid).
#ifndef TM_OFF_ITEMS
#define TM_OFF_ITEMS 8   // positions per thread (1: one per thread)
#endif
__global__ void k_offsets(const uint32_t *__restrict__ keys, uint32_t m, uint32_t n, uint32_t *__restrict__ off,
                          const uint32_t *__restrict__ m_dev)
{
    // positions [i0, i0 + TM_OFF_ITEMS) of this thread, the previous key carried
    const uint64_t i0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * TM_OFF_ITEMS;
    if (m_dev) m = min(m, *m_dev);
    if (i0 > m) return;
    uint32_t prev = i0 == 0 ? 0u : __ldg(keys + i0 - 1) + 1u;
#pragma unroll
    for (int j = 0; j < TM_OFF_ITEMS; ++j) {
        const uint64_t i = i0 + j;
        if (i > m) break;
        const uint32_t lo = prev;
        const uint32_t hi = (i == m) ? n : __ldg(keys + i);
        for (uint32_t v = lo; v <= hi && v <= n; ++v) off[v] = (uint32_t)i;
        prev = hi + 1u;
    }
}

// Pair heads in the multi-edge order (src from the sorted keys, dst gathered).
__global__ void k_pair_heads(const uint32_t *__restrict__ msrc, const uint32_t *__restrict__ mdst, uint32_t m,
                             uint32_t *__restrict__ head)
{
    const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x * kElemItems + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kElemItems; ++k) {
        const uint64_t i = i0 + (uint64_t)k * blockDim.x;
        if (i >= m) break;
        head[i] = (i == 0 || msrc[i] != msrc[i - 1] || mdst[i] != mdst[i - 1]) ? 1u : 0u;
    }
}

__global__ void k_pair_fill(const uint32_t *__restrict__ msrc, const uint32_t *__restrict__ mdst,
                            const uint32_t *__restrict__ head, const uint32_t *__restrict__ pid_excl, uint32_t m,
                            uint32_t *__restrict__ pair_off, uint32_t *__restrict__ pair_src,
                            uint32_t *__restrict__ pair_dst)
{
    const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x * kElemItems + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kElemItems; ++k) {
        const uint32_t i = (uint32_t)(i0 + (uint64_t)k * blockDim.x);
        if (i0 + (uint64_t)k * blockDim.x >= m) break;
        if (head[i]) {
            const uint32_t pid = pid_excl[i];
            pair_off[pid] = i;
            pair_src[pid] = msrc[i];
            pair_dst[pid] = mdst[i];
        }
        if (i == m - 1) pair_off[pid_excl[i] + head[i]] = m;   // the end of the last pair's list
    }
}

// where each list time falls in the same vertex's other list
// Cross ranks of both lists (blockIdx.y = 0: out-list entries into the
// owner's in-list; 1: in-list entries into the owner's out-list).
struct XR {
    const uint32_t *own_t, *owner, *other_off, *other_t;
    uint32_t *xrank;
};
// Two alternatives measured slower on 5e7 entries per list: letting the
// first and last lanes of a warp whose entries share one owner search first
// and the other lanes only the bracket those give (1.32 against 1.25 ms), and
// merging each vertex's two lists along a merge path in chunks of 128 entries
// per thread (1.44 ms: the chunk walk is one long chain of dependent loads).
// The independent searches keep the most loads in flight.
// Each thread runs TM_XR_ITEMS searches (entries i, i + stride, ...) in
// lockstep, so that many independent probes are in flight per thread.
#ifndef TM_XR_ITEMS
#define TM_XR_ITEMS 4
#endif
__global__ void k_cross_rank(XR a, XR b, uint32_t m)
{
    constexpr int K = TM_XR_ITEMS;
    const bool s1 = blockIdx.y != 0;
    const uint32_t *own_t = s1 ? b.own_t : a.own_t, *owner = s1 ? b.owner : a.owner;
    const uint32_t *other_off = s1 ? b.other_off : a.other_off, *other_t = s1 ? b.other_t : a.other_t;
    uint32_t *xrank = s1 ? b.xrank : a.xrank;
    const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x * K + threadIdx.x;
    uint32_t lo[K], len[K], key[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const uint64_t i = i0 + (uint64_t)k * blockDim.x;
        lo[k] = 0; len[k] = 0; key[k] = 0;
        if (i < m) {
            const uint32_t z = __ldg(owner + i);
            key[k] = __ldg(own_t + i);
            lo[k] = __ldg(other_off + z);
            len[k] = __ldg(other_off + z + 1) - lo[k];
        }
    }
    // the binary search of lower_idx, all K at once
    bool more = true;
    while (more) {
        more = false;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (len[k] > 0) {
                const uint32_t half = len[k] >> 1, mid = lo[k] + half;
                if (__ldg(other_t + mid) < key[k]) { lo[k] = mid + 1; len[k] -= half + 1; }
                else len[k] = half;
                more |= len[k] > 0;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const uint64_t i = i0 + (uint64_t)k * blockDim.x;
        if (i < m) xrank[i] = lo[k];
    }
}

inline unsigned blocks_for(uint64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

// Graph arrays come from a few large blocks (one allocator call each), cut
// into 256-byte aligned arrays.
struct GraphBlock {
    char *base = nullptr;
    size_t size = 0, off = 0;
};

static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

static bool gblock_open(tm_ctx *ctx, GraphBlock &b, size_t bytes)
{
    b.size = bytes ? bytes : 256;
    b.off = 0;
    b.base = (char *)dalloc(ctx, b.size);
    if (b.base) ctx->graph_bufs.push_back({b.base, b.size});
    return b.base != nullptr;
}

static uint32_t *gtake(GraphBlock &b, size_t count)
{
    size_t bytes = align256((count ? count : 1) * sizeof(uint32_t));
    if (b.off + bytes > b.size) return nullptr;
    uint32_t *p = (uint32_t *)(b.base + b.off);
    b.off += bytes;
    return p;
}

int build_csr(tm_ctx *ctx)
{
    ScratchScope scope(ctx);
    GraphBlock gb;
    cudaMemsetAsync(ctx->status, 0, 4, ctx->stream);
    const int TB = 256;
    cudaStream_t st = ctx->stream;
    uint64_t m0 = ctx->m_in;
    uint32_t n = ctx->n;
    DevGraph &g = ctx->g;
    g = DevGraph();
    g.n = n;
    int rc = TM_OK;
    // ---- statistics: t range, self loops, bad ids
    std::unique_ptr<PhaseScope> sec(new PhaseScope(ctx, TM_PH_CSR_STATS));
    Stats hs{LLONG_MAX, LLONG_MIN, 0, 0};
    Stats *ds = (Stats *)salloc(ctx, sizeof(Stats));
    if (!ds) return TM_E_NOMEM;
    copy_h2d(ctx, ds, &hs, sizeof(Stats));
    if (m0) {
        unsigned nb = std::min<uint64_t>(blocks_for(m0, TB), (uint64_t)ctx->num_sms * 8);
        launch(ctx, k_input_stats, nb, TB, ctx->in_src, ctx->in_dst, ctx->in_t, m0, n, ds);
    }
    copy_d2h(ctx, &hs, ds, sizeof(Stats));
    rc = check_cuda(ctx, cudaStreamSynchronize(st), "input statistics");
    if (rc) return rc;
    if (hs.nbad) return set_err(ctx, TM_E_ARG, "vertex id >= n in input");
    if (hs.nself && !(ctx->load_flags & TM_DROP_SELF))
        return set_err(ctx, TM_E_SELFLOOP, "input has self loops (pass TM_DROP_SELF to drop them)");
    uint64_t m1 = m0 - hs.nself;
    if (m1 >= 0xFFFFFFFFull) return set_err(ctx, TM_E_LIMIT, "more than 2^32-2 edges");
    long long tmin = m1 ? hs.tmin : 0, tmax = m1 ? hs.tmax : 0;
    // the span as an unsigned difference: no signed overflow at the int64 extremes
    if ((unsigned long long)tmax - (unsigned long long)tmin >= 0xFFFFFFFFull)
        return set_err(ctx, TM_E_LIMIT, "time span t_max - t_min must be below 2^32 - 1");
    uint32_t m = (uint32_t)m1;
    // ---- compact to (t', src, dst)
    uint32_t *T0 = (uint32_t *)salloc(ctx, (size_t)(m ? m : 1) * 4);
    uint32_t *S0 = (uint32_t *)salloc(ctx, (size_t)(m ? m : 1) * 4);
    uint32_t *D0 = (uint32_t *)salloc(ctx, (size_t)(m ? m : 1) * 4);
    if (!T0 || !S0 || !D0) return TM_E_NOMEM;
    if (hs.nself) {
        uint32_t *keep = (uint32_t *)salloc(ctx, m0 * 4), *pos = (uint32_t *)salloc(ctx, m0 * 4);
        if (!keep || !pos) return TM_E_NOMEM;
        launch(ctx, k_keep_nonself, blocks_for(m0, TB), TB, ctx->in_src, ctx->in_dst, m0, keep);
        rc = exclusive_scan_u32(ctx, keep, pos, m0, nullptr);
        if (rc) return rc;
        launch(ctx, k_compact_input, blocks_for((m0 + kElemItems - 1) / kElemItems, TB), TB, ctx->in_src, ctx->in_dst,
               ctx->in_t, m0, keep, pos, tmin, T0, S0, D0);
    } else if (m) {
        launch(ctx, k_compact_input, blocks_for((m0 + kElemItems - 1) / kElemItems, TB), TB, ctx->in_src, ctx->in_dst,
               ctx->in_t, m0, nullptr, nullptr, tmin, T0, S0, D0);
    }
    // every m- and n-sized array of the graph in one block, sized before the
    // duplicates are known (they are rare; their slots stay unused)
    {
        const size_t mf = (size_t)m, a_m = align256((mf ? mf : 1) * 4), a_n = align256(((size_t)n + 1) * 4);
        const size_t a_b = align256((mf / 32 + 1) * 4);
        // (the pair tables are sized by m too: the pair count is read only at the end)
        if (!gblock_open(ctx, gb, 20 * a_m + 256 + 3 * a_n + 3 * a_b)) return TM_E_NOMEM;
    }
    g.g_t = gtake(gb, m); g.g_src = gtake(gb, m); g.g_dst = gtake(gb, m);
    if (!g.g_t || !g.g_src || !g.g_dst) return TM_E_NOMEM;
    // ---- GLOBAL order (t', src, dst): LSD by t' straight into the graph's
    // arrays, then each run of equal t' ordered by (src, dst) in place; a run
    // longer than kBlockRunMax sends the whole array through the full LSD sort
    // by dst, src and t' instead
    sec.reset();
    sec.reset(new PhaseScope(ctx, TM_PH_CSR_GLOBAL));
    int vbits = bits_for(n ? n - 1 : 0);
    int tbits = bits_for((unsigned long long)tmax - (unsigned long long)tmin);
    {
        RsTo ts{T0, S0, D0, g.g_t, g.g_src, g.g_dst};
        rc = radix_sort_sets_to(ctx, &ts, 1, m, tbits);
        if (rc) return rc;
    }
    // ---- duplicates (and the run check, read with the same copy)
    {
        uint32_t *keep = (uint32_t *)salloc(ctx, (size_t)(m ? m : 1) * 4);
        // [0] duplicates, [1] a run too long, [2] number of listed runs
        unsigned long long *nd = (unsigned long long *)salloc(ctx, 24);
        uint2 *long_runs = (uint2 *)salloc(ctx, ((size_t)m / (kRunMax + 1) + 1) * sizeof(uint2));
        if (!keep || !nd || !long_runs) return TM_E_NOMEM;
        cudaMemsetAsync(nd, 0, 24, st);
        if (m) {
            launch(ctx, k_order_runs, blocks_for(((uint64_t)m + kElemItems - 1) / kElemItems, TB), TB,
                   (const uint32_t *)g.g_t, g.g_src, g.g_dst, m,
                   (uint32_t *)(nd + 1), long_runs, (uint32_t *)(nd + 2), nd);
            launch(ctx, k_order_long_runs, (unsigned)ctx->num_sms * 2, 256, g.g_src, g.g_dst, (const uint2 *)long_runs,
                   (const uint32_t *)(nd + 2), nd);
        }
        unsigned long long hnd[2] = {0, 0};
        copy_d2h(ctx, hnd, nd, 16);
        rc = check_cuda(ctx, cudaStreamSynchronize(st), "duplicate scan");
        if (rc) return rc;
        if (hnd[1]) {
            rc = radix_sort(ctx, g.g_dst, g.g_src, g.g_t, m, vbits);
            if (!rc) rc = radix_sort(ctx, g.g_src, g.g_dst, g.g_t, m, vbits);
            if (!rc) rc = radix_sort(ctx, g.g_t, g.g_src, g.g_dst, m, tbits);
            if (rc) return rc;
            cudaMemsetAsync(nd, 0, 8, st);
            launch(ctx, k_flag_unique, blocks_for(m, TB), TB, g.g_t, g.g_src, g.g_dst, m, keep, nd);
            copy_d2h(ctx, hnd, nd, 8);
            rc = check_cuda(ctx, cudaStreamSynchronize(st), "duplicate scan");
            if (rc) return rc;
        }
        const unsigned long long ndup = hnd[0];
        if (ndup && !(ctx->load_flags & TM_DEDUP)) {
            return set_err(ctx, TM_E_DUP, "input repeats a (u,v,t) tuple (pass TM_DEDUP to drop repeats)");
        }
        if (ndup && !hnd[1]) {   // the run kernels only counted the repeats: flag them (same count)
            cudaMemsetAsync(nd, 0, 8, st);
            launch(ctx, k_flag_unique, blocks_for(m, TB), TB, g.g_t, g.g_src, g.g_dst, m, keep, nd);
        }
        if (ndup) {
            // compact into the work arrays, then back
            uint32_t *pos = (uint32_t *)salloc(ctx, (size_t)m * 4);
            if (!pos) return TM_E_NOMEM;
            rc = exclusive_scan_u32(ctx, keep, pos, m, nullptr);
            if (rc) return rc;
            launch(ctx, k_compact3, blocks_for(m, TB), TB, g.g_t, g.g_src, g.g_dst, m, keep, pos, T0, S0, D0);
            const size_t bytes = (size_t)(m - ndup) * 4;
            cudaMemcpyAsync(g.g_t, T0, bytes, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(g.g_src, S0, bytes, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(g.g_dst, D0, bytes, cudaMemcpyDeviceToDevice, st);
        }
        m = (uint32_t)(m - ndup);
    }
    g.m = m;
    g.tmin = tmin;
    g.T = (uint32_t)((unsigned long long)tmax - (unsigned long long)tmin);
    // S0/D0/T0 are reused below as work space
    // ---- OUT and IN orders: stable sorts of gid by src and by dst, run as
    // one two-array sort; the sorted keys are out_src and in_dst themselves
    sec.reset();
    sec.reset(new PhaseScope(ctx, TM_PH_CSR_OUT));
    g.out_gid = gtake(gb, m); g.out_t = gtake(gb, m); g.out_nbr = gtake(gb, m); g.out_off = gtake(gb, (size_t)n + 1);
    g.in_gid = gtake(gb, m); g.in_t = gtake(gb, m); g.in_nbr = gtake(gb, m); g.in_off = gtake(gb, (size_t)n + 1);
    g.out_src = gtake(gb, m); g.in_dst = gtake(gb, m);
    g.out_xrank = gtake(gb, m); g.in_xrank = gtake(gb, m); g.out_pos = gtake(gb, m); g.in_pos = gtake(gb, m);
    if (!g.out_gid || !g.out_t || !g.out_nbr || !g.out_off || !g.in_gid || !g.in_t || !g.in_nbr || !g.in_off ||
        !g.out_src || !g.in_dst || !g.out_xrank || !g.in_xrank || !g.out_pos || !g.in_pos)
        return TM_E_NOMEM;
    g.in_to_out = gtake(gb, m);
    if (!g.in_to_out) return TM_E_NOMEM;
    if (m) {
        // payloads: the input index (gid), t' and the other endpoint, so every
        // list array comes out of the sort (no gathers); the last pass also
        // writes each edge's list position by gid (the inverse permutation).
        // The in-list sort then carries each edge's out-list position (read in
        // GLOBAL order), which gives the in -> out map directly.
        RsTo os{g.g_src, nullptr, g.g_t, g.out_src, g.out_gid, g.out_t};
        os.p2_in = g.g_dst; os.p2 = g.out_nbr; os.inv = g.out_pos;
        rc = radix_sort_sets_to(ctx, &os, 1, m, vbits);
        if (rc) return rc;
        RsTo is{g.g_dst, nullptr, g.g_t, g.in_dst, g.in_gid, g.in_t};
        is.p2_in = g.g_src; is.p2 = g.in_nbr; is.p3_in = g.out_pos; is.p3 = g.in_to_out; is.inv = g.in_pos;
        rc = radix_sort_sets_to(ctx, &is, 1, m, vbits);
        if (rc) return rc;
    }
    sec.reset();
    sec.reset(new PhaseScope(ctx, TM_PH_CSR_IN));
    launch(ctx, k_offsets, blocks_for(((uint64_t)m + TM_OFF_ITEMS) / TM_OFF_ITEMS, TB), TB, g.out_src, m, n, g.out_off, nullptr);
    launch(ctx, k_offsets, blocks_for(((uint64_t)m + TM_OFF_ITEMS) / TM_OFF_ITEMS, TB), TB, g.in_dst, m, n, g.in_off, nullptr);
    uint32_t *key = S0, *tmp = D0;
    // ---- multi-edge order: stable re-sort of the IN order by source
    sec.reset();
    sec.reset(new PhaseScope(ctx, TM_PH_CSR_MULTI));
    g.multi_t = gtake(gb, m);
    g.multi_to_out = gtake(gb, m);
    g.vpair_off = gtake(gb, (size_t)n + 1);
    g.own_out = gtake(gb, (size_t)m / 32 + 1); g.own_in = gtake(gb, (size_t)m / 32 + 1);
    g.own_multi = gtake(gb, (size_t)m / 32 + 1);
    if (!g.multi_t || !g.vpair_off || !g.multi_to_out || !g.own_out || !g.own_in || !g.own_multi)
        return TM_E_NOMEM;
    uint32_t np = 0;
    if (m) {
        {
            // payloads: t', the destination and each entry's out-list
            // position, straight into the multi-edge arrays
            RsTo ms{g.in_nbr, g.in_t, g.in_dst, key, g.multi_t, tmp};
            ms.p2_in = g.in_to_out;
            ms.p2 = g.multi_to_out;
            rc = radix_sort_sets_to(ctx, &ms, 1, m, vbits);
            if (rc) return rc;
        }
        // key = pair src, tmp = pair dst per multi position
        uint32_t *head = T0;
        uint32_t *pid = (uint32_t *)salloc(ctx, (size_t)m * 4);
        uint32_t *dnp = (uint32_t *)salloc(ctx, 4);
        if (!pid || !dnp) return TM_E_NOMEM;
        launch(ctx, k_pair_heads, blocks_for(((uint64_t)m + kElemItems - 1) / kElemItems, TB), TB, key, tmp, m, head);
        rc = exclusive_scan_u32(ctx, head, pid, m, dnp);
        if (rc) return rc;
        // dnp = the number of pairs (the scan's total), used on the device;
        // the pair tables are m-sized slots of the graph block
        g.pair_off = gtake(gb, (size_t)m + 1);
        g.pair_dst = gtake(gb, m);
        uint32_t *pair_src = (uint32_t *)salloc(ctx, (size_t)m * 4);
        if (!g.pair_off || !g.pair_dst || !pair_src) return TM_E_NOMEM;
        launch(ctx, k_pair_fill, blocks_for(((uint64_t)m + kElemItems - 1) / kElemItems, TB), TB, (const uint32_t *)key,
               (const uint32_t *)tmp,
               (const uint32_t *)head, (const uint32_t *)pid, m, g.pair_off, pair_src, g.pair_dst);
        launch(ctx, k_offsets, blocks_for(((uint64_t)m + TM_OFF_ITEMS) / TM_OFF_ITEMS, TB), TB, pair_src, m, n, g.vpair_off, (const uint32_t *)dnp);
        copy_d2h(ctx, ctx->status_host + 1, dnp, 4);   // pinned: read after the closing synchronize
        // cross ranks between a vertex's out- and in-lists
        launch(ctx, k_cross_rank, dim3(blocks_for(((uint64_t)m + TM_XR_ITEMS - 1) / TM_XR_ITEMS, TB), 2), TB,
               XR{g.out_t, g.out_src, g.in_off, g.in_t, g.out_xrank},
               XR{g.in_t, g.in_dst, g.out_off, g.out_t, g.in_xrank}, m);
        // owner starts of the three orders (segment heads of the weight pass's scans)
        const uint32_t words = m / 32 + 1;
        launch(ctx, k_owner_bits, blocks_for(((uint64_t)words * 32 + kElemItems - 1) / kElemItems, TB), TB,
               (const uint32_t *)g.out_src, (const uint32_t *)g.in_dst,
               (const uint32_t *)head, m, words, g.own_out, g.own_in, g.own_multi);
    } else {
        GraphBlock pbk;
        if (!gblock_open(ctx, pbk, 3 * 256)) return TM_E_NOMEM;
        g.pair_off = gtake(pbk, 1);
        g.pair_dst = gtake(pbk, 1);
        cudaMemsetAsync(g.pair_off, 0, 4, st);
        launch(ctx, k_offsets, 1, TB, key, 0, n, g.vpair_off, nullptr);
    }
    uint32_t bits = 0;
    int rc2 = read_status(ctx, &bits);   // the build's one closing synchronize
    if (rc2) return rc2;
    if (m) np = ctx->status_host[1];
    g.npairs = np;
    if (bits) return set_err(ctx, TM_E_CUDA, "CSR build: device status " + std::to_string(bits));
    return TM_OK;
}

}  // namespace timest
