// Autotuner of the batched sampler: tile size, threads per block and where
// the per-sample records live.  Every candidate draws the same samples (a
// sample's outcome depends only on its seed and id), so tuning changes speed
// only, never a result.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "tm_internal.h"

using namespace timest;

extern "C" int tm_autotune(tm_ctx *ctx, uint32_t nq, tm_motif *const *motifs, const uint64_t *k, const uint64_t *seed,
                           uint64_t target_samples, tm_tune_entry *table, uint32_t table_cap, uint32_t *nentries,
                           tm_tune_entry *best)
{
    if (!ctx || nq == 0 || !motifs || !k || !seed) return TM_E_ARG;
    for (uint32_t q = 0; q < nq; ++q)
        if (!motifs[q] || motifs[q]->ctx != ctx || !motifs[q]->have_weights || motifs[q]->graph_epoch != ctx->epoch)
            return set_err(ctx, TM_E_STATE, "autotune needs weights for every motif");
    cudaSetDevice(ctx->device);
    if (target_samples == 0) target_samples = 4000000;
    uint64_t total = 0;
    for (uint32_t q = 0; q < nq; ++q) total += k[q];
    const double scale = total > target_samples ? (double)target_samples / (double)total : 1.0;
    std::vector<BatchItem> items(nq);
    for (uint32_t q = 0; q < nq; ++q) {
        uint64_t kq = (uint64_t)((double)k[q] * scale);
        if (k[q] && kq < 256) kq = std::min<uint64_t>(k[q], 256);
        items[q] = BatchItem{motifs[q], seed[q], 0, kq};
    }
    std::vector<SampleAcc> acc(nq);
    const int tiles[] = {512, 1024, 2048, 4096, 8192, 16384};
    const int threads[] = {128, 256};
    const int staging[] = {0, 1};
    // lanes on one long search: 1 (every search per lane), or the warp's
    // active lanes together on searches of at least 256 entries
    const int coops[] = {0, 256};
    const int keep_threads = ctx->batch_threads, keep_smem = ctx->batch_smem_recs;
    const uint32_t keep_coop = ctx->coop_min;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return check_cuda(ctx, cudaGetLastError(), "autotune events");
    tm_tune_entry bestv{0, 0, 0, 0, 0.0};
    uint32_t cnt = 0;
    int rc = TM_OK;
    // warm-up launch (loads the kernels, touches the graph)
    ctx->batch_threads = 256;
    ctx->batch_smem_recs = 0;
    rc = run_batch_items(ctx, items.data(), nq, 2048, acc.data(), 0);
    for (int co : coops)
    for (int th : threads)
        for (int sm : staging)
            for (int tl : tiles) {
                if (rc) break;
                ctx->batch_threads = th;
                ctx->batch_smem_recs = sm;
                ctx->coop_min = co ? (uint32_t)co : 0xFFFFFFFFu;
                float best_ms = 1e30f;
                for (int rep = 0; rep < 2 && rc == TM_OK; ++rep) {
                    cudaEventRecord(e0, ctx->stream);
                    rc = run_batch_items(ctx, items.data(), nq, (uint32_t)tl, acc.data(), 0);
                    cudaEventRecord(e1, ctx->stream);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    best_ms = std::min(best_ms, ms);
                }
                tm_tune_entry ent{tl, th, sm, co, (double)best_ms};
                if (table && cnt < table_cap) table[cnt] = ent;
                ++cnt;
                if (bestv.tile == 0 || ent.ms < bestv.ms) bestv = ent;
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        ctx->batch_threads = keep_threads;
        ctx->batch_smem_recs = keep_smem;
        ctx->coop_min = keep_coop;
        return rc;
    }
    ctx->cfg.sample_tile = bestv.tile;
    ctx->batch_threads = bestv.threads;
    ctx->batch_smem_recs = bestv.smem_records;
    ctx->coop_min = bestv.coop_min ? (uint32_t)bestv.coop_min : 0xFFFFFFFFu;
    if (nentries) *nentries = cnt;
    if (best) *best = bestv;
    return TM_OK;
}

extern "C" int tm_batch_shape(tm_ctx *ctx, int tile, int threads, int smem_records)
{
    if (!ctx || tile < 0 || (threads != 0 && threads != 128 && threads != 256) || smem_records < 0 || smem_records > 1)
        return TM_E_ARG;
    ctx->cfg.sample_tile = tile;
    ctx->batch_threads = threads ? threads : 256;
    ctx->batch_smem_recs = smem_records;
    return TM_OK;
}

extern "C" int tm_coop_search(tm_ctx *ctx, uint32_t min_entries)
{
    if (!ctx) return TM_E_ARG;
    ctx->coop_min = min_entries ? min_entries : 0xFFFFFFFFu;
    return TM_OK;
}
