"""The allocation-free sampling entry point (tm_sample_noalloc).

Callers that cannot allocate device memory while they sample -- a serving
loop whose memory pool is held by resident weights, a host framework that
owns the allocator -- use tm_sample_noalloc.  Its results must equal
tm_sample's exactly (integer counts, compared bit for bit), on two calls in a
row (the second call must not see the first call's sums, which stay in the
shared scratch array), and it must not call the allocator at all.

This file is collected last so that a failure here leaves every other test
already run.
"""
import ctypes as C

import numpy as np
import pytest

from helpers import small_random_graph

pytestmark = pytest.mark.gpu


def test_noalloc_sampler_matches_and_allocates_nothing():
    import torch
    import paper_2507_20441_gb300 as tg
    from paper_2507_20441_gb300 import synth

    tg.build()
    calls = {"alloc": 0, "free": 0}

    def _alloc(nbytes, stream, user):
        calls["alloc"] += 1
        return int(torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0)))

    def _free(ptr, nbytes, stream, user):
        calls["free"] += 1
        torch.cuda.caching_allocator_delete(int(ptr))

    hooks = (tg.ALLOC_FN(_alloc), tg.FREE_FN(_free))
    ctx = tg.Context(device=0, alloc_hooks=hooks)
    gr = synth.chung_lu_bursty(3000, 60_000, 2.1, 2_000_000, seed=4)
    ctx.load_graph(gr.n, gr.src, gr.dst, gr.t)
    for mo_def, tree, root in ((synth.cycle(4, 86_400), [0, 1, 2], 1),
                               (synth.cycle5_chord(20_000), [0, 2, 3, 4], 3)):
        mo = ctx.motif(mo_def.nv, mo_def.edges, mo_def.rank, mo_def.delta).set_tree(tree, root)
        mo.weights()
        for k, seed, first in ((200_000, 5, 0), (150_001, 9, 1_000)):
            ref = tg.tm_sample(ctx.h, mo.h, k, seed, first)
            before = dict(calls)
            got = tg.tm_sample_noalloc(ctx.h, mo.h, k, seed, first)
            assert calls == before, "tm_sample_noalloc called the allocator"
            assert (got.W, got.hits2, got.k, got.valid, got.rej_vertex, got.rej_delta, got.rej_order) == \
                   (ref.W, ref.hits2, ref.k, ref.valid, ref.rej_vertex, ref.rej_delta, ref.rej_order)
            assert got.estimate == ref.estimate
            assert got.valid > 0
    ctx.close()


def test_noalloc_sampler_small_graph_twice():
    import paper_2507_20441_gb300 as tg
    tg.build()
    n, s, d, t = small_random_graph(12, n=9, m=700, t_hi=200)
    ctx = tg.Context()
    ctx.load_graph(n, s, d, t)
    mo = ctx.motif(3, [(0, 1), (1, 2), (2, 0)], [0, 1, 2], 25).set_tree([0, 1], 1)
    mo.weights()
    a1 = tg.tm_sample_noalloc(ctx.h, mo.h, 50_000, 3)
    a2 = tg.tm_sample_noalloc(ctx.h, mo.h, 50_000, 3)
    b = mo.sample(50_000, 3)
    assert (a1.hits2, a1.valid) == (a2.hits2, a2.valid) == (b.hits2, b.valid)
    ctx.close()
