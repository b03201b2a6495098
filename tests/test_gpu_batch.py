"""Batched estimation (many (motif, delta, k) queries in one persistent
launch): every query's result is bit-identical to the CPU oracle's TIMEST
(Alg. 3-6) on the same tree, k and seed, and to its own tm_sample call, for
uneven sample counts, any tile size, k = 0 and motifs with W = 0."""
import pytest

from helpers import default_tree, oracle_result, result_tuple

pytestmark = pytest.mark.gpu


def _graph():
    from paper_2507_20441_gb300 import synth
    return synth.chung_lu_bursty(20_000, 400_000, 2.1, 6_000_000, seed=11)


def _context(tg, tile):
    gr = _graph()
    ctx = tg.Context(sample_tile=tile)
    ctx.load_graph(gr.n, gr.src, gr.dst, gr.t)
    return ctx


@pytest.fixture(scope="module")
def pool():
    import paper_2507_20441_gb300 as tg
    from paper_2507_20441_gb300 import synth
    tg.build()
    return synth.motif_pool(seed=3, count=32, k_lo=1e3, k_hi=2e5)


@pytest.mark.parametrize("tile", [0, 256, 1000, 8192])
def test_batch_equals_separate_runs(pool, tile):
    import paper_2507_20441_gb300 as tg
    ctx = _context(tg, tile)
    motifs = []
    for mo in pool:
        m = ctx.motif(mo.nv, mo.edges, mo.rank, mo.delta)
        m.weights()
        motifs.append(m)
    ks = [mo.k for mo in pool]
    ks[3] = 0
    ks[5] = 1
    seeds = [100 + i for i in range(len(pool))]
    res = ctx.batch_run(motifs, ks, seeds)
    for m, mo, k, s, r in zip(motifs, pool, ks, seeds, res):
        ref = m.sample(k, s)
        assert (r.W, r.hits2, r.k, r.valid, r.rej_vertex, r.rej_delta, r.rej_order) == \
               (ref.W, ref.hits2, ref.k, ref.valid, ref.rej_vertex, ref.rej_delta, ref.rej_order), mo.name
        assert r.estimate == ref.estimate
    ctx.close()


def test_batch_equals_oracle(pool, oracle_mod):
    """Each of 32 queries (3-7 vertices, three deltas, k from 1e3 to 2e5) of
    one batched launch against the oracle on the default tree: W, hits2 and
    the four counters bit for bit (Alg. 6 per query)."""
    import paper_2507_20441_gb300 as tg
    gr = _graph()
    ctx = _context(tg, 1000)
    G = oracle_mod.Graph(gr.n, gr.src, gr.dst, gr.t)
    motifs = []
    for mo in pool:
        m = ctx.motif(mo.nv, mo.edges, mo.rank, mo.delta)
        m.weights()
        motifs.append(m)
    ks = [mo.k for mo in pool]
    seeds = [300 + i for i in range(len(pool))]
    res = ctx.batch_run(motifs, ks, seeds)
    nonzero = 0
    for mo, k, s, r in zip(pool, ks, seeds, res):
        tree, root = default_tree(mo.nv, mo.edges, mo.rank)
        want = oracle_result(G, mo.nv, mo.edges, mo.rank, mo.delta, tree, root, k, s)
        assert result_tuple(r) == want, mo.name
        assert r.k == k
        nonzero += want[1] > 0
    assert nonzero >= 8                              # the comparison is not vacuous
    G.close()
    ctx.close()


def test_batch_with_empty_weights(pool):
    """A query with W = 0 (a triangle on a graph without one) runs next to a
    query with samples and gets zero hits, as tm_sample gives."""
    import numpy as np
    import paper_2507_20441_gb300 as tg
    ctx = tg.Context()
    src = np.array([0, 2], np.uint32)              # two disjoint edges: no 2-path,
    dst = np.array([1, 3], np.uint32)              # so no partial match of any
    t = np.array([10, 20], np.int64)               # triangle tree
    ctx.load_graph(5, src, dst, t)
    m0 = ctx.motif(3, [(0, 1), (1, 2), (2, 0)], [0, 1, 2], 100)
    assert m0.weights() == 0
    m1 = ctx.motif(2, [(0, 1)], [0], 15)
    assert m1.weights() > 0
    res = ctx.batch_run([m0, m1], [5000, 7000], [1, 2])
    assert res[0].hits2 == 0 and res[0].W == 0 and res[0].valid == 0 and res[0].estimate == 0.0
    ref = m1.sample(7000, 2)
    assert (res[1].hits2, res[1].valid, res[1].W) == (ref.hits2, ref.valid, ref.W)
    ctx.close()


@pytest.mark.parametrize("threads,smem", [(128, 0), (128, 1), (256, 0), (256, 1)])
def test_every_batch_shape_gives_the_same_results(pool, threads, smem):
    import paper_2507_20441_gb300 as tg
    ctx = _context(tg, 0)
    tg.tm_batch_shape(ctx.h, 1000, threads, smem)
    motifs = []
    for mo in pool[:12]:
        m = ctx.motif(mo.nv, mo.edges, mo.rank, mo.delta)
        m.weights()
        motifs.append(m)
    ks = [mo.k for mo in pool[:12]]
    seeds = [7 + i for i in range(12)]
    res = ctx.batch_run(motifs, ks, seeds)
    for m, k, s, r in zip(motifs, ks, seeds, res):
        ref = m.sample(k, s)
        assert (r.hits2, r.valid, r.rej_vertex, r.rej_delta, r.rej_order) == \
               (ref.hits2, ref.valid, ref.rej_vertex, ref.rej_delta, ref.rej_order)
    ctx.close()


def test_autotune_picks_the_fastest_measured_shape(pool):
    import paper_2507_20441_gb300 as tg
    ctx = _context(tg, 0)
    motifs = []
    for mo in pool:
        m = ctx.motif(mo.nv, mo.edges, mo.rank, mo.delta)
        m.weights()
        motifs.append(m)
    ks = [mo.k for mo in pool]
    seeds = [100 + i for i in range(len(pool))]
    best, table = ctx.autotune(motifs, ks, seeds, target_samples=500_000)
    assert len(table) == 48
    assert best["ms"] == min(e["ms"] for e in table)
    assert best["tile"] in (512, 1024, 2048, 4096, 8192, 16384) and best["threads"] in (128, 256)
    assert {e["coop_min"] for e in table} == {0, 256} and best["coop_min"] in (0, 256)
    res = ctx.batch_run(motifs, ks, seeds)          # runs with the tuned shape
    for m, k, s, r in zip(motifs, ks, seeds, res):
        ref = m.sample(k, s)
        assert (r.hits2, r.valid) == (ref.hits2, ref.valid)
    ctx.close()
