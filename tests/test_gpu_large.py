"""Parity on the bench workload at full size (Chung-Lu, n = 2e6, m = 5e7,
span 1e8 s, 5-cycle + chord, delta = 3,600, k = 1e7) with the default tree:
W, every W_i, every weight of every tree edge in both layers; hits2 and the
counters of the whole k = 1e7 run in the launch bench.py times (one
tm_sample, the register-record sampler) against the oracle's 1e7 samples;
and the per-sample outcome of 200 sample ids drawn from a 1e7-sample traced
launch, each recomputed alone by the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_large_workload(oracle_mod):
    import paper_2507_20441_gb300 as tg
    from paper_2507_20441_gb300 import synth
    tg.build()
    gr = synth.make_graph("cl50m_cycle5chord")
    mo = synth.make_motif("cl50m_cycle5chord")
    ctx = tg.Context()
    ctx.load_graph(gr.n, gr.src, gr.dst, gr.t)
    m = ctx.motif(mo.nv, mo.edges, mo.rank, mo.delta)
    order, _ = m.plan()
    tree = sorted(int(x) for x in order)
    root = int(order[0])
    W = m.weights()
    G = oracle_mod.Graph(gr.n, gr.src, gr.dst, gr.t)
    del gr
    G.set_motif(mo.nv, mo.edges, mo.rank, mo.delta, tree, root)
    assert G.weights() == W
    assert np.array_equal(m.window_totals(), G.window_totals())
    for e in tree:
        for layer in (0, 1):
            assert np.array_equal(m.export_weights(e, layer), G.export_weights(e, layer)), (e, layer)
    k = mo.k
    r = m.sample(k, 3)                 # the bench's launch: k = 1e7 in one tm_sample
    ro = G.sample(k, 3)
    assert (r.hits2, r.valid, r.rej_vertex, r.rej_delta, r.rej_order) == \
           (ro.hits2, ro.valid, ro.rej_vertex, ro.rej_delta, ro.rej_order)
    assert r.valid > 0
    res, gids, contrib, reason = m.sample_trace(k, 1)
    rng = np.random.default_rng(1)
    for j in rng.choice(k, size=200, replace=False):
        r1, g1, c1, w1 = G.sample(1, 1, first=int(j), trace=True)
        assert np.array_equal(g1[0], gids[j]) and int(c1[0]) == int(contrib[j]) and int(w1[0]) == int(reason[j]), j
    ctx.close()
