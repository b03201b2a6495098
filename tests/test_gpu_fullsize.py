"""Parity at the full size of the 2M-edge workload (Chung-Lu, n = 1e5,
m = 2e6, temporal 4-cycle, delta = 86,400, k = 1e6) in the launch shape
bench.py times for it (default tree, one tm_sample of k = 1e6 samples):

* every weight of every tree edge in both layers, W and every W_i equal the
  oracle's (the oracle computes them all in seconds);
* hits2 and the reject counters of the whole 1e6-sample run equal the
  oracle's (same Philox streams, all host cores);
* a random subset of sample ids, traced by the CUDA path inside the same
  1e6-sample launch, equals the oracle's outcome for each id computed alone.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_bench_workload_full_size(oracle_mod):
    import paper_2507_20441_gb300 as tg
    from paper_2507_20441_gb300 import synth
    tg.build()
    gr = synth.make_graph("cl2m_cycle4")
    mo = synth.make_motif("cl2m_cycle4")
    ctx = tg.Context()
    ctx.load_graph(gr.n, gr.src, gr.dst, gr.t)
    m = ctx.motif(mo.nv, mo.edges, mo.rank, mo.delta)
    order, parent = m.plan()
    tree = sorted(int(x) for x in order)
    root = int(order[0])
    W = m.weights()

    G = oracle_mod.Graph(gr.n, gr.src, gr.dst, gr.t)
    G.set_motif(mo.nv, mo.edges, mo.rank, mo.delta, tree, root)
    assert G.weights() == W
    assert np.array_equal(m.window_totals(), G.window_totals())
    for e in tree:
        for layer in (0, 1):
            assert np.array_equal(m.export_weights(e, layer), G.export_weights(e, layer)), (e, layer)

    k, seed = mo.k, 1
    res, gids, contrib, reason = m.sample_trace(k, seed)
    ro = G.sample(k, seed)
    assert (res.hits2, res.valid, res.rej_vertex, res.rej_delta, res.rej_order) == \
           (ro.hits2, ro.valid, ro.rej_vertex, ro.rej_delta, ro.rej_order)
    plain = m.sample(k, seed)           # the untraced launch bench.py times
    assert (plain.hits2, plain.valid) == (res.hits2, res.valid)
    rng = np.random.default_rng(0)
    for j in rng.choice(k, size=300, replace=False):
        r1, g1, c1, w1 = G.sample(1, seed, first=int(j), trace=True)
        assert np.array_equal(g1[0], gids[j]) and int(c1[0]) == int(contrib[j]) and int(w1[0]) == int(reason[j]), j
    ctx.close()
