"""Constraint toggles of the ablation on the GPU: with Constraint 2 and/or
Constraint 3 dropped, every weight, the window totals, W, the per-sample
trees, reasons and contributions, hits2 and the reject counters equal the
oracle's under the same setting (bit-exact)."""
import numpy as np
import pytest

from helpers import SMALL_MOTIFS, small_random_graph, spanning_trees

pytestmark = pytest.mark.gpu

SETS = [(True, True), (False, True), (True, False), (False, False)]


def _case(ctx, G, nv, edges, rank, delta, tree, root, c2, c3, k=4000, seed=3):
    mo = ctx.motif(nv, edges, rank, delta).set_tree(tree, root).set_constraints(c2, c3)
    G.set_motif(nv, edges, rank, delta, tree, root)
    G.set_constraints(c2, c3)
    assert mo.weights() == G.weights()
    assert np.array_equal(mo.window_totals(), G.window_totals())
    for e in tree:
        for layer in (0, 1):
            assert np.array_equal(mo.export_weights(e, layer), G.export_weights(e, layer)), (e, layer)
    rg, tg_, cg, wg = mo.sample_trace(k, seed)
    ro, to_, co, wo = G.sample(k, seed, trace=True)
    assert np.array_equal(tg_, to_) and np.array_equal(wg, wo) and np.array_equal(cg, co)
    assert (rg.W, rg.hits2, rg.valid, rg.rej_vertex, rg.rej_delta, rg.rej_order) == \
           (ro.W, ro.hits2, ro.valid, ro.rej_vertex, ro.rej_delta, ro.rej_order)
    mo.free()
    return rg


@pytest.mark.parametrize("name", ["triangle", "cycle4", "cycle5_chord", "bowtie", "antiparallel", "in_star3"])
def test_small_motifs_every_constraint_set(oracle_mod, name):
    import paper_2507_20441_gb300 as tg
    tg.build()
    nv, edges, rank = SMALL_MOTIFS[name]
    n, s, d, t = small_random_graph(21, n=nv + 2, m=400, t_hi=300)
    ctx = tg.Context()
    ctx.load_graph(n, s, d, t)
    G = oracle_mod.Graph(n, s, d, t)
    for tree in spanning_trees(nv, edges)[:3]:
        for root in tree:
            for c2, c3 in SETS:
                _case(ctx, G, nv, edges, rank, 25, tree, root, c2, c3)
    ctx.close()


def test_chung_lu_ablation(oracle_mod):
    """The 4-cycle on a 200k-edge Chung-Lu graph under C1, C1+2 and C1+2+3
    (the paper's ablation), each equal to the oracle."""
    import paper_2507_20441_gb300 as tg
    from paper_2507_20441_gb300 import synth
    gr = synth.chung_lu_bursty(5000, 200_000, 2.1, 3_000_000, seed=3)
    ctx = tg.Context()
    ctx.load_graph(gr.n, gr.src, gr.dst, gr.t)
    G = oracle_mod.Graph(gr.n, gr.src, gr.dst, gr.t)
    nv, edges, rank = SMALL_MOTIFS["cycle4"]
    W = {}
    for c2, c3 in [(False, False), (True, False), (True, True)]:
        r = _case(ctx, G, nv, edges, rank, 86_400, [0, 1, 2], 1, c2, c3, k=50_000, seed=4)
        W[(c2, c3)] = r.W
    # Constraint 2 only removes partial matches: its candidate lists are subsets
    assert W[(True, False)] <= W[(False, False)]
    ctx.close()


def test_toggles_invalidate_weights_and_reject_unknown_flags():
    import paper_2507_20441_gb300 as tg
    n, s, d, t = small_random_graph(5, n=8, m=200, t_hi=100)
    ctx = tg.Context()
    ctx.load_graph(n, s, d, t)
    nv, edges, rank = SMALL_MOTIFS["cycle4"]
    mo = ctx.motif(nv, edges, rank, 20)
    mo.weights()
    mo.set_constraints(False, True)
    with pytest.raises(tg.TimestError) as e:
        mo.sample(100, 1)
    assert e.value.code == tg.TM_E_STATE
    rc = tg.lib().tm_set_constraints(mo.h, 4)
    assert rc == tg.TM_E_ARG
    ctx.close()
