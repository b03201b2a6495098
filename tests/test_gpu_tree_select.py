"""Tree and root selection by exact W (Alg. 7) on the GPU: every evaluated
(tree, root) candidate's W equals the oracle's W for that tree and root, the
winner is the least W under the documented tie rule (better-ranked tree, then
lower root edge), and the returned motif samples exactly like a motif pinned
to the same tree and root."""
import pytest

from helpers import SMALL_MOTIFS

pytestmark = pytest.mark.gpu


def _graph():
    from paper_2507_20441_gb300 import synth
    return synth.chung_lu_bursty(5000, 200_000, 2.1, 3_000_000, seed=3)


def _tree_of(mask):
    return [e for e in range(32) if mask >> e & 1]


@pytest.mark.parametrize("name,delta,n_c", [("cycle5_chord", 3600, 4), ("bowtie", 86_400, 3),
                                            ("cycle4", 86_400, 2), ("triangle", 20_000, 3)])
def test_selection_by_exact_w(oracle_mod, name, delta, n_c):
    import paper_2507_20441_gb300 as tg
    tg.build()
    nv, edges, order = SMALL_MOTIFS[name]
    gr = _graph()
    ctx = tg.Context()
    ctx.load_graph(gr.n, gr.src, gr.dst, gr.t)
    best, cands = ctx.select_tree(nv, edges, order, delta, n_c=n_c, all_roots=True)
    ranked = tg.tm_tree_candidates(nv, edges, order)[:n_c]
    # evaluation order: ranked trees, each with every tree edge as root in increasing id
    expect_order = [(mask, r) for mask, _ in ranked for r in _tree_of(mask)]
    assert [(c["tree_mask"], c["root"]) for c in cands] == expect_order
    G = oracle_mod.Graph(gr.n, gr.src, gr.dst, gr.t)
    for c in cands:
        assert c["status"] == tg.TM_OK
        G.set_motif(nv, edges, order, delta, _tree_of(c["tree_mask"]), c["root"])
        assert c["W"] == G.weights(), c
    win = min(range(len(cands)), key=lambda i: (cands[i]["W"], i))
    order_b, _ = best.plan()
    assert sorted(int(x) for x in order_b) == _tree_of(cands[win]["tree_mask"])
    assert int(order_b[0]) == cands[win]["root"]
    # the winner samples like a motif pinned to the same tree and root
    pinned = ctx.motif(nv, edges, order, delta).set_tree(_tree_of(cands[win]["tree_mask"]), cands[win]["root"])
    assert pinned.weights() == cands[win]["W"]
    a, b = best.sample(20_000, 11), pinned.sample(20_000, 11)
    assert (a.W, a.hits2, a.valid, a.rej_vertex, a.rej_delta, a.rej_order) == \
           (b.W, b.hits2, b.valid, b.rej_vertex, b.rej_delta, b.rej_order)
    ctx.close()


def test_single_candidate_default_root_is_the_default_plan():
    import paper_2507_20441_gb300 as tg
    nv, edges, order = SMALL_MOTIFS["cycle5_chord"]
    gr = _graph()
    ctx = tg.Context()
    ctx.load_graph(gr.n, gr.src, gr.dst, gr.t)
    best, cands = ctx.select_tree(nv, edges, order, 3600, n_c=1, all_roots=False)
    default = ctx.motif(nv, edges, order, 3600)
    assert len(cands) == 1
    assert [int(x) for x in best.plan()[0]] == [int(x) for x in default.plan()[0]]
    assert cands[0]["W"] == default.weights()
    ctx.close()
