"""Warp-cooperative searches (tm_coop_search): a sample whose candidate-list
pick or pair-list search spans at least the threshold is searched by all
active lanes of its warp together.  The draws and every comparison are the
same, so results must equal the CPU oracle's TIMEST (Alg. 3-6) bit for bit
at every threshold, in the plain, traced and batched samplers."""
import numpy as np
import pytest

from helpers import default_tree, oracle_result, result_tuple

pytestmark = pytest.mark.gpu

MOTIFS = [
    ("cycle4", 4, [(0, 1), (1, 2), (2, 3), (3, 0)], [0, 1, 2, 3]),
    ("triangle", 3, [(0, 1), (1, 2), (2, 0)], [0, 1, 2]),
    ("cycle5_chord", 5, [(0, 1), (1, 2), (0, 2), (2, 3), (3, 4), (4, 0)], [0, 1, 2, 3, 4, 5]),
    ("out_star3", 4, [(0, 1), (0, 2), (0, 3)], [1, 0, 2]),
]


@pytest.fixture(scope="module")
def graph():
    from paper_2507_20441_gb300 import synth
    return synth.chung_lu_bursty(20_000, 400_000, 2.1, 6_000_000, seed=11)


@pytest.mark.parametrize("coop", [2, 16, 256])
def test_coop_search_equals_oracle(graph, coop, oracle_mod):
    import paper_2507_20441_gb300 as tg
    tg.build()
    ctx = tg.Context()
    ctx.load_graph(graph.n, graph.src, graph.dst, graph.t)
    ctx.coop_search(coop)
    G = oracle_mod.Graph(graph.n, graph.src, graph.dst, graph.t)
    nonzero = 0
    for name, nv, edges, rank in MOTIFS:
        m = ctx.motif(nv, edges, rank, 86_400)
        m.weights()
        tree, root = default_tree(nv, edges, rank)
        r = m.sample(200_000, 17)
        want = oracle_result(G, nv, edges, rank, 86_400, tree, root, 200_000, 17)
        assert result_tuple(r) == want, (name, coop)
        nonzero += want[1] > 0
        # the traced sampler: every sampled tree, reason and contribution
        rt, gids, contrib, why = m.sample_trace(20_000, 5)
        ro, go, co, wo = G.sample(20_000, 5, trace=True)
        assert np.array_equal(gids, go) and np.array_equal(contrib, co) and np.array_equal(why, wo), name
        m.free()
    assert nonzero >= 2
    G.close()
    ctx.close()


def test_coop_search_in_the_batched_sampler(graph, oracle_mod):
    import paper_2507_20441_gb300 as tg
    ctx = tg.Context()
    ctx.load_graph(graph.n, graph.src, graph.dst, graph.t)
    ctx.coop_search(8)
    G = oracle_mod.Graph(graph.n, graph.src, graph.dst, graph.t)
    motifs, ks, seeds = [], [], []
    for i, (name, nv, edges, rank) in enumerate(MOTIFS):
        m = ctx.motif(nv, edges, rank, 86_400)
        m.weights()
        motifs.append(m); ks.append(60_000 + 10_000 * i); seeds.append(90 + i)
    res = ctx.batch_run(motifs, ks, seeds)
    for (name, nv, edges, rank), k, s_, r in zip(MOTIFS, ks, seeds, res):
        tree, root = default_tree(nv, edges, rank)
        assert result_tuple(r) == oracle_result(G, nv, edges, rank, 86_400, tree, root, k, s_), name
    G.close()
    ctx.close()
