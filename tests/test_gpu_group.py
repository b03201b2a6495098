"""Several motifs per sampling run: motifs whose spanning trees are the same
temporal pattern (here the path 0->1->2->3 rooted at its middle edge, with the
path edges in the same pi order) share one weight pass and one stream of
sampled trees; each motif's result equals the CPU oracle's TIMEST on that
motif with the same tree, k, seed and first sample id (Alg. 6 per motif, as
the paper counts the 4-vertex motifs of one table from one run) and its own
tm_sample, bit for bit."""
import numpy as np
import pytest

from helpers import oracle_result, result_tuple, small_random_graph

pytestmark = pytest.mark.gpu

PATH = [(0, 1), (1, 2), (2, 3)]
# (extra edges, pi positions of all edges); the path edges keep their relative order
GROUP = [
    ([(3, 0)], [0, 1, 2, 3]),            # 4-cycle
    ([(0, 2)], [0, 2, 3, 1]),            # chord 0->2 between the first two path edges
    ([(1, 3)], [0, 1, 2, 3]),
    ([(3, 1)], [1, 2, 3, 0]),            # the extra edge comes first
    ([(3, 0), (0, 2)], [0, 2, 3, 4, 1]),  # two non-tree edges
]


def _motifs(ctx, delta):
    out = []
    for extra, order in GROUP:
        m = ctx.motif(4, PATH + extra, order, delta).set_tree([0, 1, 2], 1)
        out.append(m)
    return out


def _same(a, b):
    return (a.W, a.hits2, a.k, a.valid, a.rej_vertex, a.rej_delta, a.rej_order, a.estimate) == \
           (b.W, b.hits2, b.k, b.valid, b.rej_vertex, b.rej_delta, b.rej_order, b.estimate)


@pytest.mark.parametrize("kind", ["dense", "chung_lu"])
def test_group_equals_separate_runs(kind, oracle_mod):
    import paper_2507_20441_gb300 as tg
    tg.build()
    if kind == "dense":
        n, s, d, t = small_random_graph(4, n=12, m=3000, t_hi=400)
        delta, k = 60, 200_000
    else:
        from paper_2507_20441_gb300 import synth
        gr = synth.chung_lu_bursty(5000, 200_000, 2.1, 3_000_000, seed=3)
        n, s, d, t = gr.n, gr.src, gr.dst, gr.t
        delta, k = 86_400, 300_000
    ctx = tg.Context()
    ctx.load_graph(n, s, d, t)
    ms = _motifs(ctx, delta)
    Ws = [m.weights() for m in ms]
    assert len(set(Ws)) == 1                      # one tree pattern, one W
    G = oracle_mod.Graph(n, s, d, t)
    for first in (0, 12_345):
        single = [m.sample(k, 9, first) for m in ms]
        group = ctx.sample_group(ms, k, 9, first)
        for (extra, order), a, b in zip(GROUP, group, single):
            assert _same(a, b)
            want = oracle_result(G, 4, PATH + extra, order, delta, [0, 1, 2], 1, k, 9, first)
            assert result_tuple(a) == want, (extra, order, first)
    assert any(r.hits2 for r in single)           # the case is not vacuous
    G.close()
    ctx.close()


def test_group_needs_first_weights_and_one_pattern():
    import paper_2507_20441_gb300 as tg
    n, s, d, t = small_random_graph(5, n=10, m=800, t_hi=200)
    ctx = tg.Context()
    ctx.load_graph(n, s, d, t)
    ms = _motifs(ctx, 50)
    with pytest.raises(tg.TimestError) as e:
        ctx.sample_group(ms, 1000, 1)             # motifs[0] has no weights
    assert e.value.code == tg.TM_E_STATE
    ms[0].weights()
    star = ctx.motif(4, [(1, 0), (1, 2), (1, 3), (3, 0)], [0, 1, 2, 3], 50).set_tree([0, 1, 2], 1)
    with pytest.raises(tg.TimestError) as e:
        ctx.sample_group([ms[0], star], 1000, 1)  # a different tree pattern
    assert e.value.code == tg.TM_E_MOTIF
    swapped = ctx.motif(4, PATH + [(3, 0)], [2, 1, 0, 3], 50).set_tree([0, 1, 2], 1)
    with pytest.raises(tg.TimestError) as e:
        ctx.sample_group([ms[0], swapped], 1000, 1)   # path edges in another pi order
    assert e.value.code == tg.TM_E_MOTIF
    assert ctx.sample_group([ms[0]], 0, 1)[0].k == 0
    ctx.close()
