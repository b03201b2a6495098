"""The untraced sampler for every spanning-tree size the plan allows (1 to 7
tree edges, 2 to 8 motif vertices) against the oracle, bit for bit: hits2 and
the reject counters (Alg. 3-6).  The library instantiates this sampler once
per tree size with the per-sample records in registers; plans whose non-tree
edges sit at consecutive pi positions (the general DeriveCnt) take the
local-memory sampler, covered here too.
"""
import numpy as np
import pytest

from helpers import small_random_graph, spanning_trees

pytestmark = pytest.mark.gpu


def _motifs():
    out = {"edge": (2, [(0, 1)], [0]), "edge_twice": (2, [(0, 1), (0, 1)], [0, 1])}
    for nv in range(3, 9):
        out[f"path{nv}"] = (nv, [(i, i + 1) for i in range(nv - 1)], list(range(nv - 1)))
        out[f"cycle{nv}"] = (nv, [(i, (i + 1) % nv) for i in range(nv)], list(range(nv)))
    # alternating directions, pi order not along the path
    out["zigzag8"] = (8, [(i, i + 1) if i % 2 == 0 else (i + 1, i) for i in range(7)], [3, 0, 5, 1, 6, 2, 4])
    # chord ranked right after the closing edge: trees without both put two
    # non-tree edges at consecutive pi positions
    out["cycle6_chord"] = (6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 0), (0, 3)], [0, 1, 2, 3, 4, 5, 6])
    return out


MOTIFS = _motifs()


@pytest.fixture(scope="module")
def tg():
    import paper_2507_20441_gb300 as tg
    tg.build()
    return tg


@pytest.mark.parametrize("name", sorted(MOTIFS))
def test_untraced_sampler_every_tree_size(tg, oracle_mod, name):
    nv, edges, rank = MOTIFS[name]
    n, s, d, t = small_random_graph(100 + nv, n=nv + 4, m=2500, t_hi=200)
    ctx = tg.Context()
    ctx.load_graph(n, s, d, t)
    G = oracle_mod.Graph(n, s, d, t)
    trees = spanning_trees(nv, edges)
    picked = [trees[i] for i in sorted({0, len(trees) // 2, len(trees) - 1})]
    valid = 0
    for delta in (40, 150):
        for tree in picked:
            for root in sorted({tree[0], tree[-1]}):
                mo = ctx.motif(nv, edges, rank, delta).set_tree(tree, root)
                G.set_motif(nv, edges, rank, delta, tree, root)
                assert mo.weights() == G.weights()
                k, seed = 4000, 11 + delta + root
                rg = mo.sample(k, seed)
                ro = G.sample(k, seed)
                assert (rg.hits2, rg.valid, rg.rej_vertex, rg.rej_delta, rg.rej_order) == \
                       (ro.hits2, ro.valid, ro.rej_vertex, ro.rej_delta, ro.rej_order), (tree, root, delta)
                valid += rg.valid
                mo.free()
    assert valid > 0
