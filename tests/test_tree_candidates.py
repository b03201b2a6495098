"""Host logic of Alg. 7's first two steps (no GPU): tm_tree_candidates lists
every spanning tree of a motif ranked by constraint looseness (Alg. 8, read
over unordered pairs of tree edges that share a vertex: |pi(e1) - pi(e2)| - 1,
summed), ties broken by the lexicographically smallest edge set.  The
expected ranking is recomputed here from that definition over a brute-force
enumeration of edge subsets."""
import itertools

import pytest

from helpers import SMALL_MOTIFS, spanning_trees


def _looseness(edges, order, tree):
    total = 0
    for e1, e2 in itertools.combinations(tree, 2):
        if set(edges[e1]) & set(edges[e2]):
            shared = len(set(edges[e1]) & set(edges[e2]))
            total += shared * (abs(order[e1] - order[e2]) - 1)
    return total


def _expected(nv, edges, order):
    trees = spanning_trees(nv, edges)            # lexicographic order
    ranked = sorted(trees, key=lambda tr: _looseness(edges, order, tr))   # stable
    return [(sum(1 << e for e in tr), _looseness(edges, order, tr)) for tr in ranked]


def _motifs():
    from paper_2507_20441_gb300 import synth
    out = dict(SMALL_MOTIFS)
    for i, mo in enumerate(synth.motif_pool(seed=7, count=32)):
        out[f"pool{i}_{mo.name}"] = (mo.nv, [tuple(e) for e in mo.edges], list(mo.rank))
    return out


@pytest.mark.parametrize("name", sorted(_motifs()))
def test_ranking_matches_definition(name):
    import paper_2507_20441_gb300 as tg
    tg.build()
    nv, edges, order = _motifs()[name]
    got = tg.tm_tree_candidates(nv, edges, order)
    assert got == _expected(nv, edges, order)


def test_antiparallel_pair_counts_both_shared_vertices():
    # edges 0->1 and 1->0 share two vertices: the pair is counted at each
    import paper_2507_20441_gb300 as tg
    tg.build()
    got = dict(tg.tm_tree_candidates(3, [(0, 1), (1, 0), (1, 2)], [0, 2, 1]))
    # trees {0,2} and {1,2}: pairs (0,2) at vertex 1: |0-1|-1 = 0; (1,2) at vertex 1: |2-1|-1 = 0
    assert got == {0b101: 0, 0b110: 0}


def test_invalid_motif_rejected():
    import paper_2507_20441_gb300 as tg
    tg.build()
    with pytest.raises(tg.TimestError):
        tg.tm_tree_candidates(3, [(0, 1), (1, 1)], [0, 1])       # self loop
    with pytest.raises(tg.TimestError):
        tg.tm_tree_candidates(4, [(0, 1), (2, 3), (1, 0)], [0, 1, 2])   # not connected
