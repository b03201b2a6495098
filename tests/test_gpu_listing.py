"""Motif listing: every valid sample's listed instances are exactly the
M-matches (Def. 1.2) whose tree edges are the sampled tree, recomputed here by
brute force over the graph (edge ids in GLOBAL order), whose total equals the
oracle's exact count O1 on the same graph; rejected samples list nothing; a
truncated listing is a prefix of the full one."""
from collections import defaultdict

import numpy as np
import pytest

from helpers import SMALL_MOTIFS, small_random_graph

pytestmark = pytest.mark.gpu


def all_matches(src, dst, tp, edges, order, delta):
    """Every M-match as a tuple of edge ids indexed by motif edge (Def. 1.2):
    an injective vertex map, edge i mapped to an edge between the images of its
    endpoints, times strictly increasing along pi, last - first <= delta."""
    ne = len(edges)
    by_pos = sorted(range(ne), key=lambda e: order[e])
    pair = defaultdict(list)
    for g in np.argsort(tp, kind="stable"):
        pair[(int(src[g]), int(dst[g]))].append(int(g))
    out = []
    phi = {}
    chosen = [None] * ne

    def rec(i, t_prev, t_first):
        if i == ne:
            out.append(tuple(chosen))
            return
        e = by_pos[i]
        a, b = edges[e]
        cand = []
        if a in phi and b in phi:
            cand = pair.get((phi[a], phi[b]), [])
        else:
            for (u, v), lst in pair.items():
                if (a in phi and phi[a] != u) or (b in phi and phi[b] != v):
                    continue
                cand.extend(lst)
        for g in cand:
            u, v, t = int(src[g]), int(dst[g]), int(tp[g])
            if t <= t_prev or (t_first is not None and t - t_first > delta):
                continue
            new = []
            ok = True
            for x, y in ((a, u), (b, v)):
                if x in phi:
                    ok &= phi[x] == y
                elif y in phi.values():
                    ok = False
                else:
                    phi[x] = y
                    new.append(x)
            if ok:
                chosen[e] = g
                rec(i + 1, t, t if t_first is None else t_first)
            for x in new:
                del phi[x]
        chosen[e] = None

    rec(0, -1, None)
    return out


CASES = [("triangle", 12), ("cycle4", 15), ("cycle5_chord", 30), ("bowtie", 20), ("path4_mixed", 10),
         ("antiparallel", 10), ("parallel", 10), ("out_star3", 8)]


@pytest.mark.parametrize("name,delta", CASES)
def test_listing_matches_brute_force(name, delta, oracle_mod):
    import paper_2507_20441_gb300 as tg
    tg.build()
    nv, edges, order = SMALL_MOTIFS[name]
    n, s, d, t = small_random_graph(11, n=7, m=90, t_hi=40)
    ctx = tg.Context()
    ctx.load_graph(n, s, d, t)
    gs, gd, gt = tg.tm_edges_export(ctx.h)
    m = ctx.motif(nv, edges, order, delta)
    m.weights()
    tree_order, _ = m.plan()
    k, seed = 3000, 5
    res, gids, contrib, reason = m.sample_trace(k, seed)
    rows, sids, total = m.sample_list(k, seed)
    matches = all_matches(gs, gd, gt, edges, order, delta)
    # the enumerator written here agrees with the oracle's exact count (O1)
    assert len(matches) == oracle_mod.Graph(n, s, d, t).brute_count(nv, edges, order, delta)
    by_tree = defaultdict(list)
    for mt in matches:
        by_tree[tuple(mt[e] for e in tree_order)].append(mt)
    listed = defaultdict(list)
    for r, j in zip(rows, sids):
        listed[int(j)].append(tuple(int(x) for x in r))
    expect_total = 0
    for j in range(k):
        want = sorted(by_tree.get(tuple(int(x) for x in gids[j]), [])) if reason[j] == 0 else []
        assert sorted(listed.get(j, [])) == want, j
        expect_total += len(want)
    assert total == expect_total == len(rows)
    if total > 3:   # truncation keeps the first rows
        r2, s2, t2 = m.sample_list(k, seed, max_inst=total // 2)
        assert t2 == total and np.array_equal(r2, rows[:total // 2]) and np.array_equal(s2, sids[:total // 2])
    ctx.close()


def test_listing_sample_ranges_compose():
    import paper_2507_20441_gb300 as tg
    nv, edges, order = SMALL_MOTIFS["cycle4"]
    n, s, d, t = small_random_graph(3, n=7, m=90, t_hi=40)
    ctx = tg.Context()
    ctx.load_graph(n, s, d, t)
    m = ctx.motif(nv, edges, order, 15)
    m.weights()
    whole = m.sample_list(2000, 8)
    a = m.sample_list(700, 8, 0)
    b = m.sample_list(1300, 8, 700)
    assert np.array_equal(whole[0], np.concatenate([a[0], b[0]]))
    assert np.array_equal(whole[1], np.concatenate([a[1], b[1]]))
    assert whole[2] == a[2] + b[2] > 0
    ctx.close()
