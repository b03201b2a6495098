"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results are compared bit-exactly: the GLOBAL edge order, every
w_{s,e} of every tree edge in both window layers, the window totals W_i, W,
the per-sample trees, contributions and reject reasons, hits2 and the reject
counters.  Inputs span several tiles of every kernel and ragged tails.
"""
import math

import numpy as np
import pytest

from helpers import SMALL_MOTIFS, small_random_graph, spanning_trees

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tg():
    import paper_2507_20441_gb300 as tg
    tg.build()
    return tg


def make_pair(tg, orc, n, s, d, t, flags=0):
    ctx = tg.Context()
    ctx.load_graph(n, s, d, t, flags=flags)
    G = orc.Graph(n, s, d, t, flags=flags)
    return ctx, G


def check_weights(ctx, mo, G, tree):
    for e in tree:
        for layer in (0, 1):
            a = mo.export_weights(e, layer)
            b = G.export_weights(e, layer)
            assert np.array_equal(a, b), (e, layer, int(np.argmax(a != b)))


def run_case(tg, ctx, G, nv, edges, rank, delta, tree, root, k=4000, seed=7, trace=True):
    mo = ctx.motif(nv, edges, rank, delta).set_tree(tree, root)
    G.set_motif(nv, edges, rank, delta, tree, root)
    Wg = mo.weights()
    Wo = G.weights()
    assert Wg == Wo
    assert np.array_equal(mo.window_totals(), G.window_totals())
    check_weights(ctx, mo, G, tree)
    if trace:
        rg, tg_, cg, why_g = mo.sample_trace(k, seed)
        ro, to_, co, why_o = G.sample(k, seed, trace=True)
        assert np.array_equal(tg_, to_)
        assert np.array_equal(why_g, why_o)
        assert np.array_equal(cg, co)
        # the untraced sampler (records in registers) on the same samples
        rs = mo.sample(k, seed)
        assert (rs.hits2, rs.valid, rs.rej_vertex, rs.rej_delta, rs.rej_order) == \
               (ro.hits2, ro.valid, ro.rej_vertex, ro.rej_delta, ro.rej_order)
    else:
        rg = mo.sample(k, seed)
        ro = G.sample(k, seed)
    assert (rg.W, rg.hits2, rg.valid, rg.rej_vertex, rg.rej_delta, rg.rej_order) == \
           (ro.W, ro.hits2, ro.valid, ro.rej_vertex, ro.rej_delta, ro.rej_order)
    assert rg.estimate == pytest.approx(ro.estimate, rel=1e-12)
    mo.free()
    return rg


def test_csr_global_order(tg, oracle_mod):
    from paper_2507_20441_gb300 import synth
    gr = synth.make_graph("tiny")
    ctx, G = make_pair(tg, oracle_mod, gr.n, gr.src, gr.dst, gr.t)
    s, d, t = ctx.edges()
    so, do, to = G.edges()
    assert ctx.m == G.m
    assert np.array_equal(s, so) and np.array_equal(d, do) and np.array_equal(t.astype(np.int64), to)
    assert ctx.t_min == G.t_min and ctx.T == G.span


@pytest.mark.parametrize("t_hi,m", [(5, 3000), (400, 3000), (1, 700), (1, 6000), (60_000, 150_000)])
def test_csr_global_order_with_equal_times(tg, oracle_mod, t_hi, m):
    """Runs of equal t' are ordered by (src, dst) after the time sort: runs of
    a few edges by one thread (t_hi = 400, 60,000), runs of hundreds by one
    block (t_hi = 5, and 1 with 700 edges), a run beyond 4096 edges by the full
    three-key sort (t_hi = 1 with 6000 edges); duplicates dropped."""
    rng = np.random.default_rng(t_hi)
    n = 50
    s = rng.integers(0, n, m).astype(np.uint32)
    d = ((s + 1 + rng.integers(0, n - 1, m)) % n).astype(np.uint32)
    t = rng.integers(0, t_hi, m).astype(np.int64) + 77
    ctx = tg.Context()
    ctx.load_graph(n, s, d, t, flags=tg.TM_DEDUP)
    G = oracle_mod.Graph(n, s, d, t, flags=oracle_mod.DEDUP)
    s1, d1, t1 = ctx.edges()
    so, do, to = G.edges()
    assert ctx.m == G.m
    assert np.array_equal(s1, so) and np.array_equal(d1, do) and np.array_equal(t1.astype(np.int64), to)
    ctx.close()


@pytest.mark.parametrize("flags", [0, 2, 4, 6])
def test_input_contract(tg, oracle_mod, flags):
    n, s, d, t = small_random_graph(3, n=12, m=300, t_hi=50)
    s = np.concatenate([s, s[:7], [5, 6]]).astype(np.uint32)   # 7 repeats, 2 self loops
    d = np.concatenate([d, d[:7], [5, 6]]).astype(np.uint32)
    t = np.concatenate([t, t[:7], [1003, 1004]]).astype(np.int64)
    ctx = tg.Context()
    if not flags & tg.TM_DROP_SELF:
        with pytest.raises(tg.TimestError) as e:
            ctx.load_graph(n, s, d, t, flags=flags)
        assert e.value.code == tg.TM_E_SELFLOOP
        return
    if not flags & tg.TM_DEDUP:
        with pytest.raises(tg.TimestError) as e:
            ctx.load_graph(n, s, d, t, flags=flags)
        assert e.value.code == tg.TM_E_DUP
        return
    ctx.load_graph(n, s, d, t, flags=flags)
    G = oracle_mod.Graph(n, s, d, t, flags=oracle_mod.DEDUP | oracle_mod.DROP_SELF)
    assert ctx.m == G.m == 300
    so, do, to = G.edges()
    s2, d2, t2 = ctx.edges()
    assert np.array_equal(s2, so) and np.array_equal(d2, do) and np.array_equal(t2.astype(np.int64), to)


@pytest.mark.parametrize("name", sorted(SMALL_MOTIFS))
def test_small_motifs_every_tree(tg, oracle_mod, name):
    nv, edges, rank = SMALL_MOTIFS[name]
    n, s, d, t = small_random_graph(40, n=nv + 3, m=400, t_hi=120)
    ctx, G = make_pair(tg, oracle_mod, n, s, d, t)
    for delta in (7, 25):
        for tree in spanning_trees(nv, edges):
            for root in tree:
                run_case(tg, ctx, G, nv, edges, rank, delta, tree, root, k=3000, seed=delta + root)


@pytest.mark.parametrize("wl", ["tiny", "dense_tiny"])
def test_workload_triangle(tg, oracle_mod, wl):
    from paper_2507_20441_gb300 import synth
    gr = synth.make_graph(wl)
    mo = synth.make_motif(wl)
    ctx, G = make_pair(tg, oracle_mod, gr.n, gr.src, gr.dst, gr.t)
    for tree in spanning_trees(mo.nv, mo.edges):
        for root in tree:
            run_case(tg, ctx, G, mo.nv, mo.edges, mo.rank, mo.delta, tree, root, k=20000, seed=1 + root, trace=True)


def test_chung_lu_cycle4_and_chord(tg, oracle_mod):
    from paper_2507_20441_gb300 import synth
    gr = synth.chung_lu_bursty(5000, 200_000, 2.1, 3_000_000, seed=3)
    ctx, G = make_pair(tg, oracle_mod, gr.n, gr.src, gr.dst, gr.t)
    c4 = synth.cycle(4, 86_400)
    run_case(tg, ctx, G, c4.nv, c4.edges, c4.rank, c4.delta, [0, 1, 2], 1, k=20000, seed=5)
    run_case(tg, ctx, G, c4.nv, c4.edges, c4.rank, c4.delta, [1, 2, 3], 3, k=20000, seed=6)
    c5 = synth.cycle5_chord(3_600)
    # ([1, 2, 3, 4], 2): the first and last pi edges are non-tree (coupled span);
    # ([0, 3, 4, 5], 4): non-tree edges at consecutive pi positions (merge path)
    for tree, root in (([0, 1, 3, 4], 1), ([0, 2, 3, 4], 3), ([1, 2, 4, 5], 2), ([1, 2, 3, 4], 2),
                       ([0, 3, 4, 5], 4)):
        run_case(tg, ctx, G, c5.nv, c5.edges, c5.rank, c5.delta, tree, root, k=20000, seed=9)


def test_default_tree_and_resume(tg, oracle_mod):
    n, s, d, t = small_random_graph(8, n=9, m=500, t_hi=200)
    ctx, G = make_pair(tg, oracle_mod, n, s, d, t)
    nv, edges, rank = SMALL_MOTIFS["cycle4"]
    mo = ctx.motif(nv, edges, rank, 30)
    order, parent = mo.plan()
    assert sorted(order.tolist()) == [0, 1, 2] and parent[0] == -1
    mo.weights()
    full = mo.sample(10_000, 3)
    a = mo.sample(4_321, 3, 0)
    b = mo.sample(10_000 - 4_321, 3, 4_321)
    assert full.hits2 == a.hits2 + b.hits2
    assert full.valid == a.valid + b.valid
    # the default plan is a tree the oracle accepts, with the same outcome
    G.set_motif(nv, edges, rank, 30, sorted(order.tolist()), int(order[0]))
    G.weights()
    ro = G.sample(10_000, 3)
    assert ro.hits2 == full.hits2


def test_edge_cases(tg, oracle_mod):
    # single edge motif, delta larger than the span, delta = 1, equal times
    n, s, d, t = small_random_graph(4, n=30, m=800, t_hi=60)
    ctx, G = make_pair(tg, oracle_mod, n, s, d, t)
    for delta in (1, 3, 10**12):
        run_case(tg, ctx, G, 2, [(0, 1)], [0], delta, [0], 0, k=5000)
        run_case(tg, ctx, G, 3, [(0, 1), (1, 2), (2, 0)], [0, 1, 2], delta, [0, 1], 0, k=5000)
    # all edges at one timestamp
    s2 = np.arange(0, 200, dtype=np.uint32) % 20
    d2 = (s2 + 1 + np.arange(200, dtype=np.uint32) // 20) % 20
    t2 = np.full(200, 77, np.int64)
    ctx2, G2 = make_pair(tg, oracle_mod, 20, s2, d2, t2)
    run_case(tg, ctx2, G2, 3, [(0, 1), (1, 2)], [0, 1], 5, [0, 1], 1, k=2000)
    # empty sample count and a graph with a single edge
    ctx3, G3 = make_pair(tg, oracle_mod, 2, np.array([0], np.uint32), np.array([1], np.uint32), np.array([5], np.int64))
    mo = ctx3.motif(2, [(0, 1)], [0], 4)
    assert mo.weights() == 1
    r = mo.sample(0, 1)
    assert r.hits2 == 0 and r.k == 0
    r = mo.sample(100, 1)
    assert r.valid == 100 and r.estimate == pytest.approx(1.0)


def test_overflow_reported(tg):
    hub = 2000
    src = np.zeros(hub, np.uint32)
    dst = np.arange(1, hub + 1, dtype=np.uint32)
    t = np.arange(hub, dtype=np.int64)
    ctx = tg.Context()
    ctx.load_graph(hub + 1, src, dst, t)
    mo = ctx.motif(8, [(0, i) for i in range(1, 8)], list(range(7)), 10_000).set_tree(list(range(7)), 0)
    with pytest.raises(tg.TimestError) as e:
        mo.weights()
    assert e.value.code == tg.TM_E_OVERFLOW


def test_estimate_within_5_percent(tg, oracle_mod):
    """Dense tiny triangle: the exact count by brute force, the estimate at
    k = 1e6 within 5% (the Chernoff bound of Thm. 3.8 with the measured W, C
    and B predicts well under 5% here)."""
    from paper_2507_20441_gb300 import synth
    gr = synth.make_graph("dense_tiny")
    mo = synth.make_motif("dense_tiny")
    ctx, G = make_pair(tg, oracle_mod, gr.n, gr.src, gr.dst, gr.t)
    C = G.brute_count(mo.nv, mo.edges, mo.rank, mo.delta)
    m = ctx.motif(mo.nv, mo.edges, mo.rank, mo.delta)
    m.weights()
    r = m.sample(1_000_000, 11)
    assert abs(r.estimate - C) / C < 0.05, (r.estimate, C)
