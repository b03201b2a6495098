"""Serving (continuous batching): queries submitted concurrently from several
threads, admitted under a weight-memory budget and sampled in shared rounds,
give exactly the result each gives alone (tm_sample on its default tree with
the same k and seed) and the CPU oracle's TIMEST on that tree (Alg. 3-6);
weights are cached and reused, evicted when the budget demands it; waits are
bounded."""
import threading
import time

import numpy as np
import pytest

from helpers import default_tree, oracle_result, result_tuple

pytestmark = pytest.mark.gpu


def _graph():
    from paper_2507_20441_gb300 import synth
    return synth.chung_lu_bursty(20_000, 400_000, 2.1, 6_000_000, seed=21)


def _queries(n, seed):
    from paper_2507_20441_gb300 import synth
    pool = synth.motif_pool(seed=seed, count=12, k_lo=2e3, k_hi=3e5)
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        mo = pool[int(rng.integers(0, len(pool)))]          # repeats exercise the weight cache
        out.append((mo, int(rng.integers(1_000, 400_000)), int(rng.integers(0, 2**40))))
    return out


def _alone(ctx, queries):
    """Each query on its own: default tree, weights, tm_sample(k, seed, 0)."""
    ref = []
    cache = {}
    for mo, k, seed in queries:
        key = (mo.name, mo.delta)
        if key not in cache:
            m = ctx.motif(mo.nv, mo.edges, mo.rank, mo.delta)
            m.weights()
            cache[key] = m
        ref.append(cache[key].sample(k, seed))
    for m in cache.values():
        m.free()
    return ref


def _oracle_check(gr, queries, served, oracle_mod, every=1):
    """Served results against the oracle on the default tree, samples 0..k-1."""
    G = oracle_mod.Graph(gr.n, gr.src, gr.dst, gr.t)
    checked = 0
    for i, ((mo, k, seed), r) in enumerate(zip(queries, served)):
        if i % every:
            continue
        tree, root = default_tree(mo.nv, mo.edges, mo.rank)
        want = oracle_result(G, mo.nv, mo.edges, mo.rank, mo.delta, tree, root, k, seed)
        assert result_tuple(r) == want, (i, mo.name, k, seed)
        checked += 1
    G.close()
    return checked


def _serve_all(ctx, queries, threads=4):
    tickets = [None] * len(queries)

    def worker(idx):
        for i in idx:
            mo, k, seed = queries[i]
            tickets[i] = ctx.submit(mo.nv, mo.edges, mo.rank, mo.delta, k, seed)
            time.sleep(0.0005 * (i % 3))

    parts = [list(range(j, len(queries), threads)) for j in range(threads)]
    ths = [threading.Thread(target=worker, args=(p,)) for p in parts]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    results = []
    for tk in tickets:
        r = ctx.poll(tk, timeout_ms=120_000)
        assert r is not None
        results.append(r)
    return results


def _same(a, b):
    return (a.W, a.hits2, a.k, a.valid, a.rej_vertex, a.rej_delta, a.rej_order) == \
           (b.W, b.hits2, b.k, b.valid, b.rej_vertex, b.rej_delta, b.rej_order)


def test_results_in_the_mix_equal_results_alone(oracle_mod):
    import paper_2507_20441_gb300 as tg
    tg.build()
    gr = _graph()
    ctx = tg.Context()
    ctx.load_graph(gr.n, gr.src, gr.dst, gr.t)
    queries = _queries(40, seed=5)
    ctx.serve_start(max_active=16, tile=2048)
    served = _serve_all(ctx, queries)
    st = ctx.serve_stats()
    ctx.serve_stop()
    assert st["completed"] == 40 and st["failed"] == 0
    assert st["cache_hits"] > 0 and st["cache_misses"] <= 12
    assert st["p99_ms"] >= st["p50_ms"] > 0 and st["qps"] > 0
    assert st["rounds"] >= 1
    ref = _alone(ctx, queries)
    for (mo, k, seed), a, b in zip(queries, served, ref):
        assert _same(a, b), (mo.name, k, seed)
        assert a.estimate == b.estimate
    ctx.close()
    assert _oracle_check(gr, queries, served, oracle_mod) == 40


def test_memory_gated_admission_evicts_and_stays_exact(oracle_mod):
    import paper_2507_20441_gb300 as tg
    gr = _graph()
    ctx = tg.Context()
    ctx.load_graph(gr.n, gr.src, gr.dst, gr.t)
    queries = _queries(24, seed=9)
    # room for only a few motifs' weights at a time
    budget = 3 * (16 + 32 * 2) * ctx.m
    ctx.serve_start(max_active=4, tile=1024, weight_budget=budget)
    served = _serve_all(ctx, queries, threads=3)
    st = ctx.serve_stats()
    ctx.serve_stop()
    assert st["completed"] == 24 and st["failed"] == 0
    assert st["evictions"] > 0
    ref = _alone(ctx, queries)
    for a, b in zip(served, ref):
        assert _same(a, b)
    ctx.close()
    assert _oracle_check(gr, queries, served, oracle_mod, every=3) == 8


def test_poll_is_bounded_and_timeouts_leave_the_context_usable():
    import paper_2507_20441_gb300 as tg
    gr = _graph()
    ctx = tg.Context()
    ctx.load_graph(gr.n, gr.src, gr.dst, gr.t)
    from paper_2507_20441_gb300 import synth
    c4 = synth.cycle(4, 86_400)
    # a 1 ms limit on each round's device wait: a 20M-sample query's round runs
    # out and the query reports TM_E_TIMEOUT instead of waiting without bound
    ctx.serve_start(max_active=2, tile=65536, round_tiles=400, poll_timeout_ms=1)
    t = ctx.submit(c4.nv, c4.edges, c4.rank, c4.delta, 20_000_000, 3)
    t0 = time.perf_counter()
    early = ctx.poll(t, timeout_ms=0)                      # never blocks: None while running
    assert time.perf_counter() - t0 < 0.5 and early is None
    with pytest.raises(tg.TimestError) as e:
        ctx.poll(t, timeout_ms=120_000)
    assert e.value.code == tg.TM_E_TIMEOUT
    ctx.serve_stop()
    # the context still serves correctly afterwards
    ctx.serve_start(max_active=2)
    t2 = ctx.submit(c4.nv, c4.edges, c4.rank, c4.delta, 50_000, 4)
    got = ctx.poll(t2, timeout_ms=120_000)
    ctx.serve_stop()
    m = ctx.motif(c4.nv, c4.edges, c4.rank, c4.delta)
    m.weights()
    assert _same(got, m.sample(50_000, 4))
    with pytest.raises(tg.TimestError):
        ctx.poll(1, timeout_ms=0)          # not serving any more
    ctx.close()


def test_submit_motif_serves_the_pinned_plan(oracle_mod):
    """tm_serve_submit_motif serves a motif handle's own plan: a pinned
    non-default tree and root, and constraint settings, served in the mix with
    default-plan queries of the same motif; each result equals tm_sample on its
    plan and the oracle on the same tree, root and constraints."""
    import paper_2507_20441_gb300 as tg
    from helpers import spanning_trees
    gr = _graph()
    ctx = tg.Context()
    ctx.load_graph(gr.n, gr.src, gr.dst, gr.t)
    nv, edges, rank, delta = 4, [(0, 1), (1, 2), (2, 3), (3, 0)], [0, 1, 2, 3], 86_400
    dtree, droot = default_tree(nv, edges, rank)
    other = [t for t in spanning_trees(nv, edges) if sorted(t) != sorted(dtree)][0]
    plans = [(other, other[0], True, True), (other, other[-1], False, True), (dtree, droot, True, False),
             (dtree, droot, True, True)]
    motifs = [ctx.motif(nv, edges, rank, delta).set_tree(t, r).set_constraints(c2, c3) for t, r, c2, c3 in plans]
    ks = [150_000, 90_000, 120_000, 60_000]
    ctx.serve_start(max_active=8, tile=2048)
    tickets = [ctx.submit_motif(m, k, 40 + i) for i, (m, k) in enumerate(zip(motifs, ks))]
    tickets.append(ctx.submit(nv, edges, rank, delta, 70_000, 99))      # default plan, same motif
    served = [ctx.poll(t, timeout_ms=120_000) for t in tickets]
    st = ctx.serve_stats()
    ctx.serve_stop()
    assert st["completed"] == 5 and st["failed"] == 0
    assert st["cache_misses"] == 5        # one weight pass per distinct plan
    G = oracle_mod.Graph(gr.n, gr.src, gr.dst, gr.t)
    for i, ((t, r, c2, c3), m, k) in enumerate(zip(plans, motifs, ks)):
        m.weights()
        alone = m.sample(k, 40 + i)
        assert _same(served[i], alone), i
        want = oracle_result(G, nv, edges, rank, delta, t, r, k, 40 + i, c2=c2, c3=c3)
        assert result_tuple(served[i]) == want, i
    want = oracle_result(G, nv, edges, rank, delta, dtree, droot, 70_000, 99)
    assert result_tuple(served[4]) == want
    G.close()
    ctx.close()
