"""Test-side helpers: small random graphs and spanning-tree enumeration.

Nothing here computes TIMEST quantities; it only builds inputs.
"""
import itertools

import numpy as np


def spanning_trees(nv, edges):
    """All sets of nv-1 motif-edge indices forming a spanning tree of the
    underlying undirected multigraph."""
    out = []
    for comb in itertools.combinations(range(len(edges)), nv - 1):
        comp = list(range(nv))
        ok = True
        for e in comb:
            a, b = edges[e]
            ca, cb = comp[a], comp[b]
            if ca == cb:
                ok = False
                break
            comp = [ca if c == cb else c for c in comp]
        if ok and len(set(comp)) == 1:
            out.append(list(comb))
    return out


def small_random_graph(seed, n=7, m=70, t_hi=40, t0=1000):
    """Dense small multigraph: unique (u,v,t), no self loops, many repeats."""
    rng = np.random.default_rng(seed)
    seen = set()
    src, dst, t = [], [], []
    while len(src) < m:
        u = int(rng.integers(0, n)); v = int(rng.integers(0, n - 1)); v += v >= u
        tt = int(rng.integers(0, t_hi))
        if (u, v, tt) in seen:
            continue
        seen.add((u, v, tt))
        src.append(u); dst.append(v); t.append(tt + t0)
    return n, np.array(src, np.uint32), np.array(dst, np.uint32), np.array(t, np.int64)


SMALL_MOTIFS = {
    "triangle": (3, [(0, 1), (1, 2), (2, 0)], [0, 1, 2]),
    "triangle_ff": (3, [(0, 1), (1, 2), (0, 2)], [0, 2, 1]),
    "cycle4": (4, [(0, 1), (1, 2), (2, 3), (3, 0)], [0, 1, 2, 3]),
    "cycle5_chord": (5, [(0, 1), (1, 2), (0, 2), (2, 3), (3, 4), (4, 0)], [0, 1, 2, 3, 4, 5]),
    "out_star3": (4, [(0, 1), (0, 2), (0, 3)], [1, 0, 2]),
    "in_star3": (4, [(1, 0), (2, 0), (3, 0)], [0, 1, 2]),
    "path4_mixed": (4, [(0, 1), (2, 1), (2, 3)], [2, 0, 1]),
    "bowtie": (5, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 2)], [3, 0, 5, 1, 4, 2]),
    "antiparallel": (3, [(0, 1), (1, 0), (1, 2)], [1, 0, 2]),
    "parallel": (3, [(0, 1), (1, 2), (0, 1)], [0, 1, 2]),
}


def default_tree(nv, edges, rank):
    """The spanning tree and root edge tm_set_motif picks by default, worked
    out on the host from its documented rule (bench.reference_tree; checked
    against the library's ranking for 42 motifs by test_bench_contract), so
    the oracle can run the same plan without taking it from the CUDA path."""
    import types
    import bench
    return bench.reference_tree(types.SimpleNamespace(nv=nv, edges=[tuple(e) for e in edges], rank=list(rank)))


def oracle_result(G, nv, edges, rank, delta, tree, root, k, seed, first=0, c2=True, c3=True):
    """The oracle's TIMEST (Alg. 3-6) on one plan: (W, hits2, valid,
    rej_vertex, rej_delta, rej_order) of samples first .. first+k-1."""
    G.set_motif(nv, [tuple(e) for e in edges], list(rank), delta, list(tree), root)
    if not (c2 and c3):
        G.set_constraints(c2, c3)
    W = G.weights()
    if W == 0 or k == 0:
        return (W, 0, 0, 0, 0, 0)
    r = G.sample(k, seed, first, threads=0)
    return (W, r.hits2, r.valid, r.rej_vertex, r.rej_delta, r.rej_order)


def result_tuple(r):
    return (r.W, r.hits2, r.valid, r.rej_vertex, r.rej_delta, r.rej_order)


def csr_by_loops(n, gs, gd, gt):
    """The temporal CSR arrays (names as oracle.csr_arrays) of a graph in
    GLOBAL order (gs, gd, gt as lists), built one edge at a time by plain
    loops: a vertex's out-list is its edges in GLOBAL order, an out entry's
    cross rank counts the owner's in-edges strictly earlier, the multi-edge
    lists group (src, dst) in time order."""
    me = len(gs)
    out_lists = [[e for e in range(me) if gs[e] == v] for v in range(n)]
    in_lists = [[e for e in range(me) if gd[e] == v] for v in range(n)]
    out_gid = [e for v in range(n) for e in out_lists[v]]
    in_gid = [e for v in range(n) for e in in_lists[v]]
    off_o, off_i = [0], [0]
    for v in range(n):
        off_o.append(off_o[-1] + len(out_lists[v]))
        off_i.append(off_i[-1] + len(in_lists[v]))
    pos_o = {e: x for x, e in enumerate(out_gid)}
    pos_i = {e: x for x, e in enumerate(in_gid)}
    pairs = sorted({(gs[e], gd[e]) for e in range(me)})
    members = {pr: sorted((f for f in range(me) if (gs[f], gd[f]) == pr), key=lambda f: gt[f]) for pr in pairs}
    multi = [e for pr in pairs for e in members[pr]]
    po = [0]
    for pr in pairs:
        po.append(po[-1] + len(members[pr]))

    def words(starts):
        w = [0] * (me // 32 + 1)
        for x in starts:
            w[x // 32] |= 1 << (x % 32)
        return w
    return {
        "out_off": off_o, "in_off": off_i, "out_gid": out_gid, "in_gid": in_gid,
        "out_t": [gt[e] for e in out_gid], "out_nbr": [gd[e] for e in out_gid], "out_src": [gs[e] for e in out_gid],
        "in_t": [gt[e] for e in in_gid], "in_nbr": [gs[e] for e in in_gid], "in_dst": [gd[e] for e in in_gid],
        "out_pos": [pos_o[e] for e in range(me)], "in_pos": [pos_i[e] for e in range(me)],
        "in_to_out": [pos_o[e] for e in in_gid],
        "out_xrank": [off_i[gs[e]] + sum(1 for f in in_lists[gs[e]] if gt[f] < gt[e]) for e in out_gid],
        "in_xrank": [off_o[gd[e]] + sum(1 for f in out_lists[gd[e]] if gt[f] < gt[e]) for e in in_gid],
        "multi_t": [gt[e] for e in multi], "multi_to_out": [pos_o[e] for e in multi],
        "pair_off": po, "pair_dst": [v for _, v in pairs],
        "vpair_off": [sum(1 for (u, _) in pairs if u < v) for v in range(n + 1)],
        "own_out": words(off_o[v] for v in range(n) if out_lists[v]),
        "own_in": words(off_i[v] for v in range(n) if in_lists[v]),
        "own_multi": words(po[:-1]),
    }


def csr_case(oracle_mod, seed, n, m, t_hi):
    """A small random graph with repeats dropped, as an oracle Graph."""
    rng = np.random.default_rng(seed)
    s = rng.integers(0, n, m)
    d = (s + 1 + rng.integers(0, n - 1, m)) % n
    t = rng.integers(0, t_hi, m) + 5
    return oracle_mod.Graph(n, s.astype(np.uint32), d.astype(np.uint32), t.astype(np.int64), flags=oracle_mod.DEDUP)
