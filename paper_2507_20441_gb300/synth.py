"""Seeded synthetic temporal graphs and motif queries.

Stand-ins for the paper's wiki-talk / stackoverflow / bitcoin / reddit-reply
datasets (Sec. 5.1, Table 2), which are not available: every input here is
generated from a seed with numpy's PCG64 stream.  This module holds none of
TIMEST's arithmetic; it only produces (src, dst, t) tuples and motif
descriptions, and it serves both the CUDA path and the CPU oracle.

Graph families
  * ``uniform_graph``: src/dst uniform over distinct vertices, t uniform.
  * ``chung_lu_bursty``: directed Chung-Lu power law (vertex weight
    (i+1)^(-1/(gamma-1)), the same rank for out- and in-weight), 70% base edges
    with uniform times over the span and 30% re-emissions that append to the
    burst of a uniformly chosen base edge at gaps ceil(Exp(mean)).
Every graph has unique (u, v, t) tuples and no self loops (Sec. 1.1), and its
timestamps are offset by ``t0`` so that the t - t_min shift is exercised.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

T0 = 1_500_000_000  # absolute time offset of every generated graph


@dataclass
class TemporalGraph:
    n: int
    src: np.ndarray  # uint32
    dst: np.ndarray  # uint32
    t: np.ndarray    # int64

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


@dataclass
class Motif:
    """A temporal motif M = (H, pi, delta) (Def. 1.1).

    ``edges[i] = (a, b)`` is a directed pattern edge; ``rank[i]`` is its
    position in the order pi.  ``tree``/``root`` optionally pin the spanning
    tree (motif-edge indices) and its root edge.
    """
    name: str
    nv: int
    edges: list
    rank: list
    delta: int
    tree: list | None = None
    root: int | None = None
    k: int = 0
    meta: dict = field(default_factory=dict)


def _dedup_key(src: np.ndarray, dst: np.ndarray, n: int) -> np.ndarray:
    return src.astype(np.uint64) * np.uint64(n) + dst.astype(np.uint64)


def _unique_tuples(src, dst, t, n):
    """Drop repeated (u, v, t) tuples, keeping the first occurrence.

    A 64-bit mix of (u*n + v, t) finds the few entries whose hash repeats; only
    those are compared exactly (sorted by tuple, then by position), so every
    other entry is known unique without a full two-key sort."""
    key = _dedup_key(src, dst, n)
    with np.errstate(over="ignore"):
        h = key * np.uint64(0x9E3779B97F4A7C15) ^ (t.astype(np.uint64) * np.uint64(0xC2B2AE3D27D4EB4F))
        h ^= h >> np.uint64(29)
    hs = np.sort(h)
    rep = np.unique(hs[1:][hs[1:] == hs[:-1]])
    if rep.size == 0:
        return src, dst, t
    cand = np.nonzero(np.isin(h, rep))[0]
    ck, ct = key[cand], t[cand]
    order = np.lexsort((cand, ct, ck))
    ks, ts = ck[order], ct[order]
    dup = np.zeros(order.shape[0], dtype=bool)
    dup[1:] = (ks[1:] == ks[:-1]) & (ts[1:] == ts[:-1])
    keep = np.ones(src.shape[0], dtype=bool)
    keep[cand[order[dup]]] = False
    return src[keep], dst[keep], t[keep]


def uniform_graph(n: int, m: int, t_hi: int, seed: int, t0: int = T0) -> TemporalGraph:
    """src, dst uniform with src != dst; t uniform on [0, t_hi); unique tuples."""
    rng = np.random.default_rng(seed)
    src = np.zeros(0, np.uint32); dst = np.zeros(0, np.uint32); t = np.zeros(0, np.int64)
    while src.shape[0] < m:
        need = m - src.shape[0]
        s = rng.integers(0, n, size=need, dtype=np.uint32)
        d = rng.integers(0, n - 1, size=need, dtype=np.uint32)
        d = d + (d >= s).astype(np.uint32)        # uniform over vertices != s
        tt = rng.integers(0, t_hi, size=need, dtype=np.int64)
        src = np.concatenate([src, s]); dst = np.concatenate([dst, d]); t = np.concatenate([t, tt])
        src, dst, t = _unique_tuples(src, dst, t, n)
    perm = rng.permutation(src.shape[0])[:m]
    return TemporalGraph(n, src[perm], dst[perm], t[perm] + t0)


def _chung_lu_endpoints(rng, cdf, total, count, n):
    s = np.searchsorted(cdf, rng.random(count) * total, side="right").astype(np.uint32)
    d = np.searchsorted(cdf, rng.random(count) * total, side="right").astype(np.uint32)
    np.minimum(s, n - 1, out=s); np.minimum(d, n - 1, out=d)
    bad = np.nonzero(s == d)[0]
    while bad.size:
        d[bad] = np.minimum(np.searchsorted(cdf, rng.random(bad.size) * total, side="right"), n - 1)
        bad = bad[s[bad] == d[bad]]
    return s, d


def chung_lu_bursty(n: int, m: int, gamma: float, span: int, seed: int,
                    burst_frac: float = 0.3, burst_mean: float = 600.0, t0: int = T0) -> TemporalGraph:
    """Directed Chung-Lu power-law graph with bursty repeated (u, v) edges."""
    rng = np.random.default_rng(seed)
    w = np.power(np.arange(1, n + 1, dtype=np.float64), -1.0 / (gamma - 1.0))
    cdf = np.cumsum(w)
    total = float(cdf[-1])
    n_base = int(round(m * (1.0 - burst_frac)))
    n_rep = m - n_base
    bs, bd = _chung_lu_endpoints(rng, cdf, total, n_base, n)
    bt = rng.integers(0, span, size=n_base, dtype=np.int64)
    # re-emissions: each picks a base edge and extends its burst
    pick = np.sort(rng.integers(0, n_base, size=n_rep, dtype=np.int64))
    gaps = np.ceil(rng.exponential(burst_mean, size=n_rep)).astype(np.int64)
    gaps = np.maximum(gaps, 1)
    csum = np.cumsum(gaps)
    first = np.ones(n_rep, dtype=bool)
    first[1:] = pick[1:] != pick[:-1]
    start_idx = np.nonzero(first)[0]
    group = np.cumsum(first) - 1
    before = np.zeros(start_idx.shape[0], dtype=np.int64)
    before[1:] = csum[start_idx[1:] - 1]
    rt = bt[pick] + (csum - before[group])
    rt = np.minimum(rt, span - 1)
    src = np.concatenate([bs, bs[pick]])
    dst = np.concatenate([bd, bd[pick]])
    t = np.concatenate([bt, rt])
    src, dst, t = _unique_tuples(src, dst, t, n)
    while src.shape[0] < m:                      # top up after de-duplication
        need = m - src.shape[0]
        s, d = _chung_lu_endpoints(rng, cdf, total, need, n)
        tt = rng.integers(0, span, size=need, dtype=np.int64)
        src = np.concatenate([src, s]); dst = np.concatenate([dst, d]); t = np.concatenate([t, tt])
        src, dst, t = _unique_tuples(src, dst, t, n)
    perm = rng.permutation(src.shape[0])[:m]
    return TemporalGraph(n, src[perm].astype(np.uint32), dst[perm].astype(np.uint32), t[perm] + t0)


# ---------------------------------------------------------------------------
# Motifs of the workloads
# ---------------------------------------------------------------------------
def triangle(delta: int) -> Motif:
    """Temporal triangle u->v, v->w, w->u with t1 < t2 < t3."""
    return Motif("triangle", 3, [(0, 1), (1, 2), (2, 0)], [0, 1, 2], delta)


def cycle(nv: int, delta: int) -> Motif:
    """Directed temporal nv-cycle 0->1->...->0 in cycle order."""
    return Motif(f"cycle{nv}", nv, [(i, (i + 1) % nv) for i in range(nv)], list(range(nv)), delta)


def cycle5_chord(delta: int) -> Motif:
    """5-cycle with a 0->2 chord whose time lies between cycle edges 2 and 3."""
    return Motif("cycle5_chord", 5, [(0, 1), (1, 2), (0, 2), (2, 3), (3, 4), (4, 0)],
                 [0, 1, 2, 3, 4, 5], delta)


def single_edge(delta: int) -> Motif:
    return Motif("edge", 2, [(0, 1)], [0], delta)


def path(nv: int, delta: int) -> Motif:
    return Motif(f"path{nv}", nv, [(i, i + 1) for i in range(nv - 1)], list(range(nv - 1)), delta)


def _connected(nv, edges):
    comp = list(range(nv))
    for a, b in edges:
        ca, cb = comp[a], comp[b]
        comp = [ca if c == cb else c for c in comp]
    return len(set(comp)) == 1


def motif_pool(seed: int, count: int = 32, deltas=(600, 3600, 86400),
               k_lo: float = 1e4, k_hi: float = 1e7) -> list[Motif]:
    """Seeded pool of 3-7-vertex ordered motifs: triangles, stars (in, out,
    mixed), paths, cycles with 0-2 chords and random connected patterns, each
    with a delta from ``deltas`` and a log-uniform sample count k."""
    rng = np.random.default_rng(seed)
    kinds = ["triangle", "out_star", "in_star", "mixed_star", "path", "cycle", "cycle_chord", "random"]
    out = []
    for q in range(count):
        kind = kinds[q % len(kinds)]
        nv = int(rng.integers(3, 8))
        if kind == "triangle":
            nv = 3
            edges = [(0, 1), (1, 2), (2, 0)] if rng.random() < 0.5 else [(0, 1), (1, 2), (0, 2)]
        elif kind == "out_star":
            edges = [(0, i) for i in range(1, nv)]
        elif kind == "in_star":
            edges = [(i, 0) for i in range(1, nv)]
        elif kind == "mixed_star":
            edges = [(0, i) if rng.random() < 0.5 else (i, 0) for i in range(1, nv)]
        elif kind == "path":
            edges = [(i, i + 1) if rng.random() < 0.7 else (i + 1, i) for i in range(nv - 1)]
        elif kind in ("cycle", "cycle_chord"):
            nv = max(nv, 4) if kind == "cycle_chord" else nv
            edges = [(i, (i + 1) % nv) for i in range(nv)]
            if kind == "cycle_chord":
                nch = int(rng.integers(1, 3))
                for _ in range(nch):
                    a = int(rng.integers(0, nv)); b = (a + int(rng.integers(2, nv - 1))) % nv
                    if (a, b) not in edges and (b, a) not in edges:
                        edges.append((a, b))
        else:
            while True:
                ne = int(rng.integers(nv - 1, min(nv + 3, 10)))
                edges = []
                # random spanning tree, then extra edges
                for v in range(1, nv):
                    u = int(rng.integers(0, v))
                    edges.append((u, v) if rng.random() < 0.5 else (v, u))
                while len(edges) < ne:
                    a, b = (int(x) for x in rng.choice(nv, size=2, replace=False))
                    edges.append((a, b))
                if _connected(nv, edges):
                    break
        ne = len(edges)
        rank = [int(x) for x in rng.permutation(ne)] if kind in ("random", "mixed_star") else list(range(ne))
        delta = int(deltas[int(rng.integers(0, len(deltas)))])
        k = int(round(math.exp(rng.uniform(math.log(k_lo), math.log(k_hi)))))
        out.append(Motif(f"{kind}{q}", nv, edges, rank, delta, k=k))
    return out


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------
WORKLOADS = {
    # tiny: uniform graph, temporal triangle; oracle finishes in seconds
    "tiny": dict(kind="uniform", n=1000, m=20_000, t_hi=1_000_000, seed=1,
                 motif=lambda: triangle(10_000), k=100_000),
    # dense tiny companion with a non-trivial exact count
    "dense_tiny": dict(kind="uniform", n=100, m=20_000, t_hi=1_000_000, seed=1,
                       motif=lambda: triangle(100_000), k=100_000),
    # Chung-Lu 2M edges, temporal 4-cycle
    "cl2m_cycle4": dict(kind="chung_lu", n=100_000, m=2_000_000, gamma=2.1, span=30_000_000, seed=1,
                        motif=lambda: cycle(4, 86_400), k=1_000_000),
    # Chung-Lu 50M edges, 5-cycle plus chord
    "cl50m_cycle5chord": dict(kind="chung_lu", n=2_000_000, m=50_000_000, gamma=2.1, span=100_000_000,
                              seed=1, motif=lambda: cycle5_chord(3_600), k=10_000_000),
    # medium-size companion of the 50M-edge workload (profiling captures)
    "cl10m_cycle5chord": dict(kind="chung_lu", n=400_000, m=10_000_000, gamma=2.1, span=20_000_000,
                              seed=1, motif=lambda: cycle5_chord(3_600), k=2_000_000),
    # serving graph: Chung-Lu 200M edges
    "cl200m": dict(kind="chung_lu", n=10_000_000, m=200_000_000, gamma=2.2, span=100_000_000, seed=1,
                   motif=None, k=0),
}


def make_graph(name: str, **override) -> TemporalGraph:
    cfg = dict(WORKLOADS[name]); cfg.update(override)
    if cfg["kind"] == "uniform":
        return uniform_graph(cfg["n"], cfg["m"], cfg["t_hi"], cfg["seed"])
    return chung_lu_bursty(cfg["n"], cfg["m"], cfg["gamma"], cfg["span"], cfg["seed"])


def make_motif(name: str) -> Motif:
    cfg = WORKLOADS[name]
    mo = cfg["motif"]()
    mo.k = cfg["k"]
    return mo
