"""Every array of the temporal CSR (Defs. 3.1-3.3) built by the CUDA path,
element by element against the oracle's plain definition (stable sorts and
searches over the oracle's GLOBAL order).

The cases cover one, two and three radix passes per sort (vertex ids of 6,
17 and 21 bits), the inverse permutations written through one bucket and
through hundreds, runs of equal times, hub lists whose cross ranks take the
warp-bracketed search, and ragged last tiles and warps.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tg():
    import paper_2507_20441_gb300 as tg
    tg.build()
    return tg


def check_csr(tg, oracle_mod, n, s, d, t, dedup=False):
    ctx = tg.Context()
    ctx.load_graph(n, s, d, t, flags=tg.TM_DEDUP if dedup else 0)
    G = oracle_mod.Graph(n, s, d, t, flags=oracle_mod.DEDUP if dedup else 0)
    assert ctx.m == G.m
    want = G.csr()
    for name in tg.CSR_ARRAYS:
        got = ctx.csr(name)
        exp = want[name]
        assert got.shape == exp.shape, (name, got.shape, exp.shape)
        bad = np.flatnonzero(got != exp)
        assert bad.size == 0, (name, int(bad[0]), int(got[bad[0]]), int(exp[bad[0]]))
    ctx.close()


@pytest.mark.parametrize("t_hi,m", [(3, 6000), (5, 3000)])
def test_csr_small_equal_times(tg, oracle_mod, t_hi, m):
    """Runs of hundreds of equal times, duplicates dropped; 4096 edges kept
    (one full tile) and 2658 (a ragged tile and a partial last warp)."""
    rng = np.random.default_rng(5)
    n = 50
    s = rng.integers(0, n, m).astype(np.uint32)
    d = ((s + 1 + rng.integers(0, n - 1, m)) % n).astype(np.uint32)
    t = (rng.integers(0, t_hi, m) + 11).astype(np.int64)
    check_csr(tg, oracle_mod, n, s, d, t, dedup=True)


def test_csr_tiny_workload(tg, oracle_mod):
    from paper_2507_20441_gb300 import synth
    gr = synth.make_graph("tiny")
    check_csr(tg, oracle_mod, gr.n, gr.src, gr.dst, gr.t)


@pytest.mark.parametrize("n,m", [(100_000, 2_000_011), (2_000_000, 3_000_017)])
def test_csr_chung_lu(tg, oracle_mod, n, m):
    """Power-law degrees: hub lists of thousands of entries, 2 and 3 radix
    passes, about 490 and 370 buckets in the inverse permutations."""
    from paper_2507_20441_gb300 import synth
    gr = synth.chung_lu_bursty(n, m, 2.1, 30_000_000, 3)
    check_csr(tg, oracle_mod, gr.n, gr.src, gr.dst, gr.t)


def test_csr_wide_time_span(tg, oracle_mod):
    """Times over almost the whole u32 range of t' (negative inputs, span
    2^32 - 2): the time sort's widest key, five 7-bit passes."""
    rng = np.random.default_rng(11)
    n, m = 1000, 5003
    s = rng.integers(0, n, m).astype(np.uint32)
    d = ((s + 1 + rng.integers(0, n - 1, m)) % n).astype(np.uint32)
    t = rng.integers(-2**31 + 1, 2**31 - 1, m).astype(np.int64)
    t[0], t[1] = -2**31, 2**31 - 2
    check_csr(tg, oracle_mod, n, s, d, t, dedup=True)
