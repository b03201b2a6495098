"""The multi-GPU layout on CPU: samples are independent units, so N ranks
each drawing a disjoint range of sample ids (tm_sample's first_index) and
adding their integer sums reproduce one run exactly.  Two gloo ranks run the
CPU oracle over their shares and combine hits2 and the counters through the
same function bench.py's torchrun path calls (bench.combine_across_ranks, one
integer all-reduce); the sum equals the single-process result."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from helpers import small_random_graph
    from paper_2507_20441_gb300.shard import sample_range, combine
    n, s, d, t = small_random_graph(31, n=9, m=400, t_hi=150)
    G = oracle.Graph(n, s, d, t)
    G.set_motif(4, [(0, 1), (1, 2), (2, 3), (3, 0)], [0, 1, 2, 3], 25, [0, 1, 2], 1)
    G.weights()
    k = 30_001
    first, cnt = sample_range(rank, world, k)
    r = G.sample(cnt, 5, first)
    import bench
    out[rank] = tuple(bench.combine_across_ranks(r))      # the bench's own combine step
    # the same sums through the limb encoding directly
    limbs = torch.tensor(combine.to_limbs(r.hits2, r.valid, r.rej_vertex, r.rej_delta, r.rej_order), dtype=torch.int64)
    dist.all_reduce(limbs)
    assert combine.from_limbs(limbs.tolist()) == out[rank]
    dist.destroy_process_group()


def _bench_layout_rank(rank, world, port, out):
    """bench.py's per-step id layout: rank r of N draws k ids from (i N + r) k."""
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from helpers import small_random_graph
    n, s, d, t = small_random_graph(33, n=9, m=500, t_hi=150)
    G = oracle.Graph(n, s, d, t)
    G.set_motif(3, [(0, 1), (1, 2), (2, 0)], [0, 1, 2], 30, [0, 1], 1)
    G.weights()
    k, step = 7_001, 3
    r = G.sample(k, 11, (step * world + rank) * k)
    out[rank] = tuple(bench.combine_across_ranks(r))
    dist.destroy_process_group()


def test_bench_rank_layout_covers_one_contiguous_range():
    import multiprocessing as mp
    import oracle
    from helpers import small_random_graph
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_bench_layout_rank, args=(r, 3, port, out)) for r in range(3)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    n, s, d, t = small_random_graph(33, n=9, m=500, t_hi=150)
    G = oracle.Graph(n, s, d, t)
    G.set_motif(3, [(0, 1), (1, 2), (2, 0)], [0, 1, 2], 30, [0, 1], 1)
    G.weights()
    whole = G.sample(3 * 7_001, 11, 3 * 3 * 7_001)
    assert whole.valid > 0
    for r in range(3):
        assert out[r] == (whole.hits2, whole.valid, whole.rej_vertex, whole.rej_delta, whole.rej_order)


def test_two_gloo_ranks_equal_one_run():
    import multiprocessing as mp
    import oracle
    from helpers import small_random_graph
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    n, s, d, t = small_random_graph(31, n=9, m=400, t_hi=150)
    G = oracle.Graph(n, s, d, t)
    G.set_motif(4, [(0, 1), (1, 2), (2, 3), (3, 0)], [0, 1, 2, 3], 25, [0, 1, 2], 1)
    G.weights()
    whole = G.sample(30_001, 5, 0)
    for r in range(2):
        assert out[r] == (whole.hits2, whole.valid, whole.rej_vertex, whole.rej_delta, whole.rej_order)


def test_sample_ranges_partition():
    from paper_2507_20441_gb300.shard import sample_range
    for world in (1, 2, 3, 8):
        for k in (0, 1, 7, 1000, 12345):
            got = [sample_range(r, world, k) for r in range(world)]
            ids = [i for f, c in got for i in range(f, f + c)]
            assert ids == list(range(k))


def test_limb_roundtrip_of_128_bit_sums():
    from paper_2507_20441_gb300.shard import combine
    big = (1 << 100) + 12345
    limbs = combine.to_limbs(big, 1, 2, 3, 4)
    assert all(0 <= x < 2**63 for x in limbs)
    assert combine.from_limbs(limbs) == (big, 1, 2, 3, 4)
    # sums of limbs over many ranks stay exact
    a = combine.to_limbs((1 << 120) - 1, 5, 0, 0, 0)
    b = combine.to_limbs(1, 6, 0, 0, 0)
    assert combine.from_limbs([x + y for x, y in zip(a, b)]) == (1 << 120, 11, 0, 0, 0)
