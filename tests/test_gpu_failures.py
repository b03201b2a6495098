"""Failure handling on the host side of the GPU path, without faulting the
GPU: a device allocator hook (tm_config.alloc) that refuses chosen requests.

* Every allocation point of a whole estimate (context, graph load and CSR
  build, weight pass, traced sampling) is made to fail once in turn: the call
  that needed the memory returns TM_E_NOMEM, the same call then succeeds on
  the same context, and the final weights, W, per-sample trace and hits2 equal
  those of a run without failures.
* Serving: weight passes refused by the allocator make admission back off
  (free unused cached weights, wait, retry) and the query still completes with
  the result it gives alone; the back-offs are counted.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


class Hook:
    """Allocator hooks over PyTorch's caching allocator that refuse the
    requests whose 1-based call numbers are in `fail`, or every request while
    `refuse` is set."""

    def __init__(self, device=0):
        import torch
        import paper_2507_20441_gb300 as tg
        self.torch = torch
        self.calls = 0
        self.fail = set()
        self.refuse = 0          # refuse this many further requests
        self.refused = 0

        def _alloc(nbytes, stream, user):
            self.calls += 1
            if self.calls in self.fail or self.refuse > 0:
                if self.refuse > 0:
                    self.refuse -= 1
                self.refused += 1
                return None
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0)))
            except Exception:
                return None

        def _free(ptr, nbytes, stream, user):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.hooks = (tg.ALLOC_FN(_alloc), tg.FREE_FN(_free))


def _graph():
    from paper_2507_20441_gb300 import synth
    return synth.chung_lu_bursty(3000, 60_000, 2.1, 2_000_000, seed=5)


CYCLE4 = (4, [(0, 1), (1, 2), (2, 3), (3, 0)], [0, 1, 2, 3], 86_400)
K_TRACE = 3_000_000      # the trace buffer (60 MB) needs a fresh scratch chunk
K = 200_000


def _pipeline(tg, hook, gr):
    """create -> load + CSR -> weights -> traced sample -> sample, retrying a
    step once when it reports TM_E_NOMEM.  Returns (results, failed steps)."""
    failed = []

    def step(name, fn):
        try:
            return fn()
        except tg.TimestError as e:
            assert e.code == tg.TM_E_NOMEM, (name, e)
            failed.append(name)
            return fn()

    ctx = step("create", lambda: tg.Context(alloc_hooks=hook.hooks))
    step("load", lambda: ctx.load_graph(gr.n, gr.src, gr.dst, gr.t))
    nv, edges, rank, delta = CYCLE4
    mo = ctx.motif(nv, edges, rank, delta)
    W = step("weights", mo.weights)
    w = [mo.export_weights(e, layer) for e in mo.plan()[0] for layer in (0, 1)]
    tr = step("trace", lambda: mo.sample_trace(K_TRACE, 3))
    r = step("sample", lambda: mo.sample(K, 4))
    out = (W, w, tr[0].hits2, tr[1], tr[2], tr[3], (r.hits2, r.valid, r.rej_vertex, r.rej_delta, r.rej_order))
    ctx.close()
    return out, failed


def _same(a, b):
    W, w, h, g, c, why, r = a
    W2, w2, h2, g2, c2, why2, r2 = b
    return (W == W2 and all(np.array_equal(x, y) for x, y in zip(w, w2)) and h == h2 and
            np.array_equal(g, g2) and np.array_equal(c, c2) and np.array_equal(why, why2) and r == r2)


def test_every_allocation_point_fails_cleanly():
    import paper_2507_20441_gb300 as tg
    tg.build()
    gr = _graph()
    clean_hook = Hook()
    clean, failed = _pipeline(tg, clean_hook, gr)
    assert failed == [] and clean_hook.refused == 0
    ncalls = clean_hook.calls
    assert ncalls >= 5, ncalls          # context, input, graph, scratch, motif, trace scratch
    seen = set()
    for n in range(1, ncalls + 1):
        hook = Hook()
        hook.fail = {n}
        got, failed = _pipeline(tg, hook, gr)
        assert hook.refused == 1, n
        assert len(failed) == 1, (n, failed)      # exactly the step that needed call n
        seen.add(failed[0])
        assert _same(got, clean), (n, failed)
    # every step that allocates was made to fail at least once
    assert {"create", "load", "weights", "trace"} <= seen, seen


def test_serving_backs_off_when_memory_runs_out():
    import paper_2507_20441_gb300 as tg
    gr = _graph()
    hook = Hook()
    ctx = tg.Context(alloc_hooks=hook.hooks)
    ctx.load_graph(gr.n, gr.src, gr.dst, gr.t)
    nv, edges, rank, delta = CYCLE4
    alone = ctx.motif(nv, edges, rank, delta)
    alone.weights()
    want = alone.sample(K, 9)
    alone.free()
    ctx.serve_start(max_active=4)
    hook.refuse = 6                      # the admission's first weight passes find no memory
    t = ctx.submit(nv, edges, rank, delta, K, 9)
    got = ctx.poll(t, timeout_ms=120_000)
    st = ctx.serve_stats()
    ctx.serve_stop()
    assert hook.refused == 6
    assert st["completed"] == 1 and st["failed"] == 0
    assert st["nomem_retries"] >= 1
    assert (got.W, got.hits2, got.valid, got.rej_vertex, got.rej_delta, got.rej_order) == \
           (want.W, want.hits2, want.valid, want.rej_vertex, want.rej_delta, want.rej_order)
    ctx.close()
