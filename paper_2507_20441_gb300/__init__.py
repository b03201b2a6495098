"""GB300-native TIMEST: temporal-motif count estimation by spanning-tree
sampling (Pan, Bhalerao, Seshadhri, Talati, arXiv 2507.20441).

A thin ctypes binding of the C ABI in ``include/timest.h`` -- the functions
below carry the same names (``tm_create``, ``tm_graph_load``, ...) and only
marshal arguments; every step of the estimator runs in the CUDA library
``_build/libtimest_gb300.so``.  PyTorch supplies device memory (its caching
allocator, through the allocator hooks of ``tm_config``) and the CUDA stream.

There is no CPU fallback: if the library is missing or cannot be loaded,
every call raises ``TimestUnavailable``.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# TIMEST_GB300_LIB names another build of the same library (e.g. one compiled
# with different launch bounds for a comparison)
LIB_PATH = os.environ.get("TIMEST_GB300_LIB") or os.path.join(_HERE, "_build", "libtimest_gb300.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "timest.h")

TM_OK, TM_E_ARG, TM_E_DUP, TM_E_SELFLOOP, TM_E_MOTIF, TM_E_NOMEM, TM_E_OVERFLOW, TM_E_STATE, TM_E_TIMEOUT, \
    TM_E_CUDA, TM_E_LIMIT, TM_E_PENDING = range(12)
TM_C2, TM_C3 = 1, 2
TM_HOST, TM_DEVICE, TM_DEDUP, TM_DROP_SELF, TM_PREPROCESS = 0, 1, 2, 4, 8
_STATUS_NAMES = {0: "TM_OK", 1: "TM_E_ARG", 2: "TM_E_DUP", 3: "TM_E_SELFLOOP", 4: "TM_E_MOTIF", 5: "TM_E_NOMEM",
                 6: "TM_E_OVERFLOW", 7: "TM_E_STATE", 8: "TM_E_TIMEOUT", 9: "TM_E_CUDA", 10: "TM_E_LIMIT",
                 11: "TM_E_PENDING"}


class TimestUnavailable(RuntimeError):
    """The CUDA library is not built or cannot be loaded."""


class TimestError(RuntimeError):
    def __init__(self, code: int, what: str, msg: str = ""):
        super().__init__(f"{what} failed: {_STATUS_NAMES.get(code, code)} {msg}".strip())
        self.code = code


class tm_u128(C.Structure):
    _fields_ = [("lo", C.c_uint64), ("hi", C.c_uint64)]

    @property
    def value(self) -> int:
        return int(self.lo) | (int(self.hi) << 64)


class tm_tree_cand(C.Structure):
    _fields_ = [("tree_mask", C.c_uint32), ("root", C.c_uint32), ("looseness", C.c_uint32), ("status", C.c_int32),
                ("W", tm_u128)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class tm_config(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p), ("device", C.c_int),
                ("sample_threads", C.c_int), ("sample_tile", C.c_int), ("profile", C.c_int),
                ("reserved", C.c_int * 7)]


class tm_result(C.Structure):
    _fields_ = [("W", tm_u128), ("hits2", tm_u128), ("k", C.c_uint64), ("valid", C.c_uint64),
                ("rej_vertex", C.c_uint64), ("rej_delta", C.c_uint64), ("rej_order", C.c_uint64),
                ("estimate", C.c_double)]


@dataclass
class Result:
    W: int
    hits2: int
    k: int
    valid: int
    rej_vertex: int
    rej_delta: int
    rej_order: int
    estimate: float

    @staticmethod
    def of(r: tm_result) -> "Result":
        return Result(r.W.value, r.hits2.value, int(r.k), int(r.valid), int(r.rej_vertex), int(r.rej_delta),
                      int(r.rej_order), float(r.estimate))


class tm_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 96), ("ms", C.c_double), ("launches", C.c_uint64)]


class tm_tune_entry(C.Structure):
    _fields_ = [("tile", C.c_int), ("threads", C.c_int), ("smem_records", C.c_int), ("coop_min", C.c_int),
                ("ms", C.c_double)]

    def as_dict(self):
        return {"tile": self.tile, "threads": self.threads, "smem_records": self.smem_records,
                "coop_min": self.coop_min, "ms": self.ms}


class tm_serve_cfg(C.Structure):
    _fields_ = [("max_active", C.c_uint32), ("tile", C.c_uint32), ("round_tiles", C.c_uint32),
                ("poll_timeout_ms", C.c_int32), ("weight_budget", C.c_uint64), ("reserved", C.c_int32 * 8)]


class tm_serve_stats_t(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("cache_hits", C.c_uint64), ("cache_misses", C.c_uint64), ("evictions", C.c_uint64),
                ("rounds", C.c_uint64), ("resident_bytes", C.c_uint64), ("waiting", C.c_uint64),
                ("active", C.c_uint64), ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double),
                ("qps", C.c_double), ("nomem_retries", C.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
_load_error = None


def _declare(L):
    vp, u32, u64, i32, i64 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int, C.c_int64
    pv = C.POINTER(C.c_void_p)
    L.tm_config_default.argtypes = [C.POINTER(tm_config)]; L.tm_config_default.restype = None
    L.tm_create.argtypes = [pv, C.POINTER(tm_config), vp]
    L.tm_destroy.argtypes = [vp]; L.tm_destroy.restype = None
    L.tm_last_error.argtypes = [vp]; L.tm_last_error.restype = C.c_char_p
    L.tm_graph_load.argtypes = [vp, u32, u64, vp, vp, vp, i32]
    L.tm_preprocess.argtypes = [vp]
    L.tm_graph_info.argtypes = [vp, C.POINTER(u64), C.POINTER(i64), C.POINTER(i64)]
    L.tm_edges_export.argtypes = [vp, vp, vp, vp]
    L.tm_csr_export.argtypes = [vp, i32, vp, u64, C.POINTER(u64)]
    L.tm_set_motif.argtypes = [vp, u32, u32, vp, vp, i64, pv]
    L.tm_set_tree.argtypes = [vp, vp, u32]
    L.tm_set_constraints.argtypes = [vp, i32]
    L.tm_tree_candidates.argtypes = [u32, u32, vp, vp, u32, vp, vp, C.POINTER(u32)]
    L.tm_sample_list.argtypes = [vp, vp, u64, u64, u64, u64, vp, vp, C.POINTER(u64)]
    L.tm_sample_group.argtypes = [vp, vp, u32, u64, u64, u64, vp]
    L.tm_select_tree.argtypes = [vp, u32, u32, vp, vp, i64, u32, i32, pv, vp, u32, C.POINTER(u32)]
    L.tm_motif_plan.argtypes = [vp, vp, vp]
    L.tm_weights.argtypes = [vp, vp, C.POINTER(tm_u128)]
    L.tm_weights_export.argtypes = [vp, vp, u32, u32, vp]
    L.tm_window_totals.argtypes = [vp, vp, vp, u64, C.POINTER(u64)]
    L.tm_sample.argtypes = [vp, vp, u64, u64, u64, C.POINTER(tm_result)]
    L.tm_sample_trace.argtypes = [vp, vp, u64, u64, u64, vp, vp, vp, C.POINTER(tm_result)]
    L.tm_sample_noalloc.argtypes = [vp, vp, u64, u64, u64, C.POINTER(tm_result)]
    L.tm_batch_run.argtypes = [vp, u32, vp, vp, vp, vp]
    L.tm_motif_free.argtypes = [vp]; L.tm_motif_free.restype = None
    L.tm_phase_times.argtypes = [vp, vp, vp, i32, C.POINTER(i32)]
    L.tm_autotune.argtypes = [vp, u32, vp, vp, vp, u64, C.POINTER(tm_tune_entry), u32, C.POINTER(u32),
                              C.POINTER(tm_tune_entry)]
    L.tm_batch_shape.argtypes = [vp, i32, i32, i32]
    L.tm_coop_search.argtypes = [vp, u32]
    L.tm_serve_start.argtypes = [vp, C.POINTER(tm_serve_cfg)]
    L.tm_serve_submit.argtypes = [vp, u32, u32, vp, vp, i64, u64, u64, C.POINTER(u64)]
    L.tm_serve_submit_motif.argtypes = [vp, vp, u64, u64, C.POINTER(u64)]
    L.tm_serve_poll.argtypes = [vp, u64, C.POINTER(tm_result), i32]
    L.tm_serve_stats.argtypes = [vp, C.POINTER(tm_serve_stats_t)]
    L.tm_serve_stop.argtypes = [vp]
    L.tm_io_bytes.argtypes = [vp, C.POINTER(u64), C.POINTER(u64)]
    L.tm_kernel_times.argtypes = [vp, C.POINTER(tm_kernel_time), u32, C.POINTER(u32)]
    return L


def lib():
    """Load the CUDA library (raises TimestUnavailable if it is not built)."""
    global _lib, _load_error
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise TimestUnavailable(f"TIMEST CUDA library not built ({LIB_PATH}); run __graft_entry__.build()")
    try:
        _lib = _declare(C.CDLL(LIB_PATH))
    except OSError as e:
        _load_error = e
        raise TimestUnavailable(f"cannot load {LIB_PATH}: {e}") from e
    return _lib


def build(force: bool = False) -> str:
    from . import _build
    path = _build.build(force=force)
    return path


def _ptr(a) -> C.c_void_p:
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(int(a.data_ptr()))   # torch tensor


def _check(rc: int, ctx, what: str):
    if rc != TM_OK:
        msg = lib().tm_last_error(ctx).decode() if ctx else ""
        raise TimestError(rc, what, msg)


# ---------------------------------------------------------------------------
# torch allocator hooks (device memory comes from PyTorch's caching allocator)
# ---------------------------------------------------------------------------
class _TorchAllocator:
    def __init__(self, device: int):
        import torch
        self.torch = torch
        self.device = device

        def _alloc(nbytes, stream, user):
            try:
                return int(self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0)))
            except Exception:
                return None

        def _free(ptr, nbytes, stream, user):
            try:
                self.torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


# ---------------------------------------------------------------------------
# C-ABI functions under their own names
# ---------------------------------------------------------------------------
def tm_create(device: int = 0, stream=None, torch_allocator: bool = True, sample_threads: int = 0,
              sample_tile: int = 0, alloc_hooks=None, profile: bool = False):
    """Returns an opaque context handle (c_void_p) plus the objects that must
    stay alive with it."""
    L = lib()
    cfg = tm_config()
    L.tm_config_default(C.byref(cfg))
    cfg.device = device
    cfg.sample_threads = sample_threads
    cfg.sample_tile = sample_tile
    cfg.profile = int(profile)
    keep = []
    if alloc_hooks is not None:
        cfg.alloc, cfg.free = alloc_hooks
        keep.append(alloc_hooks)
    elif torch_allocator:
        ta = _TorchAllocator(device)
        cfg.alloc, cfg.free = ta.alloc, ta.free
        keep.append(ta)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream(device).cuda_stream
    h = C.c_void_p()
    rc = L.tm_create(C.byref(h), C.byref(cfg), C.c_void_p(int(stream) if stream else 0))
    if rc != TM_OK:
        raise TimestError(rc, "tm_create")
    return h, keep


def tm_destroy(ctx):
    lib().tm_destroy(ctx)


def tm_last_error(ctx) -> str:
    return lib().tm_last_error(ctx).decode()


def tm_graph_load(ctx, n, src, dst, t, flags=TM_HOST):
    """src/dst (uint32) and t (int64): numpy arrays (TM_HOST) or CUDA tensors
    (pass TM_DEVICE)."""
    m = len(src)
    if flags & TM_DEVICE:
        import torch
        torch.cuda.synchronize()          # inputs written on torch's streams
        ps, pd, pt = _ptr(src), _ptr(dst), _ptr(t)
    else:
        src = np.ascontiguousarray(src, dtype=np.uint32)
        dst = np.ascontiguousarray(dst, dtype=np.uint32)
        t = np.ascontiguousarray(t, dtype=np.int64)
        ps, pd, pt = _ptr(src), _ptr(dst), _ptr(t)
    _check(lib().tm_graph_load(ctx, int(n), m, ps, pd, pt, flags), ctx, "tm_graph_load")


def tm_preprocess(ctx):
    _check(lib().tm_preprocess(ctx), ctx, "tm_preprocess")


def tm_graph_info(ctx):
    m, tmin, T = C.c_uint64(), C.c_int64(), C.c_int64()
    _check(lib().tm_graph_info(ctx, C.byref(m), C.byref(tmin), C.byref(T)), ctx, "tm_graph_info")
    return int(m.value), int(tmin.value), int(T.value)


def tm_edges_export(ctx):
    m, _, _ = tm_graph_info(ctx)
    s = np.zeros(m, np.uint32); d = np.zeros(m, np.uint32); t = np.zeros(m, np.uint32)
    _check(lib().tm_edges_export(ctx, _ptr(s), _ptr(d), _ptr(t)), ctx, "tm_edges_export")
    return s, d, t


CSR_ARRAYS = ("out_off", "out_t", "out_nbr", "out_gid", "out_src", "out_pos", "out_xrank",
              "in_off", "in_t", "in_nbr", "in_gid", "in_dst", "in_pos", "in_xrank", "in_to_out",
              "vpair_off", "pair_off", "pair_dst", "multi_t", "multi_to_out", "own_out", "own_in", "own_multi")


def tm_csr_export(ctx, name):
    """One array of the temporal CSR (names as CSR_ARRAYS; see tm_csr_export in timest.h)."""
    which = CSR_ARRAYS.index(name)
    n = C.c_uint64()
    _check(lib().tm_csr_export(ctx, which, None, 0, C.byref(n)), ctx, "tm_csr_export")
    out = np.zeros(n.value, np.uint32)
    _check(lib().tm_csr_export(ctx, which, _ptr(out), n.value, C.byref(n)), ctx, "tm_csr_export")
    return out


def tm_set_motif(ctx, nv, edges, order, delta):
    e = np.ascontiguousarray(np.array(edges, dtype=np.uint32).reshape(-1))
    o = np.ascontiguousarray(np.array(order, dtype=np.uint32))
    h = C.c_void_p()
    _check(lib().tm_set_motif(ctx, int(nv), len(o), _ptr(e), _ptr(o), int(delta), C.byref(h)), ctx, "tm_set_motif")
    return h


def tm_set_tree(ctx, motif, tree, root):
    tr = np.ascontiguousarray(np.array(tree, dtype=np.uint32))
    _check(lib().tm_set_tree(motif, _ptr(tr), int(root)), ctx, "tm_set_tree")


def tm_set_constraints(ctx, motif, c2=True, c3=True):
    """Keep or drop Constraints 2 and 3 of a motif (ablation)."""
    flags = (TM_C2 if c2 else 0) | (TM_C3 if c3 else 0)
    _check(lib().tm_set_constraints(motif, flags), ctx, "tm_set_constraints")


def tm_tree_candidates(nv, edges, order):
    """Every spanning tree, best looseness first: [(edge mask, looseness)]."""
    e = np.ascontiguousarray(np.array(edges, dtype=np.uint32).reshape(-1))
    o = np.ascontiguousarray(np.array(order, dtype=np.uint32))
    total = C.c_uint32()
    rc = lib().tm_tree_candidates(int(nv), len(o), _ptr(e), _ptr(o), 0, None, None, C.byref(total))
    if rc != TM_OK:
        raise TimestError(rc, "tm_tree_candidates")
    n = total.value
    masks = np.zeros(max(n, 1), np.uint32); loose = np.zeros(max(n, 1), np.uint32)
    rc = lib().tm_tree_candidates(int(nv), len(o), _ptr(e), _ptr(o), n, _ptr(masks), _ptr(loose), C.byref(total))
    if rc != TM_OK:
        raise TimestError(rc, "tm_tree_candidates")
    return [(int(masks[i]), int(loose[i])) for i in range(n)]


def tm_select_tree(ctx, nv, edges, order, delta, n_c, all_roots=True):
    """Alg. 7 on the current graph: (winning motif handle, evaluated candidates)."""
    e = np.ascontiguousarray(np.array(edges, dtype=np.uint32).reshape(-1))
    o = np.ascontiguousarray(np.array(order, dtype=np.uint32))
    cap = max(1, int(n_c)) * max(1, int(nv) - 1)
    cands = (tm_tree_cand * cap)()
    n = C.c_uint32()
    h = C.c_void_p()
    _check(lib().tm_select_tree(ctx, int(nv), len(o), _ptr(e), _ptr(o), int(delta), int(n_c), 1 if all_roots else 0,
                                C.byref(h), C.cast(cands, C.c_void_p), cap, C.byref(n)), ctx, "tm_select_tree")
    out = [{"tree_mask": int(c.tree_mask), "root": int(c.root), "looseness": int(c.looseness),
            "status": int(c.status), "W": c.W.value} for c in cands[:min(n.value, cap)]]
    return h, out


def tm_sample_list(ctx, motif, ne, k, seed, first_index=0, max_inst=1_000_000):
    """Motif instances extending the valid samples: (edge ids [rows, ne],
    sample ids [rows], total instances)."""
    cap = int(max_inst)
    gids = np.zeros((max(cap, 1), int(ne)), np.uint32)
    sids = np.zeros(max(cap, 1), np.uint64)
    n = C.c_uint64()
    _check(lib().tm_sample_list(ctx, motif, int(k), int(seed), int(first_index), cap, _ptr(gids), _ptr(sids),
                                C.byref(n)), ctx, "tm_sample_list")
    rows = min(cap, n.value)
    return gids[:rows], sids[:rows], int(n.value)


def tm_sample_group(ctx, motifs, k, seed, first_index=0):
    """One sampling run for motifs sharing a tree pattern: a Result per motif."""
    n = len(motifs)
    hs = (C.c_void_p * n)(*[m for m in motifs])
    res = (tm_result * n)()
    _check(lib().tm_sample_group(ctx, C.cast(hs, C.c_void_p), n, int(k), int(seed), int(first_index),
                                 C.cast(res, C.c_void_p)), ctx, "tm_sample_group")
    return [Result.of(r) for r in res]


def tm_motif_plan(motif, ntree):
    order = np.zeros(ntree, np.int32); parent = np.zeros(ntree, np.int32)
    rc = lib().tm_motif_plan(motif, _ptr(order), _ptr(parent))
    if rc != TM_OK:
        raise TimestError(rc, "tm_motif_plan")
    return order, parent


def tm_weights(ctx, motif) -> int:
    W = tm_u128()
    _check(lib().tm_weights(ctx, motif, C.byref(W)), ctx, "tm_weights")
    return W.value


def tm_weights_export(ctx, motif, tree_edge, layer, m):
    out = np.zeros(m, np.uint64)
    _check(lib().tm_weights_export(ctx, motif, int(tree_edge), int(layer), _ptr(out)), ctx, "tm_weights_export")
    return out


def tm_window_totals(ctx, motif):
    nw = C.c_uint64()
    _check(lib().tm_window_totals(ctx, motif, None, 0, C.byref(nw)), ctx, "tm_window_totals")
    out = np.zeros(int(nw.value), np.uint64)
    _check(lib().tm_window_totals(ctx, motif, _ptr(out), len(out), C.byref(nw)), ctx, "tm_window_totals")
    return out


def tm_sample(ctx, motif, k, seed, first_index=0) -> Result:
    r = tm_result()
    _check(lib().tm_sample(ctx, motif, int(k), int(seed), int(first_index), C.byref(r)), ctx, "tm_sample")
    return Result.of(r)


def tm_sample_noalloc(ctx, motif, k, seed, first_index=0) -> Result:
    """tm_sample without any device allocation (scratch in a fixed array)."""
    r = tm_result()
    _check(lib().tm_sample_noalloc(ctx, motif, int(k), int(seed), int(first_index), C.byref(r)), ctx,
           "tm_sample_noalloc")
    return Result.of(r)


def tm_sample_trace(ctx, motif, k, seed, first_index, ntree):
    r = tm_result()
    g = np.zeros(int(k) * ntree, np.uint32); c = np.zeros(int(k), np.uint64); why = np.zeros(int(k), np.int32)
    _check(lib().tm_sample_trace(ctx, motif, int(k), int(seed), int(first_index), _ptr(g), _ptr(c), _ptr(why),
                                 C.byref(r)), ctx, "tm_sample_trace")
    return Result.of(r), g.reshape(int(k), ntree), c, why


def tm_batch_run(ctx, motifs, ks, seeds):
    nq = len(motifs)
    arr = (C.c_void_p * nq)(*[m.value for m in motifs])
    k = np.ascontiguousarray(np.array(ks, dtype=np.uint64))
    s = np.ascontiguousarray(np.array(seeds, dtype=np.uint64))
    res = (tm_result * nq)()
    _check(lib().tm_batch_run(ctx, nq, arr, _ptr(k), _ptr(s), res), ctx, "tm_batch_run")
    return [Result.of(res[i]) for i in range(nq)]


def tm_motif_free(motif):
    lib().tm_motif_free(motif)


def tm_batch_shape(ctx, tile=0, threads=0, smem_records=0):
    _check(lib().tm_batch_shape(ctx, int(tile), int(threads), int(smem_records)), ctx, "tm_batch_shape")


def tm_coop_search(ctx, min_entries=0):
    """Warp-cooperative searches from min_entries entries on (0 = off)."""
    _check(lib().tm_coop_search(ctx, int(min_entries)), ctx, "tm_coop_search")


def tm_autotune(ctx, motifs, ks, seeds, target_samples=0):
    """Tune the batched sampler for this batch; returns (best, table)."""
    nq = len(motifs)
    arr = (C.c_void_p * nq)(*[m.value for m in motifs])
    k = np.ascontiguousarray(np.array(ks, dtype=np.uint64))
    s = np.ascontiguousarray(np.array(seeds, dtype=np.uint64))
    table = (tm_tune_entry * 64)()
    n = C.c_uint32()
    best = tm_tune_entry()
    _check(lib().tm_autotune(ctx, nq, arr, _ptr(k), _ptr(s), int(target_samples), table, 64, C.byref(n),
                             C.byref(best)), ctx, "tm_autotune")
    return best.as_dict(), [table[i].as_dict() for i in range(min(n.value, 64))]


def tm_serve_start(ctx, max_active=0, tile=0, round_tiles=0, poll_timeout_ms=0, weight_budget=0):
    cfg = tm_serve_cfg(max_active, tile, round_tiles, poll_timeout_ms, weight_budget)
    _check(lib().tm_serve_start(ctx, C.byref(cfg)), ctx, "tm_serve_start")


def tm_serve_submit(ctx, nv, edges, order, delta, k, seed) -> int:
    e = np.ascontiguousarray(np.array(edges, dtype=np.uint32).reshape(-1))
    o = np.ascontiguousarray(np.array(order, dtype=np.uint32))
    t = C.c_uint64()
    _check(lib().tm_serve_submit(ctx, int(nv), len(o), _ptr(e), _ptr(o), int(delta), int(k), int(seed),
                                 C.byref(t)), ctx, "tm_serve_submit")
    return int(t.value)


def tm_serve_submit_motif(ctx, motif, k, seed) -> int:
    """Queue a query on a motif handle's plan (pinned tree, root, constraints)."""
    t = C.c_uint64()
    _check(lib().tm_serve_submit_motif(ctx, motif, int(k), int(seed), C.byref(t)), ctx, "tm_serve_submit_motif")
    return int(t.value)


def tm_serve_poll(ctx, ticket, timeout_ms=0):
    """Result of a finished query, or None while it is still running."""
    r = tm_result()
    rc = lib().tm_serve_poll(ctx, int(ticket), C.byref(r), int(timeout_ms))
    if rc == TM_E_PENDING:
        return None
    _check(rc, ctx, "tm_serve_poll")
    return Result.of(r)


def tm_serve_stats(ctx) -> dict:
    st = tm_serve_stats_t()
    _check(lib().tm_serve_stats(ctx, C.byref(st)), ctx, "tm_serve_stats")
    return st.as_dict()


def tm_serve_stop(ctx):
    _check(lib().tm_serve_stop(ctx), ctx, "tm_serve_stop")


PHASES = ["load", "csr", "windows", "dp", "prefix", "root", "sample", "batch",
          "csr.stats", "csr.global", "csr.out", "csr.in", "csr.multi"]


def tm_phase_times(ctx):
    """{phase: (ms, kernel launches)} accumulated since the last call."""
    ms = np.zeros(16, np.float64); ln = np.zeros(16, np.uint64); n = C.c_int()
    _check(lib().tm_phase_times(ctx, _ptr(ms), _ptr(ln), 16, C.byref(n)), ctx, "tm_phase_times")
    return {PHASES[i] if i < len(PHASES) else str(i): (float(ms[i]), int(ln[i])) for i in range(n.value)}


def tm_kernel_times(ctx):
    """{kernel name: (ms, launches)} since the last call (profile=2 contexts)."""
    n = C.c_uint32()
    _check(lib().tm_kernel_times(ctx, None, 0, C.byref(n)), ctx, "tm_kernel_times")
    cap = max(1, n.value + 8)
    arr = (tm_kernel_time * cap)()
    _check(lib().tm_kernel_times(ctx, arr, cap, C.byref(n)), ctx, "tm_kernel_times")
    return {arr[i].name.decode(): (float(arr[i].ms), int(arr[i].launches)) for i in range(min(n.value, cap))}


def tm_io_bytes(ctx):
    h, d = C.c_uint64(), C.c_uint64()
    _check(lib().tm_io_bytes(ctx, C.byref(h), C.byref(d)), ctx, "tm_io_bytes")
    return int(h.value), int(d.value)


# ---------------------------------------------------------------------------
# Convenience objects over the same calls
# ---------------------------------------------------------------------------
class Motif:
    def __init__(self, ctx: "Context", nv, edges, order, delta, handle=None):
        self.ctx = ctx
        self.nv = int(nv)
        self.ntree = self.nv - 1
        self.edges = list(edges)
        self.order = list(order)
        self.delta = int(delta)
        self.h = handle if handle is not None else tm_set_motif(ctx.h, nv, edges, order, delta)
        ctx._motifs.append(self)

    def set_tree(self, tree, root):
        tm_set_tree(self.ctx.h, self.h, tree, root)
        return self

    def set_constraints(self, c2=True, c3=True):
        """Keep or drop Constraints 2 and 3 (ablation); weights must be recomputed."""
        tm_set_constraints(self.ctx.h, self.h, c2, c3)
        return self

    def plan(self):
        return tm_motif_plan(self.h, self.ntree)

    def weights(self) -> int:
        return tm_weights(self.ctx.h, self.h)

    def export_weights(self, tree_edge, layer):
        return tm_weights_export(self.ctx.h, self.h, tree_edge, layer, self.ctx.m)

    def window_totals(self):
        return tm_window_totals(self.ctx.h, self.h)

    def sample(self, k, seed, first_index=0) -> Result:
        return tm_sample(self.ctx.h, self.h, k, seed, first_index)

    def sample_trace(self, k, seed, first_index=0):
        return tm_sample_trace(self.ctx.h, self.h, k, seed, first_index, self.ntree)

    def sample_list(self, k, seed, first_index=0, max_inst=1_000_000):
        return tm_sample_list(self.ctx.h, self.h, len(self.edges), k, seed, first_index, max_inst)

    def free(self):
        if self.h:
            tm_motif_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    """One device context: a preprocessed temporal graph plus motifs."""

    def __init__(self, device: int = 0, stream=None, torch_allocator: bool = True, **kw):
        self.h, self._keep = tm_create(device, stream, torch_allocator, **kw)
        self.m = 0
        self._motifs = []

    def load_graph(self, n, src, dst, t, flags=TM_HOST, preprocess=True):
        if preprocess:   # one call: device inputs are read in place
            tm_graph_load(self.h, n, src, dst, t, flags | TM_PREPROCESS)
            self.m, self.t_min, self.T = tm_graph_info(self.h)
        else:
            tm_graph_load(self.h, n, src, dst, t, flags)
        return self

    def preprocess(self):
        tm_preprocess(self.h)
        self.m, self.t_min, self.T = tm_graph_info(self.h)

    def edges(self):
        return tm_edges_export(self.h)

    def csr(self, name):
        return tm_csr_export(self.h, name)

    def motif(self, nv, edges, order, delta) -> Motif:
        return Motif(self, nv, edges, order, delta)

    def sample_group(self, motifs, k, seed, first_index=0):
        """Several motifs sharing a spanning-tree pattern, one sampling run
        (weights of motifs[0] are used): a Result per motif."""
        return tm_sample_group(self.h, [m.h for m in motifs], k, seed, first_index)

    def select_tree(self, nv, edges, order, delta, n_c=4, all_roots=True):
        """Tree and root of least exact W among the n_c best looseness trees
        (Alg. 7): the winning Motif, weights computed, and the candidates."""
        h, cands = tm_select_tree(self.h, nv, edges, order, delta, n_c, all_roots)
        return Motif(self, nv, edges, order, delta, handle=h), cands

    # ---- serving (continuous batching); only these calls while serving
    def serve_start(self, **cfg):
        tm_serve_start(self.h, **cfg)

    def submit(self, nv, edges, order, delta, k, seed) -> int:
        return tm_serve_submit(self.h, nv, edges, order, delta, k, seed)

    def submit_motif(self, motif: "Motif", k, seed) -> int:
        """Serve a motif with its pinned tree and constraint settings."""
        return tm_serve_submit_motif(self.h, motif.h, k, seed)

    def poll(self, ticket, timeout_ms=0):
        return tm_serve_poll(self.h, ticket, timeout_ms)

    def serve_stats(self) -> dict:
        return tm_serve_stats(self.h)

    def serve_stop(self):
        tm_serve_stop(self.h)

    def phase_times(self):
        return tm_phase_times(self.h)

    def io_bytes(self):
        return tm_io_bytes(self.h)

    def kernel_times(self):
        return tm_kernel_times(self.h)

    def coop_search(self, min_entries=0):
        tm_coop_search(self.h, min_entries)

    def autotune(self, motifs, ks, seeds, target_samples=0):
        return tm_autotune(self.h, [m.h for m in motifs], ks, seeds, target_samples)

    def batch_run(self, motifs, ks, seeds):
        return tm_batch_run(self.h, [m.h for m in motifs], ks, seeds)

    def close(self):
        if self.h:
            for mo in self._motifs:
                mo.free()
            self._motifs = []
            tm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
