"""TIMEST CPU oracle (arXiv 2507.20441) -- TEST INFRASTRUCTURE ONLY.

A ctypes view of ``timest_oracle.c``: the brute-force enumerator (O1), the
per-window partial-match brute force (O2), the CPU TIMEST with the same
Philox streams (O3) and the exact counter over every partial match (O4).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline /
reference arm may import this package.  The CUDA product path never does.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "timest_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libtimest_oracle.so")

OK, E_ARG, E_DUP, E_SELFLOOP, E_MOTIF, E_NOMEM, E_OVERFLOW, E_STATE, E_LIMIT = range(9)
DEDUP, DROP_SELF = 1, 2
RS_VALID, RS_VERTEX, RS_DELTA, RS_ORDER = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP for the sample loop)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Result(C.Structure):
    _fields_ = [("W_lo", C.c_uint64), ("W_hi", C.c_uint64),
                ("hits2_lo", C.c_uint64), ("hits2_hi", C.c_uint64),
                ("k", C.c_uint64), ("valid", C.c_uint64), ("rej_vertex", C.c_uint64),
                ("rej_delta", C.c_uint64), ("rej_order", C.c_uint64), ("estimate", C.c_double)]


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


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = os.environ.get("TIMEST_ORACLE_LIB") or build()
        L = C.CDLL(path)
        vp, i64, u64, i32 = C.c_void_p, C.c_int64, C.c_uint64, C.c_int
        L.or_create.argtypes = [i64, i64, vp, vp, vp, i32, C.POINTER(vp)]
        L.or_free.argtypes = [vp]
        L.or_num_edges.argtypes = [vp]; L.or_num_edges.restype = i64
        L.or_time_min.argtypes = [vp]; L.or_time_min.restype = i64
        L.or_time_span.argtypes = [vp]; L.or_time_span.restype = i64
        L.or_export_edges.argtypes = [vp, vp, vp, vp]
        L.or_set_motif.argtypes = [vp, i32, i32, vp, vp, vp, i64, vp, i32]
        L.or_set_constraints.argtypes = [vp, i32, i32]
        L.or_plan_info.argtypes = [vp, vp, vp, vp, vp]
        L.or_weights.argtypes = [vp, C.POINTER(u64), C.POINTER(u64)]
        L.or_export_weights.argtypes = [vp, i32, i32, vp]
        L.or_num_windows.argtypes = [vp]; L.or_num_windows.restype = i64
        L.or_window_totals.argtypes = [vp, vp]
        L.or_sample.argtypes = [vp, u64, u64, u64, i32, C.POINTER(_Result), vp, vp, vp]
        L.or_partial_count.argtypes = [vp, i64, C.POINTER(u64), vp, i64, C.POINTER(i64)]
        L.or_exact_by_trees.argtypes = [vp, C.POINTER(u64), C.POINTER(u64)]
        L.or_brute_count.argtypes = [vp, i32, i32, vp, vp, vp, i64, C.POINTER(u64)]
        L.or_philox4x32_10.argtypes = [vp, vp, vp]
        L.or_uniform_u64.argtypes = [u64, u64, C.c_uint32, u64, C.POINTER(C.c_uint32)]
        L.or_uniform_u64.restype = u64
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def uniform_u64(seed: int, j: int, d0: int, n: int):
    d = C.c_uint32(0)
    x = lib().or_uniform_u64(seed, j, d0, n, C.byref(d))
    return int(x), int(d.value)


class Graph:
    """The oracle's copy of a temporal graph plus (optionally) one motif plan."""

    def __init__(self, n, src, dst, t, flags: int = 0):
        L = lib()
        self.src_in = np.ascontiguousarray(src, dtype=np.uint32)
        self.dst_in = np.ascontiguousarray(dst, dtype=np.uint32)
        self.t_in = np.ascontiguousarray(t, dtype=np.int64)
        h = C.c_void_p()
        rc = L.or_create(int(n), len(self.src_in), _p(self.src_in), _p(self.dst_in), _p(self.t_in), flags, C.byref(h))
        if rc != OK:
            raise OracleError(rc, "or_create")
        self.h = h
        self.n = int(n)
        self.m = int(L.or_num_edges(h))
        self.ntree = 0

    def close(self):
        if getattr(self, "h", None):
            lib().or_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def t_min(self) -> int:
        return int(lib().or_time_min(self.h))

    @property
    def span(self) -> int:
        return int(lib().or_time_span(self.h))

    def edges(self):
        """GLOBAL order (t', src, dst): arrays indexed by gid."""
        s = np.zeros(self.m, np.uint32); d = np.zeros(self.m, np.uint32); t = np.zeros(self.m, np.int64)
        lib().or_export_edges(self.h, _p(s), _p(d), _p(t))
        return s, d, t

    def csr(self):
        """The temporal CSR of this graph (see csr_arrays)."""
        s, d, t = self.edges()
        return csr_arrays(self.n, s, d, t)

    def set_motif(self, nv, edges, rank, delta, tree, root):
        ea = np.array([e[0] for e in edges], np.int32)
        eb = np.array([e[1] for e in edges], np.int32)
        rk = np.array(rank, np.int32)
        tr = np.array(tree, np.int32)
        rc = lib().or_set_motif(self.h, nv, len(edges), _p(ea), _p(eb), _p(rk), int(delta), _p(tr), int(root))
        if rc != OK:
            raise OracleError(rc, "or_set_motif")
        self.ntree = nv - 1
        self.ne = len(edges)
        return rc

    def set_constraints(self, c2=True, c3=True):
        """Constraint toggles of the ablation (R8); weights must be recomputed."""
        rc = lib().or_set_constraints(self.h, 1 if c2 else 0, 1 if c3 else 0)
        if rc != OK:
            raise OracleError(rc, "or_set_constraints")
        return rc

    def plan_info(self):
        order = np.zeros(self.ntree, np.int32)
        parent = np.zeros(self.ne, np.int32); meet = np.zeros(self.ne, np.int32); height = np.zeros(self.ne, np.int32)
        lib().or_plan_info(self.h, _p(order), _p(parent), _p(meet), _p(height))
        return order, parent, meet, height

    def weights(self, allow_overflow: bool = False):
        lo, hi = C.c_uint64(), C.c_uint64()
        rc = lib().or_weights(self.h, C.byref(lo), C.byref(hi))
        if rc == E_OVERFLOW and allow_overflow:
            return None
        if rc != OK:
            raise OracleError(rc, "or_weights")
        return int(lo.value) | (int(hi.value) << 64)

    def export_weights(self, s: int, layer: int) -> np.ndarray:
        out = np.zeros(self.m, np.uint64)
        rc = lib().or_export_weights(self.h, s, layer, _p(out))
        if rc != OK:
            raise OracleError(rc, "or_export_weights")
        return out

    def window_totals(self) -> np.ndarray:
        nw = int(lib().or_num_windows(self.h))
        out = np.zeros(nw, np.uint64)
        rc = lib().or_window_totals(self.h, _p(out))
        if rc != OK:
            raise OracleError(rc, "or_window_totals")
        return out

    def sample(self, k: int, seed: int, first: int = 0, threads: int = 0, trace: bool = False):
        r = _Result()
        tg = tc = tr = None
        if trace:
            tg = np.zeros(k * self.ntree, np.uint32); tc = np.zeros(k, np.uint64); tr = np.zeros(k, np.int32)
        rc = lib().or_sample(self.h, k, seed, first, threads, C.byref(r),
                             _p(tg) if trace else None, _p(tc) if trace else None, _p(tr) if trace else None)
        if rc != OK:
            raise OracleError(rc, "or_sample")
        res = Result(W=r.W_lo | (r.W_hi << 64), hits2=r.hits2_lo | (r.hits2_hi << 64), k=r.k,
                     valid=r.valid, rej_vertex=r.rej_vertex, rej_delta=r.rej_delta,
                     rej_order=r.rej_order, estimate=r.estimate)
        if trace:
            return res, tg.reshape(k, self.ntree), tc, tr
        return res

    def partial_count(self, window: int, want_list: bool = False, cap: int = 0):
        cnt = C.c_uint64(); ln = C.c_int64()
        buf = np.zeros(max(cap, 1) * max(self.ntree, 1), np.uint32) if want_list else None
        rc = lib().or_partial_count(self.h, window, C.byref(cnt), _p(buf) if want_list else None,
                                    cap if want_list else 0, C.byref(ln))
        if rc != OK:
            raise OracleError(rc, "or_partial_count")
        if want_list:
            n = min(int(ln.value), cap)
            return int(cnt.value), buf[: n * self.ntree].reshape(n, self.ntree)
        return int(cnt.value)

    def exact_by_trees(self) -> int:
        """O4: returns 2C (the sum of 2*cnt/N_phi over windows and partial matches)."""
        lo, hi = C.c_uint64(), C.c_uint64()
        rc = lib().or_exact_by_trees(self.h, C.byref(lo), C.byref(hi))
        if rc != OK:
            raise OracleError(rc, "or_exact_by_trees")
        return int(lo.value) | (int(hi.value) << 64)

    def brute_count(self, nv, edges, rank, delta) -> int:
        ea = np.array([e[0] for e in edges], np.int32)
        eb = np.array([e[1] for e in edges], np.int32)
        rk = np.array(rank, np.int32)
        out = C.c_uint64()
        rc = lib().or_brute_count(self.h, nv, len(edges), _p(ea), _p(eb), _p(rk), int(delta), C.byref(out))
        if rc != OK:
            raise OracleError(rc, "or_brute_count")
        return int(out.value)


def csr_arrays(n: int, src, dst, t) -> dict:
    """The temporal CSR (Sec. 3 preamble, Defs. 3.1-3.3) of a graph given in
    GLOBAL order (edges sorted by (t', src, dst); gid = position), written out
    with stable sorts and searches:

    * OUT order (src, t', dst): the GLOBAL order stably sorted by src; IN order
      (dst, t', src): stably sorted by dst; MULTI order (src, dst, t').
    * *_off: list starts per vertex; *_pos: position of each gid in a list
      order; in_to_out / multi_to_out: the OUT position of the same edge.
    * out_xrank[x]: the first IN position of x's source whose time is >= x's
      time (the end of that in-list if none); in_xrank the same with OUT and
      IN swapped.
    * pair_off / pair_dst: runs of equal (src, dst) in MULTI order;
      vpair_off: first pair of each source.
    * own_*: bit x of word x // 32 set when position x starts a new owner.

    Names and layouts follow tm_csr_export."""
    src = np.asarray(src, np.uint64); dst = np.asarray(dst, np.uint64); t = np.asarray(t, np.uint64)
    m = src.shape[0]
    ar = np.arange(m, dtype=np.uint64)
    out_gid = np.argsort(src, kind="stable")
    in_gid = np.argsort(dst, kind="stable")
    multi = np.lexsort((t, dst, src))
    out_pos = np.empty(m, np.uint64); out_pos[out_gid] = ar
    in_pos = np.empty(m, np.uint64); in_pos[in_gid] = ar

    def offsets(keys):
        return np.concatenate([[0], np.cumsum(np.bincount(keys.astype(np.int64), minlength=n))]).astype(np.uint64)

    out_key = (src[out_gid] << np.uint64(32)) | t[out_gid]
    in_key = (dst[in_gid] << np.uint64(32)) | t[in_gid]
    ms, md = src[multi], dst[multi]
    head = np.ones(m, bool)
    if m:
        head[1:] = (ms[1:] != ms[:-1]) | (md[1:] != md[:-1])
    heads = np.flatnonzero(head)

    def bits(starts):
        words = np.zeros(m // 32 + 1, np.uint64)
        x = np.flatnonzero(starts).astype(np.uint64)
        np.bitwise_or.at(words, (x >> np.uint64(5)).astype(np.int64), np.uint64(1) << (x & np.uint64(31)))
        return words

    def starts(owner):
        b = np.ones(m, bool)
        if m:
            b[1:] = owner[1:] != owner[:-1]
        return b

    r = {
        "out_off": offsets(src), "out_t": t[out_gid], "out_nbr": dst[out_gid], "out_gid": out_gid.astype(np.uint64),
        "out_src": src[out_gid], "out_pos": out_pos,
        "out_xrank": np.searchsorted(in_key, out_key, side="left").astype(np.uint64),
        "in_off": offsets(dst), "in_t": t[in_gid], "in_nbr": src[in_gid], "in_gid": in_gid.astype(np.uint64),
        "in_dst": dst[in_gid], "in_pos": in_pos,
        "in_xrank": np.searchsorted(out_key, in_key, side="left").astype(np.uint64),
        "in_to_out": out_pos[in_gid],
        "vpair_off": offsets(ms[heads]), "pair_off": np.concatenate([heads, [m]]).astype(np.uint64),
        "pair_dst": md[heads], "multi_t": t[multi], "multi_to_out": out_pos[multi],
        "own_out": bits(starts(src[out_gid])), "own_in": bits(starts(dst[in_gid])), "own_multi": bits(head),
    }
    return {k: v.astype(np.uint32) for k, v in r.items()}
