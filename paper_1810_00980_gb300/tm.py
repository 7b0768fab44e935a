"""Python binding of libtmotif (C ABI in include/tm.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  There is no CPU fallback -- if libtmotif.so has not been built
(``python -c "import __graft_entry__ as g; g.build()"``) every call raises.

Arrays may be numpy arrays / CPU tensors (host) or CUDA torch tensors
(device).  Names follow the C ABI without the ``tm_`` prefix.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# TMOTIF_CHECKED=1 selects the bounds-checked build (libtmotif_checked.so; see tm_check_status)
LIB_PATH = os.path.join(HERE, "_build", "libtmotif_checked.so" if os.environ.get("TMOTIF_CHECKED") == "1"
                        else "libtmotif.so")

TM_OK, TM_EINVAL, TM_EUNSORTED, TM_ERANGE, TM_ENOMEM, TM_EADMIT, TM_ETIMEOUT = range(7)
TM_ESTACK, TM_EOVERFLOW, TM_ECUDA, TM_PENDING, TM_ENOTFOUND, TM_ECANCELLED, TM_ESHUTDOWN = range(7, 14)
TM_MODE_EXACT, TM_MODE_ESTIMATE = 0, 1
TM_Q_UNIFORM, TM_Q_EDGES, TM_Q_AUTO = 0, 1, 2
TM_AUTO_PILOT_P = 0.05
TM_AUTO_PILOT_SEED_XOR = 0xA5A5A5A5A5A5A5A5
L_MAX = 8
K_MAX = 8

_c_i32, _c_i64, _c_u64, _c_dbl, _vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p


class GraphInfo(ctypes.Structure):
    _fields_ = [("m", _c_i64), ("n_nodes", _c_i32), ("pad0", _c_i32), ("n_pairs", _c_i64),
                ("t_min", _c_i64), ("t_max", _c_i64), ("device_bytes", _c_i64)]


class WindowRec(ctypes.Structure):
    _fields_ = [("k", _c_i32), ("kept", _c_i32), ("j", _c_i64), ("start", _c_i64), ("lo", _c_i64),
                ("hi", _c_i64), ("count", _c_i64), ("w_int", _c_u64), ("w_frac", _c_u64), ("q", _c_dbl)]


class QueryC(ctypes.Structure):
    _fields_ = [("motif", _vp), ("delta", _c_i64), ("mode", _c_i32), ("c", _c_i32), ("p", _c_dbl),
                ("seed", _c_u64), ("b", _c_i32), ("q_mode", _c_i32)]


class ResultC(ctypes.Structure):
    _fields_ = [("status", _c_i32), ("pad0", _c_i32), ("count", _c_i64), ("estimate", _c_dbl),
                ("windows", _c_i64), ("windows_kept", _c_i64), ("first_edges", _c_i64),
                ("cand_edges", _c_i64), ("last_ranges", _c_i64), ("inst_read", _c_i64),
                ("var_hat", _c_dbl), ("shift_var", _c_dbl), ("p_used", _c_dbl)]


class TuningC(ctypes.Structure):
    _fields_ = [("block_threads", _c_i32), ("blocks_per_sm", _c_i32), ("chunk_items", _c_i32),
                ("enum_threshold", _c_i32)]


class ServeCfg(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", _c_i64), ("max_batch", _c_i32), ("n_streams", _c_i32)]


class ProfileC(ctypes.Structure):
    _fields_ = [("graph_ms", _c_dbl), ("windows_ms", _c_dbl), ("level2_ms", _c_dbl), ("match_ms", _c_dbl),
                ("fold_ms", _c_dbl), ("batch_ms", _c_dbl), ("match_items", _c_i64), ("first_edges", _c_i64),
                ("launches", _c_i64), ("sizing_ms", _c_dbl), ("scan_ms", _c_dbl),
                ("ride_ms", _c_dbl), ("ride_records", _c_i64)]


class TmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        lib = _LIB
        detail = lib.tm_last_error().decode() if lib is not None else ""
        name = lib.tm_strerror(status).decode() if lib is not None else str(status)
        super().__init__(f"{where}: {name} ({status}) {detail}")


_LIB = None

_SIGS = {
    "tm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "tm_last_error": (ctypes.c_char_p, []),
    "tm_version": (ctypes.c_char_p, []),
    "tm_graph_load": (ctypes.c_int, [_vp, _vp, _vp, _c_i64, _c_i32, _vp]),
    "tm_graph_load_device": (ctypes.c_int, [_vp, _vp, _vp, _c_i64, _c_i32, _vp, _vp]),
    "tm_graph_free": (None, [_vp]),
    "tm_graph_get_info": (ctypes.c_int, [_vp, _vp]),
    "tm_motif_compile": (ctypes.c_int, [_vp, _vp, _c_i32, _vp]),
    "tm_motif_free": (None, [_vp]),
    "tm_count_exact": (ctypes.c_int, [_vp, _vp, _c_i64, _vp]),
    "tm_count_exact_plain": (ctypes.c_int, [_vp, _vp, _c_i64, _vp]),
    "tm_count_exact_noalloc": (ctypes.c_int, [_vp, _vp, _c_i64, _vp, _vp]),
    "tm_estimate": (ctypes.c_int, [_vp, _vp, _c_i64, _c_i32, _c_dbl, _c_u64, _vp]),
    "tm_estimate_windows": (ctypes.c_int, [_vp, _vp, _c_i64, _c_i32, _c_dbl, _c_u64, _c_i32, _c_i32,
                                           _vp, _c_i64, _vp, _vp]),
    "tm_run_batch": (ctypes.c_int, [_vp, _vp, _c_i32, _vp, _vp]),
    "tm_stream_run": (ctypes.c_int, [_vp, _vp, _vp, _c_i64, _c_i32, _vp, _c_i32, _c_i64, _vp, _vp]),
    "tm_batch_create": (ctypes.c_int, [_vp, _vp, _c_i32, _vp]),
    "tm_batch_launch": (ctypes.c_int, [_vp, _vp]),
    "tm_batch_results": (ctypes.c_int, [_vp, _vp, _vp]),
    "tm_batch_free": (None, [_vp]),
    "tm_get_tuning": (ctypes.c_int, [_vp]),
    "tm_set_tuning": (ctypes.c_int, [_vp]),
    "tm_set_ride_capacity": (ctypes.c_int, [_c_i64]),
    "tm_autotune": (ctypes.c_int, [_vp, _vp, _c_i32, _vp]),
    "tm_profile_enable": (ctypes.c_int, [_c_i32]),
    "tm_profile_last": (ctypes.c_int, [_vp]),
    "tm_release_cached_memory": (ctypes.c_int, []),
    "tm_check_status": (ctypes.c_int, [_vp, _c_i32]),
    "tm_check_selftest": (ctypes.c_int, []),
    "tm_serve_create": (ctypes.c_int, [_vp, _vp]),
    "tm_serve_attach_graph": (ctypes.c_int, [_vp, _vp, _vp]),
    "tm_serve_submit": (ctypes.c_int, [_vp, _c_i32, _vp, _vp]),
    "tm_serve_poll": (ctypes.c_int, [_vp, _c_u64, _vp]),
    "tm_serve_wait": (ctypes.c_int, [_vp, _c_u64, _c_i64, _vp]),
    "tm_serve_wait_any": (ctypes.c_int, [_vp, _c_i64, _vp, _vp]),
    "tm_serve_cancel": (ctypes.c_int, [_vp, _c_u64]),
    "tm_serve_destroy": (None, [_vp]),
}


def lib():
    """Load libtmotif.so (raises if it was not built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libtmotif.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def check_status(clear: bool = True) -> int:
    """tm_check_status: the bits of the failed bounds checks since the last clear (checked
    build only; the ordinary build raises TmError(TM_EINVAL))."""
    w = ctypes.c_uint32(0)
    _check(lib().tm_check_status(ctypes.byref(w), 1 if clear else 0), "tm_check_status")
    return w.value


def check_selftest():
    """tm_check_selftest: one deliberately out-of-range index through the checks."""
    _check(lib().tm_check_selftest(), "tm_check_selftest")


def _check(status: int, where: str):
    if status != TM_OK:
        raise TmError(status, where)


def _is_cuda_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and bool(getattr(x, "is_cuda"))


def _host(x, dtype):
    if hasattr(x, "numpy") and not _is_cuda_tensor(x):
        x = x.numpy()
    return np.ascontiguousarray(x, dtype=dtype)


def _ptr(a) -> int:
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def current_stream_handle() -> int:
    import torch
    return torch.cuda.current_stream().cuda_stream


class Graph:
    """A resident temporal graph (tm_graph)."""

    def __init__(self, src, dst, t, n_nodes: int = -1, stream=None):
        L = lib()
        h = _vp()
        if _is_cuda_tensor(src):
            import torch
            assert src.dtype == torch.int32 and dst.dtype == torch.int32 and t.dtype == torch.int64
            assert src.is_contiguous() and dst.is_contiguous() and t.is_contiguous()
            st = current_stream_handle() if stream is None else int(stream)
            s = L.tm_graph_load_device(_ptr(src), _ptr(dst), _ptr(t), int(t.numel()), int(n_nodes),
                                       st, ctypes.byref(h))
        elif hasattr(src, "data_ptr") and hasattr(src, "is_pinned") and src.is_pinned():
            s = L.tm_graph_load(_ptr(src), _ptr(dst), _ptr(t), int(t.numel()), int(n_nodes), ctypes.byref(h))
        else:
            self._keep = (_host(src, np.int32), _host(dst, np.int32), _host(t, np.int64))
            a, b, c = self._keep
            s = L.tm_graph_load(_ptr(a), _ptr(b), _ptr(c), len(c), int(n_nodes), ctypes.byref(h))
            self._keep = None
        _check(s, "tm_graph_load")
        self.handle = h.value

    def info(self) -> GraphInfo:
        gi = GraphInfo()
        _check(lib().tm_graph_get_info(self.handle, ctypes.byref(gi)), "tm_graph_get_info")
        return gi

    def free(self):
        if getattr(self, "handle", None):
            lib().tm_graph_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.free()


class Motif:
    """An ordered motif edge list (tm_motif)."""

    def __init__(self, msrc, mdst):
        a = np.ascontiguousarray(msrc, np.int32)
        b = np.ascontiguousarray(mdst, np.int32)
        if len(a) != len(b):
            raise ValueError("msrc and mdst differ in length")
        h = _vp()
        _check(lib().tm_motif_compile(_ptr(a), _ptr(b), len(a), ctypes.byref(h)), "tm_motif_compile")
        self.handle = h.value
        self.l = len(a)

    def free(self):
        if getattr(self, "handle", None):
            lib().tm_motif_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def count_exact(g: Graph, m: Motif, delta: int) -> int:
    out = _c_i64()
    _check(lib().tm_count_exact(g.handle, m.handle, int(delta), ctypes.byref(out)), "tm_count_exact")
    return out.value


def count_exact_plain(g: Graph, m: Motif, delta: int) -> int:
    out = _c_i64()
    _check(lib().tm_count_exact_plain(g.handle, m.handle, int(delta), ctypes.byref(out)),
           "tm_count_exact_plain")
    return out.value


NOALLOC_MAX_EDGES = 262144


def count_exact_noalloc(g: Graph, m: Motif, delta: int, stream=None) -> int:
    """tm_count_exact_noalloc: the exact count with no device allocation (static
    scratch inside the library; graphs of at most NOALLOC_MAX_EDGES edges)."""
    out = _c_i64()
    st = 0 if stream is None else int(stream)
    _check(lib().tm_count_exact_noalloc(g.handle, m.handle, int(delta), st, ctypes.byref(out)),
           "tm_count_exact_noalloc")
    return out.value


def estimate(g: Graph, m: Motif, delta: int, c: int, p: float, seed: int) -> float:
    out = _c_dbl()
    _check(lib().tm_estimate(g.handle, m.handle, int(delta), int(c), float(p), int(seed) & (2**64 - 1),
                             ctypes.byref(out)), "tm_estimate")
    return out.value


def estimate_windows(g: Graph, m: Motif, delta: int, c: int, p: float, seed: int, k: int = 0,
                     all_windows: bool = False):
    """(shift, [window dicts]) for repetition k: the kept windows (or all)."""
    L = lib()
    n = _c_i64()
    s = _c_i64()
    _check(L.tm_estimate_windows(g.handle, m.handle, int(delta), int(c), float(p), int(seed) & (2**64 - 1),
                                 int(k), int(all_windows), None, 0, ctypes.byref(n), ctypes.byref(s)),
           "tm_estimate_windows")
    cap = n.value
    recs = (WindowRec * max(cap, 1))()
    _check(L.tm_estimate_windows(g.handle, m.handle, int(delta), int(c), float(p), int(seed) & (2**64 - 1),
                                 int(k), int(all_windows), ctypes.cast(recs, _vp), cap, ctypes.byref(n),
                                 ctypes.byref(s)), "tm_estimate_windows")
    out = []
    for i in range(min(cap, n.value)):
        r = recs[i]
        out.append(dict(k=r.k, kept=bool(r.kept), j=r.j, start=r.start, lo=r.lo, hi=r.hi, count=r.count,
                        w_int=r.w_int, w_frac=r.w_frac, q=r.q))
    return s.value, out


@dataclass
class Query:
    motif: Motif
    delta: int
    mode: int = TM_MODE_EXACT
    c: int = 1
    p: float = 1.0
    seed: int = 0
    b: int = 1
    q_mode: int = TM_Q_UNIFORM

    def to_c(self) -> QueryC:
        return QueryC(self.motif.handle, int(self.delta), int(self.mode), int(self.c), float(self.p),
                      int(self.seed) & (2**64 - 1), int(self.b), int(self.q_mode))


def exact_query(motif: Motif, delta: int) -> Query:
    return Query(motif, delta, TM_MODE_EXACT)


def estimate_query(motif: Motif, delta: int, c: int, p: float, seed: int, b: int = 1,
                   q_mode: int = TM_Q_UNIFORM) -> Query:
    return Query(motif, delta, TM_MODE_ESTIMATE, c, p, seed, b, q_mode)


def _result_dict(r: ResultC) -> dict:
    return {f: getattr(r, f) for f, _ in ResultC._fields_ if f != "pad0"}


class Batch:
    """Queries marshalled once into C structs, for repeated tm_run_batch calls."""

    def __init__(self, g: Graph, queries):
        self.g = g
        self.queries = list(queries)
        self.n = len(self.queries)
        self.qarr = (QueryC * max(self.n, 1))(*[q.to_c() for q in self.queries])
        self.rarr = (ResultC * max(self.n, 1))()

    def run(self, stream=None, check: bool = True):
        st = 0 if stream is None else int(stream)
        s = lib().tm_run_batch(self.g.handle, ctypes.cast(self.qarr, _vp), self.n,
                               ctypes.cast(self.rarr, _vp), st)
        if check:
            _check(s, "tm_run_batch")
        return s

    def results(self):
        return [_result_dict(self.rarr[i]) for i in range(self.n)]


class StreamStatsC(ctypes.Structure):
    _fields_ = [("segments", _c_i64), ("edges_copied", _c_i64), ("max_segment_edges", _c_i64),
                ("wall_ms", _c_dbl), ("copy_wait_ms", _c_dbl)]


def stream_run(src, dst, t, queries, segment_edges: int, n_nodes: int, check: bool = True):
    """tm_stream_run: the queries over a time-sorted edge list in host memory (numpy
    arrays or CPU tensors, pinned tensors copied directly), in chronological segments
    of about `segment_edges` edges.  Returns (results, stats)."""
    if hasattr(src, "data_ptr") and hasattr(src, "is_pinned") and src.is_pinned():
        keep = (src, dst, t)
    else:
        keep = (_host(src, np.int32), _host(dst, np.int32), _host(t, np.int64))
    a, b, c = keep
    m = int(c.numel()) if hasattr(c, "numel") else len(c)
    qs = list(queries)
    qarr = (QueryC * max(len(qs), 1))(*[q.to_c() for q in qs])
    rarr = (ResultC * max(len(qs), 1))()
    st = StreamStatsC()
    s = lib().tm_stream_run(_ptr(a), _ptr(b), _ptr(c), m, int(n_nodes), ctypes.cast(qarr, _vp), len(qs),
                            int(segment_edges), ctypes.cast(rarr, _vp), ctypes.byref(st))
    if check:
        _check(s, "tm_stream_run")
    return [_result_dict(rarr[i]) for i in range(len(qs))], {f: getattr(st, f) for f, _ in StreamStatsC._fields_}


class PreparedBatch:
    """tm_batch_*: queries prepared once and replayed as one CUDA graph."""

    def __init__(self, g: Graph, queries):
        self.g = g
        self.queries = list(queries)
        self.n = len(self.queries)
        self.qarr = (QueryC * max(self.n, 1))(*[q.to_c() for q in self.queries])
        self.rarr = (ResultC * max(self.n, 1))()
        h = _vp()
        _check(lib().tm_batch_create(g.handle, ctypes.cast(self.qarr, _vp), self.n, ctypes.byref(h)),
               "tm_batch_create")
        self.handle = h.value

    def launch(self, stream=None):
        _check(lib().tm_batch_launch(self.handle, 0 if stream is None else int(stream)), "tm_batch_launch")

    def results(self, stream=None, check: bool = True):
        s = lib().tm_batch_results(self.handle, 0 if stream is None else int(stream), ctypes.cast(self.rarr, _vp))
        if check:
            _check(s, "tm_batch_results")
        return [_result_dict(self.rarr[i]) for i in range(self.n)]

    def free(self):
        if getattr(self, "handle", None):
            lib().tm_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def run_batch(g: Graph, queries, stream=None, check: bool = True):
    b = Batch(g, queries)
    b.run(stream, check)
    return b.results()


def get_tuning() -> dict:
    t = TuningC()
    _check(lib().tm_get_tuning(ctypes.byref(t)), "tm_get_tuning")
    return {f: getattr(t, f) for f, _ in TuningC._fields_}


def set_tuning(**kw):
    t = TuningC(**{k: int(v) for k, v in kw.items()})
    _check(lib().tm_set_tuning(ctypes.byref(t)), "tm_set_tuning")


def set_ride_capacity(records: int):
    _check(lib().tm_set_ride_capacity(int(records)), "tm_set_ride_capacity")


def autotune(g: Graph, queries) -> dict:
    b = Batch(g, queries)
    t = TuningC()
    _check(lib().tm_autotune(g.handle, ctypes.cast(b.qarr, _vp), b.n, ctypes.byref(t)), "tm_autotune")
    return {f: getattr(t, f) for f, _ in TuningC._fields_}


def profile_enable(on: bool = True):
    _check(lib().tm_profile_enable(int(bool(on))), "tm_profile_enable")


def profile_last() -> dict:
    p = ProfileC()
    _check(lib().tm_profile_last(ctypes.byref(p)), "tm_profile_last")
    return {f: getattr(p, f) for f, _ in ProfileC._fields_}


def release_cached_memory():
    _check(lib().tm_release_cached_memory(), "tm_release_cached_memory")


class Server:
    """Continuous-batching server (tm_serve_*)."""

    def __init__(self, mem_budget_bytes: int = 0, max_batch: int = 0, n_streams: int = 0):
        cfg = ServeCfg(int(mem_budget_bytes), int(max_batch), int(n_streams))
        h = _vp()
        _check(lib().tm_serve_create(ctypes.byref(cfg), ctypes.byref(h)), "tm_serve_create")
        self.handle = h.value
        self._graphs = []
        self._pending = {}

    def attach(self, g: Graph) -> int:
        gid = _c_i32()
        _check(lib().tm_serve_attach_graph(self.handle, g.handle, ctypes.byref(gid)), "tm_serve_attach_graph")
        self._graphs.append(g)
        return gid.value

    def submit(self, graph_id: int, q: Query) -> int:
        t = _c_u64()
        qc = q.to_c()
        _check(lib().tm_serve_submit(self.handle, int(graph_id), ctypes.byref(qc), ctypes.byref(t)),
               "tm_serve_submit")
        self._pending[t.value] = q   # keep the motif alive
        return t.value

    def poll(self, ticket: int):
        """None while pending, else (status, result dict)."""
        r = ResultC()
        s = lib().tm_serve_poll(self.handle, int(ticket), ctypes.byref(r))
        if s == TM_PENDING:
            return None
        self._pending.pop(ticket, None)
        return s, _result_dict(r)

    def wait(self, ticket: int, timeout_ms: int = 60_000):
        r = ResultC()
        s = lib().tm_serve_wait(self.handle, int(ticket), int(timeout_ms), ctypes.byref(r))
        if s == TM_ETIMEOUT:
            return None
        self._pending.pop(ticket, None)
        return s, _result_dict(r)

    def wait_any(self, timeout_ms: int = 60_000):
        """Next finished ticket in completion order: (ticket, status, result), or None on timeout."""
        r = ResultC()
        t = _c_u64()
        s = lib().tm_serve_wait_any(self.handle, int(timeout_ms), ctypes.byref(t), ctypes.byref(r))
        if s == TM_ETIMEOUT:
            return None
        self._pending.pop(t.value, None)
        return t.value, s, _result_dict(r)

    def cancel(self, ticket: int) -> int:
        return lib().tm_serve_cancel(self.handle, int(ticket))

    def close(self):
        if getattr(self, "handle", None):
            lib().tm_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
