"""ctypes binding of librpq.so (include/rpq.h).

Argument marshalling only: every step of a query runs in the library's CUDA
kernels.  The functions keep the C names (``rpq_graph_load``,
``rpq_nfa_compile``, ``rpq_query``, ...) and take numpy arrays, torch tensors
or raw pointers; results come back as numpy arrays (host outputs) or are
written into the torch tensors passed in (device outputs).

If librpq.so is missing the first call raises: there is no other execution
path.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librpq.so")

RPQ_OK, RPQ_ERR_INVALID, RPQ_ERR_PARSE, RPQ_ERR_OOM = 0, 1, 2, 3
RPQ_ERR_CUDA, RPQ_ERR_TIMEOUT, RPQ_ERR_CAPACITY, RPQ_ERR_BUSY = 4, 5, 6, 7
STATUS_NAMES = {0: "RPQ_OK", 1: "RPQ_ERR_INVALID", 2: "RPQ_ERR_PARSE", 3: "RPQ_ERR_OOM",
                4: "RPQ_ERR_CUDA", 5: "RPQ_ERR_TIMEOUT", 6: "RPQ_ERR_CAPACITY", 7: "RPQ_ERR_BUSY"}

# Every symbol include/rpq.h declares.
EXPORTED = (
    "rpq_set_allocator", "rpq_graph_load", "rpq_graph_free", "rpq_graph_info", "rpq_graph_export",
    "rpq_graph_autotune", "rpq_graph_autotune_batch", "rpq_graph_set_hybrid",
    "rpq_graph_set_rare_plan",
    "rpq_nfa_compile", "rpq_nfa_from_transitions", "rpq_nfa_free", "rpq_nfa_info",
    "rpq_nfa_export", "rpq_nfa_accepts", "rpq_nfa_reverse", "rpq_query", "rpq_last_answer",
    "rpq_query_noalloc",
    "rpq_query_bitset", "rpq_query_multi", "rpq_query_sdr", "rpq_query_levels",
    "rpq_query_witness",
    "rpq_query_batch", "rpq_serve_create", "rpq_serve_submit", "rpq_serve_poll",
    "rpq_serve_drain", "rpq_serve_stats", "rpq_serve_stats_get", "rpq_serve_destroy",
    "rpq_last_error",
    "rpq_version", "rpq_kernel_launches",
)


class RpqError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class RpqStats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int64), ("visited_pairs", ctypes.c_int64),
                ("expanded_pairs", ctypes.c_int64), ("product_edges", ctypes.c_int64),
                ("push_bytes", ctypes.c_int64), ("answer_count", ctypes.c_int64),
                ("push_unit_levels", ctypes.c_int64), ("pull_unit_levels", ctypes.c_int64),
                ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64),
                ("device_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RpqServeConfig(ctypes.Structure):
    _fields_ = [("max_lanes", ctypes.c_int32), ("max_states", ctypes.c_int32),
                ("queue_capacity", ctypes.c_int32), ("memory_budget", ctypes.c_int64),
                ("max_levels", ctypes.c_int32), ("engine", ctypes.c_int32)]


class RpqServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("level_steps", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("elapsed_s", ctypes.c_double), ("qps", ctypes.c_double),
                ("peak_in_flight", ctypes.c_int64), ("peak_bytes", ctypes.c_int64),
                ("oom_retries", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None


def lib():
    """The loaded librpq.so; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2412_10287_gb300.build` "
                "(there is no fallback path)")
        L = ctypes.CDLL(LIB_PATH)
        i32, i64, u64, p, st = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                ctypes.c_void_p, ctypes.c_int)
        pp = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "rpq_set_allocator": [p, p, p],
            "rpq_graph_load": [i32, i32, i64, p, p, p, p, pp],
            "rpq_graph_info": [p, i32, p, p, p],
            "rpq_graph_export": [p, i32, i32, p, p, i64],
            "rpq_graph_autotune": [p, i32, p, p, p, p, p, p],
            "rpq_graph_set_hybrid": [p, i64],
            "rpq_graph_autotune_batch": [p, i32, p, p, p, p, p],
            "rpq_graph_set_rare_plan": [p, i64],
            "rpq_nfa_compile": [ctypes.c_char_p, i32, pp],
            "rpq_nfa_from_transitions": [i32, i32, i32, p, p, p, i32, p, i32, p, pp],
            "rpq_nfa_info": [p, p, p, p],
            "rpq_nfa_export": [p, p, p, p, i32, p, p],
            "rpq_nfa_accepts": [p, p, i32, p],
            "rpq_nfa_reverse": [p, pp],
            "rpq_query": [p, p, i32, i32, p, i64, p, p, p],
            "rpq_last_answer": [p, p],
            "rpq_query_noalloc": [p, p, i32, i32, p, i64, p, p],
            "rpq_query_bitset": [p, p, i32, i32, p, p, p, p],
            "rpq_query_multi": [p, p, i32, p, i32, p, i64, p, p, p],
            "rpq_query_sdr": [p, p, i32, i32, p, i64, p, p, p],
            "rpq_query_levels": [p, p, i32, p, i32, p, p, i64, p, p],
            "rpq_query_witness": [p, p, i32, p, i32, i32, p, p, i32, p, p],
            "rpq_query_batch": [p, i32, p, p, i32, p, p, i64, p, p],
            "rpq_serve_create": [p, p, pp],
            "rpq_serve_submit": [p, p, i32, p],
            "rpq_serve_poll": [p, u64, p, i64, p],
            "rpq_serve_drain": [p, i64],
            "rpq_serve_stats": [p, p],
            "rpq_serve_stats_get": [p, p],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = st
        for name in ("rpq_graph_free", "rpq_nfa_free", "rpq_serve_destroy"):
            getattr(L, name).argtypes = [p]
            getattr(L, name).restype = None
        L.rpq_last_error.restype = ctypes.c_char_p
        L.rpq_version.restype = ctypes.c_char_p
        L.rpq_kernel_launches.argtypes = []
        L.rpq_kernel_launches.restype = ctypes.c_uint64
        _LIB = L
    return _LIB


def _check(status: int, allow=()):
    if status != RPQ_OK and status not in allow:
        raise RpqError(status, lib().rpq_last_error().decode(errors="replace"))
    return status


def _stream_handle(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _host_i32(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1))
    return a, ctypes.c_void_p(a.ctypes.data if a.size else 0)


def _ptr(x):
    """Raw pointer of a numpy array or torch tensor."""
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(x.ctypes.data)


# ------------------------------------------------------------- allocator --

_ALLOC_CB = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_CB = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
# Every callback pair ever installed stays referenced until exit: memory a
# pair allocated goes back through that pair's free callback, possibly after
# another allocator has been installed (a graph loaded under the first one
# and freed later).
_alloc_refs = []


def rpq_set_allocator(alloc=None, free=None):
    """Install Python callables (size -> int pointer, pointer -> None) as the
    device allocator, or restore cudaMalloc with no arguments.  Buffers
    allocated before the change are still freed through the callable that
    allocated them, so that callable must keep working until they are."""
    if alloc is None:
        _check(lib().rpq_set_allocator(None, None, None))
        return
    a = _ALLOC_CB(lambda size, ctx: int(alloc(int(size)) or 0))
    f = _FREE_CB(lambda ptr, ctx: free(int(ptr)))
    _alloc_refs.append((a, f))
    _check(lib().rpq_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p),
                                   None))


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching
    allocator (memory then shows up in torch.cuda.memory_allocated)."""
    import torch

    dev = torch.cuda.current_device()

    def alloc(size):
        return torch.cuda.caching_allocator_alloc(size, dev)

    def free(ptr):
        torch.cuda.caching_allocator_delete(ptr)

    rpq_set_allocator(alloc, free)


# ----------------------------------------------------------------- graph --

class Graph:
    """Handle of a device-resident graph (per-label CSR + CSC)."""

    def __init__(self, handle, n, n_labels):
        self.h = handle
        self.n = n
        self.n_labels = n_labels

    def close(self):
        if self.h:
            lib().rpq_graph_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def n_edges(self, label: int = -1) -> int:
        m = ctypes.c_int64()
        _check(lib().rpq_graph_info(self.h, label, None, None, ctypes.byref(m)))
        return m.value


def rpq_graph_load(n_vertices, n_labels, src, dst, label, stream=None) -> Graph:
    s, ps = _host_i32(src)
    d, pd = _host_i32(dst)
    l, pl = _host_i32(label)
    if not (s.size == d.size == l.size):
        raise ValueError("src, dst, label must have the same length")
    out = ctypes.c_void_p()
    _check(lib().rpq_graph_load(int(n_vertices), int(n_labels), s.size, ps, pd, pl,
                                _stream_handle(stream), ctypes.byref(out)))
    return Graph(out, int(n_vertices), int(n_labels))


def rpq_graph_free(g: Graph):
    g.close()


def rpq_graph_info(g: Graph, label: int = -1):
    n, L, m = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib().rpq_graph_info(g.h, label, ctypes.byref(n), ctypes.byref(L), ctypes.byref(m)))
    return n.value, L.value, m.value


def rpq_graph_export(g: Graph, label: int, inverse: bool):
    off = np.zeros(g.n + 1, np.int64)
    _check(lib().rpq_graph_export(g.h, label, int(inverse), _ptr(off), None, 0))
    nbr = np.zeros(max(int(off[-1]), 1), np.int32)
    _check(lib().rpq_graph_export(g.h, label, int(inverse), _ptr(off), _ptr(nbr), nbr.size))
    return off, nbr[: int(off[-1])]


def rpq_graph_autotune_batch(g: Graph, nfas, sources, stream=None):
    """Tunes the bit-lane engine (inline row length, pull divisor) on sample
    queries; returns (lane_hub, pull_div)."""
    n = len(nfas)
    handles = (ctypes.c_void_p * n)(*[x.h.value for x in nfas])
    src, psrc = _host_i32(sources)
    h, pdv = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().rpq_graph_autotune_batch(g.h, n, handles, psrc, ctypes.byref(h), ctypes.byref(pdv),
                                          _stream_handle(stream)))
    return h.value, pdv.value


def rpq_graph_set_hybrid(g: Graph, switch_pairs: int):
    """Algorithm 2 while fewer than ``switch_pairs`` pairs are visited, then
    Algorithm 1 (section 5.1's hybrid); 0 turns it off."""
    _check(lib().rpq_graph_set_hybrid(g.h, int(switch_pairs)))


def rpq_graph_set_rare_plan(g: Graph, max_edges: int):
    """Rare label first for single queries whose accepted words all read a
    label direction with at most ``max_edges`` edges; 0 turns it off."""
    _check(lib().rpq_graph_set_rare_plan(g.h, int(max_edges)))


def rpq_graph_autotune(g: Graph, nfas, sources, stream=None):
    """Measures the push/pull threshold and the one-CTA level size on sample
    queries and stores them in the graph; returns (alpha, min_pull,
    solo_mass)."""
    n = len(nfas)
    handles = (ctypes.c_void_p * n)(*[x.h.value for x in nfas])
    src, psrc = _host_i32(sources)
    a, m, so = ctypes.c_float(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().rpq_graph_autotune(g.h, n, handles, psrc, ctypes.byref(a), ctypes.byref(m),
                                    ctypes.byref(so), _stream_handle(stream)))
    return a.value, m.value, so.value


# ------------------------------------------------------------- automaton --

class Nfa:
    def __init__(self, handle):
        self.h = handle

    def close(self):
        if self.h:
            lib().rpq_nfa_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        S, T, L = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().rpq_nfa_info(self.h, ctypes.byref(S), ctypes.byref(T), ctypes.byref(L)))
        return S.value, T.value, L.value

    def accepts(self, word) -> bool:
        w, pw = _host_i32(word)
        r = ctypes.c_int32()
        _check(lib().rpq_nfa_accepts(self.h, pw, w.size, ctypes.byref(r)))
        return bool(r.value)

    def export(self):
        S, T, L = self.info()
        f = np.zeros(max(T, 1), np.int32); t = np.zeros(max(T, 1), np.int32)
        a = np.zeros(max(T, 1), np.int32)
        sm, fm = ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().rpq_nfa_export(self.h, _ptr(f), _ptr(t), _ptr(a), max(T, 1),
                                    ctypes.byref(sm), ctypes.byref(fm)))
        return {"n_states": S, "n_labels": L, "from": f[:T], "to": t[:T], "label": a[:T],
                "starts": [q for q in range(64) if (sm.value >> q) & 1],
                "finals": [q for q in range(64) if (fm.value >> q) & 1]}


def rpq_nfa_compile(regex: str, n_labels: int) -> Nfa:
    out = ctypes.c_void_p()
    _check(lib().rpq_nfa_compile(regex.encode(), int(n_labels), ctypes.byref(out)))
    return Nfa(out)


def rpq_nfa_from_transitions(n_states, n_labels, transitions, starts, finals) -> Nfa:
    tr = list(transitions)
    f, pf = _host_i32([t[0] for t in tr])
    a, pa = _host_i32([t[1] for t in tr])
    t, pt = _host_i32([t[2] for t in tr])
    s, ps = _host_i32(starts)
    fi, pfi = _host_i32(finals)
    out = ctypes.c_void_p()
    _check(lib().rpq_nfa_from_transitions(int(n_states), int(n_labels), len(tr), pf, pt, pa,
                                          s.size, ps, fi.size, pfi, ctypes.byref(out)))
    return Nfa(out)


def rpq_nfa_reverse(nfa: Nfa) -> Nfa:
    out = ctypes.c_void_p()
    _check(lib().rpq_nfa_reverse(nfa.h, ctypes.byref(out)))
    return Nfa(out)


def rpq_nfa_accepts(nfa: Nfa, word) -> bool:
    return nfa.accepts(word)


def rpq_nfa_free(nfa: Nfa):
    nfa.close()


# ----------------------------------------------------------------- query --

def rpq_query(g: Graph, nfa: Nfa, source: int, max_levels: int = 0, out=None, stream=None,
              with_stats: bool = False):
    """Single-source query.  Without ``out`` the answer comes back as a sorted
    int32 numpy array (host copy made by the library); with a device tensor
    ``out`` the library writes into it and the count is returned."""
    st = RpqStats() if with_stats else None
    cnt = ctypes.c_int64()
    sp = ctypes.byref(st) if st is not None else None
    if out is None:
        # no buffer: the library keeps the answer in pinned host memory
        # (written there by the kernel); one copy into the result array
        _check(lib().rpq_query(g.h, nfa.h, int(source), int(max_levels), None, 0,
                               ctypes.byref(cnt), sp, _stream_handle(stream)),
               allow=(RPQ_ERR_CAPACITY,))
        ptr, n = ctypes.POINTER(ctypes.c_int32)(), ctypes.c_int64()
        _check(lib().rpq_last_answer(ctypes.byref(ptr), ctypes.byref(n)))
        res = _copy_answer(ptr, n.value)
    else:
        _check(lib().rpq_query(g.h, nfa.h, int(source), int(max_levels), _ptr(out), out.numel(),
                               ctypes.byref(cnt), sp, _stream_handle(stream)))
        res = int(cnt.value)
    return (res, st.as_dict()) if with_stats else res


# Host answers of at least this many vertices are copied out of the
# library's buffer by several threads (numpy releases the GIL while it
# copies): on the Grace host an 80 MB answer moves at 13 GB/s on one
# thread, 58 GB/s on eight (64 on twelve, 60 on sixteen).
_PARALLEL_COPY_MIN = 1 << 20
_copy_pool = None


def _copy_answer(ptr, n: int):
    """A numpy copy of the n-entry answer at ptr (the library's per-thread
    host buffer, overwritten by this thread's next query)."""
    global _copy_pool
    if n == 0:
        return np.empty(0, np.int32)
    src = np.ctypeslib.as_array(ptr, shape=(n,))
    if n < _PARALLEL_COPY_MIN:
        return src.copy()
    if _copy_pool is None:
        import concurrent.futures as cf

        _copy_pool = cf.ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1)))
    dst = np.empty(n, np.int32)
    k = _copy_pool._max_workers
    cut = [n * i // k for i in range(k + 1)]
    list(_copy_pool.map(lambda i: np.copyto(dst[cut[i]:cut[i + 1]], src[cut[i]:cut[i + 1]]),
                        range(k)))
    return dst


class QueryRunner:
    """Repeated single-source queries into one device tensor ``out`` on one
    stream: the ctypes arguments that do not change between calls are built
    once, so a call costs the library's own work and one foreign call.
    ``run(nfa, source)`` returns the answer count; with ``with_stats`` the
    statistics of the last call are in ``self.stats`` (an :class:`RpqStats`,
    overwritten by the next call)."""

    def __init__(self, g: Graph, out, stream=None, max_levels: int = 0,
                 with_stats: bool = False):
        self._g, self._out = g, out  # kept alive while the runner is
        self._f = lib().rpq_query
        self._gh = g.h
        self._optr = _ptr(out)
        self._cap = ctypes.c_int64(out.numel())
        self._levels = ctypes.c_int32(int(max_levels))
        self._cnt = ctypes.c_int64()
        self._pcnt = ctypes.byref(self._cnt)
        self.stats = RpqStats() if with_stats else None
        self._pst = ctypes.byref(self.stats) if with_stats else None
        self._sh = _stream_handle(stream)

    def run(self, nfa: Nfa, source: int) -> int:
        st = self._f(self._gh, nfa.h, source, self._levels, self._optr, self._cap, self._pcnt,
                     self._pst, self._sh)
        if st != RPQ_OK:
            _check(st)
        return self._cnt.value


def _answer_call(call, out, with_stats):
    """Shared marshalling of the calls that return one answer like rpq_query:
    ``call(out_ptr, capacity, count_ref, stats_ref)``."""
    st = RpqStats() if with_stats else None
    cnt = ctypes.c_int64()
    sp = ctypes.byref(st) if st is not None else None
    if out is None:
        _check(call(None, 0, ctypes.byref(cnt), sp), allow=(RPQ_ERR_CAPACITY,))
        if cnt.value == 0:
            res = np.empty(0, np.int32)
        else:
            ptr, n = ctypes.POINTER(ctypes.c_int32)(), ctypes.c_int64()
            _check(lib().rpq_last_answer(ctypes.byref(ptr), ctypes.byref(n)))
            res = _copy_answer(ptr, n.value)
    else:
        _check(call(_ptr(out), out.numel(), ctypes.byref(cnt), sp))
        res = int(cnt.value)
    return (res, st.as_dict()) if with_stats else res


def rpq_query_multi(g: Graph, nfa: Nfa, sources, max_levels: int = 0, out=None, stream=None,
                    with_stats: bool = False):
    """Query from a set of sources V_s (level 0 = Q_S x V_s): the vertices
    reached from some source; same outputs as :func:`rpq_query`."""
    src, psrc = _host_i32(sources)
    return _answer_call(lambda o, c, n, sp: lib().rpq_query_multi(
        g.h, nfa.h, src.size, psrc, int(max_levels), o, c, n, sp, _stream_handle(stream)),
        out, with_stats)


def rpq_query_sdr(g: Graph, nfa: Nfa, target: int, max_levels: int = 0, out=None, stream=None,
                  with_stats: bool = False):
    """Single-destination query: the vertices from which some 2-path to
    ``target`` spells an accepted word; same outputs as :func:`rpq_query`."""
    return _answer_call(lambda o, c, n, sp: lib().rpq_query_sdr(
        g.h, nfa.h, int(target), int(max_levels), o, c, n, sp, _stream_handle(stream)),
        out, with_stats)


def rpq_query_levels(g: Graph, nfa: Nfa, sources, max_levels: int = 0, stream=None):
    """Answer of the query from ``sources`` with each vertex's level of first
    reach (the length of a shortest accepted word that labels a 2-path to
    it); returns (vertices, levels) as int32 numpy arrays."""
    src, psrc = _host_i32(sources)
    cnt = ctypes.c_int64()
    cap = g.n
    v = np.empty(max(cap, 1), np.int32)
    lv = np.empty(max(cap, 1), np.int32)
    _check(lib().rpq_query_levels(g.h, nfa.h, src.size, psrc, int(max_levels), _ptr(v), _ptr(lv),
                                  cap, ctypes.byref(cnt), _stream_handle(stream)))
    return v[: cnt.value].copy(), lv[: cnt.value].copy()


def rpq_query_witness(g: Graph, nfa: Nfa, sources, target: int, max_levels: int = 0,
                      stream=None):
    """A shortest witness of ``target``: (vertices, symbols) with k + 1
    vertices from a source to the target and the k symbols of the word (a <
    L: label a forward; a >= L: label a - L walked backwards), or None when
    the target is not in the answer."""
    src, psrc = _host_i32(sources)
    cap = 1024
    while True:
        pv = np.empty(cap, np.int32)
        ps = np.empty(cap, np.int32)
        ln = ctypes.c_int32()
        s = _check(lib().rpq_query_witness(g.h, nfa.h, src.size, psrc, int(target),
                                           int(max_levels), _ptr(pv), _ptr(ps), cap,
                                           ctypes.byref(ln), _stream_handle(stream)),
                   allow=(RPQ_ERR_CAPACITY,))
        if s == RPQ_OK:
            break
        cap = ln.value + 1
    if ln.value < 0:
        return None
    return pv[: ln.value + 1].copy(), ps[: ln.value].copy()


def rpq_query_noalloc(g: Graph, nfa: Nfa, source: int, out, max_levels: int = 0,
                      stream=None) -> int:
    """Single-source query through the entry point that allocates no device
    memory (its workspace is a fixed array inside the library).  ``out`` is a
    device int32 tensor; returns the number of answer vertices written."""
    cnt = ctypes.c_int64()
    _check(lib().rpq_query_noalloc(g.h, nfa.h, int(source), int(max_levels), _ptr(out),
                                   out.numel(), ctypes.byref(cnt), _stream_handle(stream)))
    return int(cnt.value)


def rpq_query_bitset(g: Graph, nfa: Nfa, source: int, max_levels: int = 0, out=None,
                     stream=None, with_stats: bool = False):
    st = RpqStats() if with_stats else None
    W = (g.n + 63) // 64
    bits = out if out is not None else np.zeros(W, np.uint64)
    cnt = ctypes.c_int64()
    _check(lib().rpq_query_bitset(g.h, nfa.h, int(source), int(max_levels), _ptr(bits),
                                  ctypes.byref(cnt), ctypes.byref(st) if st is not None else None,
                                  _stream_handle(stream)))
    return (bits, int(cnt.value), st.as_dict()) if with_stats else (bits, int(cnt.value))


def rpq_query_batch(g: Graph, nfas, sources, max_levels: int = 0, stream=None,
                    with_stats: bool = False):
    """Batch of single-source queries in one launch; returns a list of sorted
    int32 arrays (and per-query stats dicts if asked)."""
    n = len(nfas)
    handles = (ctypes.c_void_p * max(n, 1))(*[x.h.value if isinstance(x.h, ctypes.c_void_p)
                                              else x.h for x in nfas])
    src, psrc = _host_i32(sources)
    offs = np.zeros(n + 1, np.int64)
    stats = (RpqStats * max(n, 1))() if with_stats else None
    # room for every answer up to 2^27 ids (pages are only touched as written),
    # so that a second traversal for a larger buffer is rarely needed
    cap = max(1, min(n * g.n, 1 << 27))
    while True:
        buf = np.empty(max(cap, 1), np.int32)
        s = _check(lib().rpq_query_batch(g.h, n, handles, psrc, int(max_levels), _ptr(offs),
                                         _ptr(buf), cap, stats, _stream_handle(stream)),
                   allow=(RPQ_ERR_CAPACITY,))
        if s == RPQ_OK:
            break
        cap = int(offs[-1])
    res = [buf[offs[i]:offs[i + 1]].copy() for i in range(n)]
    if with_stats:
        return res, [stats[i].as_dict() for i in range(n)]
    return res


# --------------------------------------------------------------- serving --

class Server:
    def __init__(self, g: Graph, max_lanes=0, max_states=0, queue_capacity=0, memory_budget=0,
                 max_levels=0, engine=0):
        cfg = RpqServeConfig(max_lanes, max_states, queue_capacity, memory_budget, max_levels,
                             engine)
        out = ctypes.c_void_p()
        _check(lib().rpq_serve_create(g.h, ctypes.byref(cfg), ctypes.byref(out)))
        self.h = out
        self.graph = g
        self._nfas = {}

    def submit(self, nfa: Nfa, source: int) -> int:
        t = ctypes.c_uint64()
        _check(lib().rpq_serve_submit(self.h, nfa.h, int(source), ctypes.byref(t)))
        self._nfas[t.value] = nfa  # keep the automaton alive until polled
        return t.value

    def poll(self, ticket: int):
        """Answer array when done, None while running."""
        cnt = ctypes.c_int64()
        cap = 1 << 16
        while True:
            buf = np.empty(cap, np.int32)
            s = _check(lib().rpq_serve_poll(self.h, ticket, _ptr(buf), cap, ctypes.byref(cnt)),
                       allow=(RPQ_ERR_BUSY, RPQ_ERR_CAPACITY))
            if s == RPQ_ERR_BUSY:
                return None
            if s == RPQ_OK:
                self._nfas.pop(ticket, None)
                n = int(cnt.value)
                # a small answer is copied out of the 64K-entry buffer; a
                # large one (the buffer was sized for it) is returned as is
                return buf if n == cap else buf[:n].copy()
            cap = int(cnt.value)

    def drain(self, timeout_ms: int = 600000):
        _check(lib().rpq_serve_drain(self.h, int(timeout_ms)))

    def stats(self):
        st = RpqServeStats()
        _check(lib().rpq_serve_stats(self.h, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if self.h:
            lib().rpq_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rpq_serve_create(g: Graph, **cfg) -> Server:
    return Server(g, **cfg)


def rpq_version() -> str:
    return lib().rpq_version().decode()


def rpq_last_error() -> str:
    return lib().rpq_last_error().decode(errors="replace")


def rpq_kernel_launches() -> int:
    """Kernels the library has launched in this process so far."""
    return int(lib().rpq_kernel_launches())
