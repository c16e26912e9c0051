"""CPU oracle for single-source 2-RPQ.

TEST INFRASTRUCTURE, not product code: only ``tests/``,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
it.  It shares no code with the GPU library and the GPU library never calls
it.

Functions and the passages they follow (paper arXiv:2412.10287):

* :func:`ssr` -- the pair BFS of ``rpq_oracle.c``: the single-source
  reachability answer of section 2 computed level by level as in
  Algorithm 1 (section 4), one level per word length (appendix invariant).
* :meth:`OracleGraph.query` -- the same search from a set of sources V_s
  (the 2-RPQ of section 2 takes a set of starting vertices), optionally with
  the level of first reach of every answer vertex: the length of the
  shortest accepted word labelling a 2-path from a source to it.
* :meth:`OracleGraph.sdr` -- single-destination reachability (section 2) by its own
  definition: the vertices u whose single-source answer contains v_f.
* :func:`check_witness` -- whether a given vertex/symbol sequence is a 2-path
  from a source that spells an accepted word (a checker for path outputs).
* :func:`alg1_dense` -- Algorithm 1 written with dense Boolean matrices in the
  paper's own notation: M <- (OR_a (N^a)^T x M x G^a)<not P>, P <- P + M,
  until M = 0; result F x P (section 3 operations, section 4 listing).
* :func:`alg2_dense` -- Algorithm 2 (no traversal matrix): P <- P + OR_a
  (N^a)^T x P x G^a until P stops changing.
* :func:`brute_force` -- the definition itself on tiny inputs: every word of
  length <= k over the 2-way alphabet, the vertices reachable from v_s along a
  2-path spelling it, kept when the automaton accepts the word.

Readings of the paper taken here (each listed with its reason in the design
notes): level 0 is Q_S x {v_s} (zero-length paths count, section 2); the
mask applies to the produced pairs (the listing of Algorithm 1); labels
a >= L denote a^- and are traversed through the transpose (section 3:
G^{a^-} = (G^a)^T); ``max_levels = k`` yields P_k, the pairs reached by words
of length <= k (section 4).
"""

from __future__ import annotations

import ctypes
import itertools
import os

import numpy as np

from .regex_nfa import Nfa, compile_regex, inverse_nfa, RegexError  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

COUNTER_NAMES = ("levels", "visited", "product_edges", "push_bytes", "expanded", "answer")


def lib_path() -> str:
    return os.path.join(_HERE, "librpq_oracle.so")


def build(force: bool = False) -> str:
    """Compile ``rpq_oracle.c`` with gcc (plain C, -O2)."""
    from .build_oracle import build_library

    return build_library(force=force)


def _lib():
    global _LIB
    if _LIB is None:
        path = build()
        L = ctypes.CDLL(path)
        i32, i64, p = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        L.oracle_graph_new.restype = p
        L.oracle_graph_new.argtypes = [i32, i32, i64, p, p, p]
        L.oracle_graph_free.restype = None
        L.oracle_graph_free.argtypes = [p]
        L.oracle_ssr_graph.restype = ctypes.c_int
        L.oracle_ssr_graph.argtypes = [p, i32, i32, p, p, p, i32, p, i32, p, i32, i32,
                                       p, p, p, i32, p]
        L.oracle_query_graph.restype = ctypes.c_int
        L.oracle_query_graph.argtypes = [p, i32, i32, p, p, p, i32, p, i32, p, i32, p, i32,
                                         p, p, p, i32, p, p]
        _LIB = L
    return _LIB


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else None


class OracleGraph:
    """Adjacency lists of a COO edge list, built once for many queries."""

    def __init__(self, n: int, n_labels: int, src, dst, lab):
        self.n = int(n)
        self.L = int(n_labels)
        self._src = np.ascontiguousarray(src, dtype=np.int32)
        self._dst = np.ascontiguousarray(dst, dtype=np.int32)
        self._lab = np.ascontiguousarray(lab, dtype=np.int32)
        m = self._src.size
        dummy = np.zeros(1, np.int32)
        h = _lib().oracle_graph_new(
            self.n, self.L, m,
            _ptr(self._src) or _ptr(dummy), _ptr(self._dst) or _ptr(dummy),
            _ptr(self._lab) or _ptr(dummy))
        if not h:
            raise ValueError("oracle_graph_new rejected the graph")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib().oracle_graph_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def ssr(self, nfa: Nfa, source: int, max_levels: int = 0, want_visited: bool = False,
            level_cap: int = 0, want_first_level: bool = False):
        """Run one query.  Returns a dict with ``answer`` (sorted int32 vertex
        ids), ``counters`` (dict), optionally ``visited`` (S x n bool),
        ``level_sizes`` (pairs per level) and ``first_level`` (n int32: level
        of first reach of each answer vertex, -1 elsewhere)."""
        return self.query(nfa, [int(source)], max_levels, want_visited, level_cap,
                          want_first_level)

    def query(self, nfa: Nfa, sources, max_levels: int = 0, want_visited: bool = False,
              level_cap: int = 0, want_first_level: bool = False):
        """The query from the set of sources ``sources`` (level 0 = Q_S x
        V_s); same outputs as :meth:`ssr`."""
        S, tf, tl, tt, st, fi = nfa.arrays()
        i32 = lambda x: np.ascontiguousarray(np.asarray(x, dtype=np.int32).reshape(-1))
        tf, tl, tt, st, fi = i32(tf), i32(tl), i32(tt), i32(st), i32(fi)
        srcs = i32(sources)
        ans = np.zeros(self.n, np.uint8)
        vis = np.zeros((S, self.n), np.uint8) if want_visited else None
        lv = np.zeros(level_cap, np.int64) if level_cap > 0 else None
        fl = np.zeros(self.n, np.int32) if want_first_level else None
        cnt = np.zeros(len(COUNTER_NAMES), np.int64)
        rc = _lib().oracle_query_graph(
            self._h, S, tf.size, _ptr(tf), _ptr(tl), _ptr(tt), st.size, _ptr(st),
            fi.size, _ptr(fi), srcs.size, _ptr(srcs), int(max_levels), _ptr(ans), _ptr(vis),
            _ptr(lv), int(level_cap), _ptr(cnt), _ptr(fl))
        if rc != 0:
            raise ValueError(f"oracle_query_graph failed with status {rc}")
        out = {
            "answer": np.flatnonzero(ans).astype(np.int32),
            "counters": dict(zip(COUNTER_NAMES, (int(x) for x in cnt))),
        }
        if vis is not None:
            out["visited"] = vis.astype(bool)
        if lv is not None:
            out["level_sizes"] = lv
        if fl is not None:
            out["first_level"] = fl
        return out

    def sdr(self, nfa: Nfa, target: int, candidates=None):
        """Single-destination reachability (section 2): the sorted vertices u
        such that some 2-path from u to ``target`` spells an accepted word,
        i.e. whose single-source answer holds ``target`` -- the definition,
        one single-source query per candidate u (all vertices by default)."""
        cand = range(self.n) if candidates is None else candidates
        hit = [int(u) for u in cand if target in set(self.ssr(nfa, int(u))["answer"].tolist())]
        return np.array(sorted(hit), dtype=np.int32)


def ssr(n, n_labels, src, dst, lab, nfa: Nfa, source: int, max_levels: int = 0, **kw):
    """One-shot single-source query (builds and frees the adjacency lists)."""
    g = OracleGraph(n, n_labels, src, dst, lab)
    try:
        return g.ssr(nfa, source, max_levels, **kw)
    finally:
        g.close()


# ------------------------------------------------ dense restatements -------

def _label_matrices(n, L, src, dst, lab):
    """G^a for a in [0, 2L): G^a[u, v] = 1 iff u -a-> v; G^{a+L} = (G^a)^T."""
    G = np.zeros((2 * L, n, n), dtype=bool)
    for u, v, a in zip(src, dst, lab):
        G[a, u, v] = True
    for a in range(L):
        G[a + L] = G[a].T
    return G


def _nfa_matrices(nfa: Nfa):
    S, L = nfa.n_states, nfa.n_labels
    N = np.zeros((2 * L, S, S), dtype=bool)
    for q, a, r in nfa.transitions:
        N[a, q, r] = True
    return N


def _bmm(A, B):
    return (A.astype(np.int64) @ B.astype(np.int64)) > 0


def alg1_dense(n, L, src, dst, lab, nfa: Nfa, source: int, max_levels: int = 0):
    """Algorithm 1 with dense Boolean matrices.  Returns (P, F x P, levels)."""
    G = _label_matrices(n, L, src, dst, lab)
    N = _nfa_matrices(nfa)
    S = nfa.n_states
    M = np.zeros((S, n), dtype=bool)
    for q in nfa.starts:
        M[q, source] = True
    P = M.copy()  # reading: P_0 = M_0 (zero-length paths)
    F = np.zeros((1, S), dtype=bool)
    for q in nfa.finals:
        F[0, q] = True
    labels = [a for a in range(2 * L) if N[a].any() and G[a].any()]  # Sigma^<-> cap L^<->
    levels = 0
    while M.any() and (max_levels == 0 or levels < max_levels):
        acc = np.zeros((S, n), dtype=bool)
        for a in labels:
            acc |= _bmm(_bmm(N[a].T, M), G[a])
        M = acc & ~P
        P = P | M
        if M.any():
            levels += 1  # counts non-empty levels after level 0
    return P, _bmm(F, P)[0], levels


def alg2_dense(n, L, src, dst, lab, nfa: Nfa, source: int):
    """Algorithm 2 (no traversal matrix) with dense Boolean matrices."""
    G = _label_matrices(n, L, src, dst, lab)
    N = _nfa_matrices(nfa)
    S = nfa.n_states
    P = np.zeros((S, n), dtype=bool)
    for q in nfa.starts:
        P[q, source] = True
    F = np.zeros((1, S), dtype=bool)
    for q in nfa.finals:
        F[0, q] = True
    labels = [a for a in range(2 * L) if N[a].any() and G[a].any()]
    while True:
        acc = P.copy()
        for a in labels:
            acc |= _bmm(_bmm(N[a].T, P), G[a])
        if (acc == P).all():
            break
        P = acc
    return P, _bmm(F, P)[0]


# ----------------------------------------------------------- brute force ---

def brute_force_levels(n, L, src, dst, lab, source, accepts, max_len: int):
    """answers[k] for k = 0..max_len: the query answer restricted to words of
    length <= k, straight from the definition (section 2, single-source
    reachability over 2-paths): every word w over the 2-way alphabet, the set
    reach(w) of vertices at the end of a 2-path from ``source`` spelling w
    (a forward symbol a walks u -a-> v from u to v, the symbol a + L walks it
    from v to u), and the union of reach(w) over the accepted words.  Words
    are enumerated depth-first; a word whose reach set is empty is not
    extended, since no 2-path spells any of its extensions.  ``accepts`` is
    any word-membership predicate.  ``source`` may also be a collection of
    vertices (a set of sources V_s): a 2-path may then start at any of
    them."""
    edges = {s: [] for s in range(2 * L)}
    for u, v, a in zip(map(int, src), map(int, dst), map(int, lab)):
        edges[a].append((u, v))
        edges[a + L].append((v, u))
    per_len = [set() for _ in range(max_len + 1)]

    def dfs(word, reach):
        if accepts(word):
            per_len[len(word)].update(reach)
        if len(word) == max_len:
            return
        for s in range(2 * L):
            nxt = {y for (x, y) in edges[s] if x in reach}
            if nxt:
                dfs(word + (s,), nxt)

    start = {int(source)} if np.ndim(source) == 0 else {int(x) for x in source}
    dfs((), start)
    out, acc = [], set()
    for k in range(max_len + 1):
        acc |= per_len[k]
        out.append(np.array(sorted(acc), dtype=np.int32))
    return out


def brute_force(n, L, src, dst, lab, source, accepts, max_len: int):
    """Answer restricted to words of length <= max_len (see brute_force_levels)."""
    return brute_force_levels(n, L, src, dst, lab, source, accepts, max_len)[-1]


def first_levels_from(levels_answers, n):
    """Level of first reach per vertex from per-bound answers (answers[k] =
    the answer restricted to words of length <= k): the smallest k whose
    answer holds v, -1 if none does."""
    out = np.full(n, -1, np.int32)
    for k in range(len(levels_answers) - 1, -1, -1):
        out[np.asarray(levels_answers[k], dtype=np.int64)] = k
    return out


def check_witness(n, L, src, dst, lab, accepts, sources, target, vertices, symbols):
    """Whether vertices[0..k] / symbols[0..k-1] is a witness of ``target``:
    vertices[0] is a source, vertices[-1] is the target, step i walks an
    edge vertices[i] -a-> vertices[i+1] of label a = symbols[i] (a < L) or,
    for a >= L, an edge vertices[i+1] -(a-L)-> vertices[i] backwards (the
    2-path of section 2), and the word of symbols is accepted.  Returns
    (ok, reason)."""
    vertices = [int(x) for x in vertices]
    symbols = [int(x) for x in symbols]
    if len(vertices) != len(symbols) + 1:
        return False, "vertices must be one longer than symbols"
    if vertices[0] not in {int(x) for x in np.atleast_1d(sources)}:
        return False, "does not start at a source"
    if vertices[-1] != int(target):
        return False, "does not end at the target"
    edges = set(zip(map(int, src), map(int, dst), map(int, lab)))
    for i, a in enumerate(symbols):
        u, v = vertices[i], vertices[i + 1]
        if not 0 <= a < 2 * L:
            return False, f"symbol {a} out of range"
        if a < L and (u, v, a) not in edges:
            return False, f"step {i}: no edge {u} -{a}-> {v}"
        if a >= L and (v, u, a - L) not in edges:
            return False, f"step {i}: no edge {v} -{a - L}-> {u} to walk backwards"
    if not accepts(tuple(symbols)):
        return False, "word not accepted"
    return True, ""
