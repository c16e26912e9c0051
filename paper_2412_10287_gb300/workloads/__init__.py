"""Seeded synthetic inputs for single-source 2-RPQ (graphs, queries, arrivals).

This module holds no part of the query method: it only samples graphs (COO
edge lists with labels) and query descriptions (regular expressions over
label ids, sources, arrival times).  The GPU library and the CPU oracle both
consume these inputs; neither imports the other.

The paper's datasets (Wikidata, Yago-2S, RPQBench; section 5.2) are not
available, so the workloads are synthetic graphs with their shapes: power-law
degrees, many labels with heavily skewed label frequencies (cf. Table 4, one
label carrying most edges and some labels fewer than 200 edges), and query
templates of the kinds listed in Table 3 (a*, a.b*, (a|b)*.c, inverse labels,
chains and repeated pairs).

All sampling is in ``rpqgen.c`` (xoshiro256**, alias tables); its outputs
are bit-identical across x86-64 and aarch64 for a given seed.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rpqgen.c")
_OUT = os.path.join(_HERE, "librpqgen.so")
_LIB = None


def build(force: bool = False) -> str:
    """Compile the generator library with gcc (no FMA contraction, so that
    results match across architectures)."""
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    tmp = _OUT + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                    "-Wall", "-shared", "-fPIC", "-fvisibility=hidden", "-o", tmp, _SRC],
                   check=True)
    os.replace(tmp, _OUT)
    return _OUT


def _lib():
    global _LIB
    if _LIB is None:
        L = ctypes.CDLL(build())
        i32, i64, u64, d, p = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                               ctypes.c_double, ctypes.c_void_p)
        L.rpqgen_draw_u64.argtypes = [u64, u64, i64, p]
        L.rpqgen_below.argtypes = [u64, u64, i64, u64, p]
        L.rpqgen_zipf.argtypes = [i64, d, u64, u64, i64, p]
        L.rpqgen_exponential.argtypes = [d, u64, u64, i64, p]
        L.rpqgen_er.argtypes = [i64, i64, i32, u64, p, p, p]
        L.rpqgen_rmat.argtypes = [i32, i64, d, d, d, i32, d, u64, p, p, p]
        L.rpqgen_chung_lu.argtypes = [i64, i64, d, i32, d, u64, p, p, p]
        for f in ("rpqgen_det_pow", "rpqgen_det_log", "rpqgen_det_exp"):
            getattr(L, f).restype = d
        L.rpqgen_det_pow.argtypes = [d, d]
        L.rpqgen_det_log.argtypes = [d]
        L.rpqgen_det_exp.argtypes = [d]
        _LIB = L
    return _LIB


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"{what} failed with status {rc}")


# --------------------------------------------------------------- streams --

def below(seed: int, stream: int, count: int, bound: int) -> np.ndarray:
    out = np.empty(max(count, 1), np.int64)
    _check(_lib().rpqgen_below(seed, stream, count, bound, _p(out)), "rpqgen_below")
    return out[:count]


def zipf(k: int, s: float, seed: int, stream: int, count: int) -> np.ndarray:
    out = np.empty(max(count, 1), np.int32)
    _check(_lib().rpqgen_zipf(k, s, seed, stream, count, _p(out)), "rpqgen_zipf")
    return out[:count]


def exponential(rate: float, seed: int, stream: int, count: int) -> np.ndarray:
    out = np.empty(max(count, 1), np.float64)
    _check(_lib().rpqgen_exponential(rate, seed, stream, count, _p(out)), "rpqgen_exponential")
    return out[:count]


# ---------------------------------------------------------------- graphs --

@dataclass
class Graph:
    """Edge-labelled graph as COO triples (section 2 data model): edge
    src[i] -lab[i]-> dst[i], labels in [0, n_labels).  May hold duplicate
    triples and self-loops."""

    name: str
    n: int
    n_labels: int
    src: np.ndarray
    dst: np.ndarray
    lab: np.ndarray

    @property
    def m(self) -> int:
        return int(self.src.size)


def er_graph(n: int, m: int, n_labels: int, seed: int) -> Graph:
    src = np.empty(m, np.int32); dst = np.empty(m, np.int32); lab = np.empty(m, np.int32)
    _check(_lib().rpqgen_er(n, m, n_labels, seed, _p(src), _p(dst), _p(lab)), "rpqgen_er")
    return Graph(f"er_n{n}_m{m}_L{n_labels}_s{seed}", n, n_labels, src, dst, lab)


def rmat_graph(scale: int, samples: int, n_labels: int, seed: int,
               a=0.57, b=0.19, c=0.19, zipf_s=1.0) -> Graph:
    src = np.empty(samples, np.int32); dst = np.empty(samples, np.int32)
    lab = np.empty(samples, np.int32)
    _check(_lib().rpqgen_rmat(scale, samples, a, b, c, n_labels, zipf_s, seed,
                              _p(src), _p(dst), _p(lab)), "rpqgen_rmat")
    return Graph(f"rmat{scale}_e{samples}_L{n_labels}_s{seed}", 1 << scale, n_labels,
                 src, dst, lab)


def chung_lu_graph(n: int, m: int, gamma: float, n_labels: int, zipf_s: float,
                   seed: int) -> Graph:
    src = np.empty(m, np.int32); dst = np.empty(m, np.int32); lab = np.empty(m, np.int32)
    _check(_lib().rpqgen_chung_lu(n, m, gamma, n_labels, zipf_s, seed,
                                  _p(src), _p(dst), _p(lab)), "rpqgen_chung_lu")
    return Graph(f"kb_n{n}_m{m}_L{n_labels}_s{seed}", n, n_labels, src, dst, lab)


def tiny_graph(seed: int, max_n: int = 8, max_m: int = 16, max_labels: int = 3) -> Graph:
    """Random tiny multigraph for exhaustive checks: 1..max_n vertices,
    0..max_m edges (duplicates and self-loops allowed), 1..max_labels labels."""
    r = below(seed, 7, 4, 1 << 30)
    n = 1 + int(r[0] % max_n)
    L = 1 + int(r[1] % max_labels)
    m = int(r[2] % (max_m + 1))
    x = below(seed, 8, 3 * max(m, 1), 1 << 30)
    src = (x[0::3][:m] % n).astype(np.int32)
    dst = (x[1::3][:m] % n).astype(np.int32)
    lab = (x[2::3][:m] % L).astype(np.int32)
    return Graph(f"tiny_s{seed}", n, L, src, dst, lab)


def tiny_automaton(seed: int, n_labels: int, max_states: int = 4, max_trans: int = 8):
    """Random transition-labelled automaton (section 2, 2-NFA) as plain lists:
    (n_states, transitions [(q, a, q')], starts, finals), a in [0, 2L)."""
    r = below(seed, 9, 4, 1 << 30)
    S = 1 + int(r[0] % max_states)
    T = int(r[1] % (max_trans + 1))
    x = below(seed, 10, 3 * max(T, 1) + 2 * S, 1 << 30)
    trans = sorted({(int(x[3 * i] % S), int(x[3 * i + 1] % (2 * n_labels)), int(x[3 * i + 2] % S))
                    for i in range(T)})
    sel = x[3 * max(T, 1):]
    starts = sorted({q for q in range(S) if sel[q] % 3 == 0} or {0})
    finals = sorted({q for q in range(S) if sel[S + q] % 2 == 0})
    return S, trans, starts, finals


# --------------------------------------------------------------- queries --

@dataclass
class Query:
    regex: str
    source: int
    template: str = ""
    arrival_s: float = 0.0


@dataclass
class Workload:
    name: str
    graph: Graph
    queries: list = field(default_factory=list)
    notes: str = ""


def _fill(template: str, labels) -> str:
    out = template
    for k, a in enumerate(labels):
        out = out.replace("{%s}" % "abcdefghijklmnop"[k], str(int(a)))
    return out


def _template_labels(template: str) -> int:
    return sum(1 for ch in "abcdefghijklmnop" if "{%s}" % ch in template)


def _draw_distinct_labels(k: int, L: int, s: float, seed: int, stream: int, count: int):
    """`count` tuples of k distinct labels, each drawn with Zipf(s) weights
    (labels are drawn by edge frequency)."""
    pool = zipf(L, s, seed, stream, count * k * 64 + 64)
    out, i = [], 0
    for _ in range(count):
        chosen = []
        while len(chosen) < k:
            a = int(pool[i]); i += 1
            if a not in chosen or k > L:
                chosen.append(a)
        out.append(chosen)
    return out


def _sources_with_degree(g: Graph, seed: int, stream: int, count: int):
    deg = np.bincount(g.src, minlength=g.n) + np.bincount(g.dst, minlength=g.n)
    cand = np.flatnonzero(deg > 0)
    if cand.size == 0:
        cand = np.arange(g.n)
    idx = below(seed, stream, count, cand.size)
    return cand[idx].astype(np.int64)


def make_queries(g: Graph, templates, per_template: int, seed: int, zipf_s: float,
                 stream_base: int = 100):
    qs = []
    for t_i, tpl in enumerate(templates):
        k = _template_labels(tpl)
        labs = _draw_distinct_labels(k, g.n_labels, zipf_s, seed, stream_base + 2 * t_i,
                                     per_template)
        srcs = _sources_with_degree(g, seed, stream_base + 2 * t_i + 1, per_template)
        for j in range(per_template):
            qs.append(Query(_fill(tpl, labs[j]), int(srcs[j]), tpl))
    return qs


# Query templates.  {a}, {b}, ... are distinct labels; ^x is the inverse.
TEMPLATES_SMALL = ["{a}*", "{a}/{b}*", "({a}|{b})*/{c}", "^{a}/{b}*"]
TEMPLATES_KB = ["{a}/{b}*/{c}", "({a}|^{b})+", "{a}*/{b}*",
                "{a}/{b}/{c}*", "{a}/{b}/{c}/{d}*", "{a}/{b}/{c}/{d}/{e}/{f}*",
                "({a}/{b})*", "{a}/({b}|^{c})*/{d}"]
TEMPLATES_MIXED = TEMPLATES_SMALL + [
    "({a}/{b})*", "{a}/{b}/({c}|{d})*", "{a}/{b}/{c}/({d}|{e})*",
    "{a}/{b}/{c}/{d}/{e}/({f}|{g})*", "{a}/{b}/{c}/{d}/{e}/{f}/{g}/{h}/({i}|{j})*",
    "{a}/{b}/{c}/{d}/{e}/{f}/{g}/{h}/{i}/{j}/{k}/({l}|{m})*", "({a}/{b}/{c})*",
    "{a}/({b}|^{c})*/{d}",
]


def config1() -> Workload:
    """Tiny ER graph: 1,000 vertices, 5,000 distinct edges, 3 uniform labels,
    seed 0; one query 0/1* (a.b*) from vertex 0."""
    g = er_graph(1000, 5000, 3, seed=0)
    return Workload("er1k", g, [Query("0/1*", 0, "{a}/{b}*")],
                    "ER G(n,M) n=1000 M=5000 L=3 uniform labels, seed 0")


def config2_graph() -> Graph:
    """R-MAT scale 20 (2^24 samples, a=0.57 b=c=0.19), 8 labels Zipf(1.0),
    random vertex relabelling, seed 1."""
    return rmat_graph(20, 1 << 24, 8, seed=1)


def config2(per_template: int = 100) -> Workload:
    g = config2_graph()
    qs = make_queries(g, TEMPLATES_SMALL, per_template, seed=1, zipf_s=1.0)
    return Workload("rmat20", g, qs,
                    "R-MAT scale 20, 2^24 samples, 8 labels Zipf(1.0), seed 1; "
                    f"templates {TEMPLATES_SMALL}, {per_template} sources each")


def config3_graph(n: int = 20_000_000, m: int = 200_000_000) -> Graph:
    """Knowledge-base-shaped graph: Chung-Lu power law (out-degree exponent
    2.1, destinations skewed under an independent permutation), 500 labels
    Zipf(1.1), seed 2."""
    return chung_lu_graph(n, m, 2.1, 500, 1.1, seed=2)


def config3(per_template: int = 100, n: int = 20_000_000, m: int = 200_000_000) -> Workload:
    g = config3_graph(n, m)
    qs = make_queries(g, TEMPLATES_KB, per_template, seed=2, zipf_s=1.1)
    return Workload("kb20m", g, qs,
                    f"Chung-Lu n={n} m={m} gamma=2.1, 500 labels Zipf(1.1), seed 2; "
                    f"templates {TEMPLATES_KB}")


def config4(g: Graph | None = None, n_queries: int = 256) -> Workload:
    g = g or config2_graph()
    per = -(-n_queries // len(TEMPLATES_MIXED))
    qs = make_queries(g, TEMPLATES_MIXED, per, seed=3, zipf_s=1.0, stream_base=300)
    # interleave templates, then cut to n_queries
    order = below(3, 299, len(qs), 1 << 62)
    qs = [q for _, q in sorted(zip(order.tolist(), qs), key=lambda t: t[0])][:n_queries]
    return Workload("rmat20_batch", g, qs, f"{n_queries} mixed queries, seed 3")


def config5(g: Graph | None = None, rate: float = 2000.0, duration_s: float = 10.0,
            warmup_s: float = 1.0) -> Workload:
    g = g or config2_graph()
    n_expect = int((duration_s + warmup_s) * rate * 1.2) + 64
    gaps = exponential(rate, 4, 400, n_expect)
    t = np.cumsum(gaps)
    n = int(np.searchsorted(t, duration_s + warmup_s))
    per = -(-n // len(TEMPLATES_MIXED))
    qs = make_queries(g, TEMPLATES_MIXED, per, seed=4, zipf_s=1.0, stream_base=500)
    order = below(4, 499, len(qs), 1 << 62)
    qs = [q for _, q in sorted(zip(order.tolist(), qs), key=lambda t: t[0])][:n]
    for q, ti in zip(qs, t[:n]):
        q.arrival_s = float(ti)
    return Workload("rmat20_serve", g, qs,
                    f"Poisson arrivals rate {rate}/s for {duration_s}s after {warmup_s}s warm-up, seed 4")


# ------------------------------------------------------- random queries --

_SYM_FWD = "abcdefgh"
_SYM_INV = "ABCDEFGH"


class _Draws:
    def __init__(self, seed: int, stream: int):
        self.buf = below(seed, stream, 4096, 1 << 30)
        self.i = 0

    def __call__(self, k: int) -> int:
        v = int(self.buf[self.i % self.buf.size]) % k
        self.i += 1
        return v


def random_regex(seed: int, n_labels: int, depth: int = 3):
    """A random regular expression over labels [0, n_labels) (n_labels <= 8)
    and their inverses, rendered twice: in the query syntax
    (``rpq_text``) and as a Python ``re`` pattern over one character per
    symbol (label a -> 'a'+a, a^- -> 'A'+a), with the inverse operator ``^``
    expanded (reverse the word, invert each symbol).  Returns
    (rpq_text, re_pattern, symbol_chars) where symbol_chars[s] is the
    character of symbol s in [0, 2L)."""
    if not 1 <= n_labels <= 8:
        raise ValueError("n_labels must be in [1, 8]")
    d = _Draws(seed, 11)

    def gen(k):
        # node: ('sym', a) | ('cat', x, y) | ('alt', x, y) | ('star'|'plus'|'opt', x) | ('inv', x)
        r = d(10) if k > 0 else 0
        if r <= 2:
            a = d(2 * n_labels)
            return ("sym", a)
        if r <= 4:
            return ("cat", gen(k - 1), gen(k - 1))
        if r == 5:
            return ("alt", gen(k - 1), gen(k - 1))
        if r == 6:
            return ("star", gen(k - 1))
        if r == 7:
            return ("plus", gen(k - 1))
        if r == 8:
            return ("opt", gen(k - 1))
        return ("inv", gen(k - 1))

    def rpq(t):
        k = t[0]
        if k == "sym":
            a = t[1]
            return str(a) if a < n_labels else "^" + str(a - n_labels)
        if k == "cat":
            return "(" + rpq(t[1]) + "/" + rpq(t[2]) + ")"
        if k == "alt":
            return "(" + rpq(t[1]) + "|" + rpq(t[2]) + ")"
        if k in ("star", "plus", "opt"):
            return "(" + rpq(t[1]) + ")" + {"star": "*", "plus": "+", "opt": "?"}[k]
        return "^(" + rpq(t[1]) + ")"

    def pyre(t, inv=False):
        k = t[0]
        if k == "sym":
            a = t[1]
            fwd = a < n_labels
            if inv:
                fwd = not fwd
            return (_SYM_FWD if fwd else _SYM_INV)[a % n_labels]
        if k == "cat":
            x, y = (t[2], t[1]) if inv else (t[1], t[2])
            return "(?:" + pyre(x, inv) + pyre(y, inv) + ")"
        if k == "alt":
            return "(?:" + pyre(t[1], inv) + "|" + pyre(t[2], inv) + ")"
        if k in ("star", "plus", "opt"):
            return "(?:" + pyre(t[1], inv) + ")" + {"star": "*", "plus": "+", "opt": "?"}[k]
        return pyre(t[1], not inv)

    tree = gen(depth)
    chars = [_SYM_FWD[a] for a in range(n_labels)] + [_SYM_INV[a] for a in range(n_labels)]
    return rpq(tree), pyre(tree), chars
