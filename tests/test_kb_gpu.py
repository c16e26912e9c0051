"""Knowledge-base-shaped graphs (power-law degrees, 500 Zipf(1.1) labels,
most of them hypersparse): GPU answers against the CPU oracle, at a scaled
size and, in a slow test, at the full 20M-vertex / 200M-edge size."""

import numpy as np
import pytest

from oracle import oracle as O
from oracle.regex_nfa import compile_regex as oracle_compile
from paper_2412_10287_gb300 import rpq as R
from paper_2412_10287_gb300 import workloads as W

from conftest import gpu_available

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2412_10287_gb300 import build as B

    B.build()


def test_kb_scaled_parity():
    g = W.chung_lu_graph(1_000_000, 10_000_000, 2.1, 500, 1.1, seed=2)
    qs = W.make_queries(g, W.TEMPLATES_KB, 3, seed=2, zipf_s=1.1)
    gg = R.rpq_graph_load(g.n, g.n_labels, g.src, g.dst, g.lab)
    og = O.OracleGraph(g.n, g.n_labels, g.src, g.dst, g.lab)
    nonempty = 0
    for q in qs:
        exp = og.ssr(oracle_compile(q.regex, g.n_labels), q.source)["answer"]
        got = R.rpq_query(gg, R.rpq_nfa_compile(q.regex, g.n_labels), q.source)
        assert got.tolist() == exp.tolist(), q
        nonempty += exp.size > 1
    assert nonempty >= 3  # the sample exercises real traversals


@pytest.mark.slow
def test_kb20m_full_size():
    """Full size (20M vertices, 200M edges, 500 labels): the first query of
    every benchmark template -- inverse labels included -- against the
    oracle, and properties that hold at any size (P_k grows with k; union of
    languages = union of answers)."""
    import concurrent.futures as cf
    import os

    w = W.config3(per_template=1)
    g = w.graph
    assert sorted({q.template for q in w.queries}) == sorted(W.TEMPLATES_KB)
    gg = R.rpq_graph_load(g.n, g.n_labels, g.src, g.dst, g.lab)
    og = O.OracleGraph(g.n, g.n_labels, g.src, g.dst, g.lab)

    def oracle_answer(q):
        return og.ssr(oracle_compile(q.regex, g.n_labels), q.source)["answer"]

    with cf.ThreadPoolExecutor(max_workers=len(os.sched_getaffinity(0))) as ex:
        exp = list(ex.map(oracle_answer, w.queries))
    og.close()
    assert any(q.template.count("^") for q in w.queries)
    for q, e in zip(w.queries, exp):
        got = R.rpq_query(gg, R.rpq_nfa_compile(q.regex, g.n_labels), q.source)
        assert got.tolist() == e.tolist(), q
    for q in w.queries[:4]:
        nfa = R.rpq_nfa_compile(q.regex, g.n_labels)
        prev = set()
        for k in (1, 2, 4, 0):
            cur = set(R.rpq_query(gg, nfa, q.source, k).tolist())
            assert prev <= cur
            prev = cur
    a, b = w.queries[0], w.queries[1]
    s = a.source
    ua = set(R.rpq_query(gg, R.rpq_nfa_compile(a.regex, g.n_labels), s).tolist())
    ub = set(R.rpq_query(gg, R.rpq_nfa_compile(b.regex, g.n_labels), s).tolist())
    uab = set(R.rpq_query(gg, R.rpq_nfa_compile(f"({a.regex})|({b.regex})", g.n_labels), s).tolist())
    assert uab == ua | ub
