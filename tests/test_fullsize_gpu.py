"""Parity at the full sizes the benchmark runs, against the CPU oracle.

The R-MAT scale-20 graph (2^24 edge samples, 8 labels) carries three of the
workloads: single queries one at a time, 256 mixed queries per batch call,
and a Poisson stream through the server.  Here every answer of the batch
(both engines) and of the first 512 served queries (both server engines,
arrivals paced as in the stream) is compared element by element with the
oracle's, on the same graph and queries the benchmark uses.  Answers are
sets: parity is exact equality of the sorted vertex lists.
"""

import concurrent.futures as cf
import os
import time

import pytest

from oracle import oracle as O
from oracle.regex_nfa import compile_regex as oracle_compile
from paper_2412_10287_gb300 import rpq as R
from paper_2412_10287_gb300 import workloads as W

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2412_10287_gb300 import build as B

    B.build()


def oracle_answers(og, L, jobs):
    """Oracle answers of (regex, source) jobs, on every host core (the oracle
    releases the interpreter lock while it runs)."""
    cache = {}

    def one(job):
        text, s = job
        nfa = cache.get(text) or oracle_compile(text, L)
        cache[text] = nfa
        return og.ssr(nfa, s)["answer"].tolist()

    with cf.ThreadPoolExecutor(max_workers=len(os.sched_getaffinity(0))) as ex:
        return list(ex.map(one, jobs))


@pytest.fixture(scope="module")
def rmat20():
    g = W.config2_graph()
    gg = R.rpq_graph_load(g.n, g.n_labels, g.src, g.dst, g.lab)
    og = O.OracleGraph(g.n, g.n_labels, g.src, g.dst, g.lab)
    yield g, gg, og
    og.close()
    gg.close()


def test_config2_graph_build_matches_definition(rmat20):
    """The device CSR and CSC of every label of the R-MAT scale-20 graph
    equal the definition: distinct (u, v, a) triples, rows sorted."""
    import numpy as np

    g, gg, _ = rmat20
    trip = np.unique(np.stack([g.lab, g.src, g.dst], 1).astype(np.int64), axis=0)
    assert gg.n_edges() == trip.shape[0]
    for a in range(g.n_labels):
        t = trip[trip[:, 0] == a]
        off, nbr = R.rpq_graph_export(gg, a, False)
        exp_off = np.zeros(g.n + 1, np.int64)
        np.add.at(exp_off, t[:, 1] + 1, 1)
        assert (off == np.cumsum(exp_off)).all() and (nbr == t[:, 2]).all(), a
        tt = t[np.lexsort((t[:, 1], t[:, 2]))]
        off, nbr = R.rpq_graph_export(gg, a, True)
        exp_off = np.zeros(g.n + 1, np.int64)
        np.add.at(exp_off, tt[:, 2] + 1, 1)
        assert (off == np.cumsum(exp_off)).all() and (nbr == tt[:, 1]).all(), a


@pytest.fixture(scope="module")
def batch_case(rmat20):
    g, gg, og = rmat20
    w = W.config4(g, 256)
    exp = oracle_answers(og, g.n_labels, [(q.regex, q.source) for q in w.queries])
    return w, exp


@pytest.mark.parametrize("engine", ["slots", "lanes"])
def test_config4_batch_every_answer(rmat20, batch_case, engine, monkeypatch):
    """256 mixed queries of 2-12 DFA states in one rpq_query_batch call, on
    each engine, three calls in a row: every answer equals the oracle's."""
    g, gg, _ = rmat20
    w, exp = batch_case
    monkeypatch.setenv("RPQ_BATCH_ENGINE", engine)
    nfas = [R.rpq_nfa_compile(q.regex, g.n_labels) for q in w.queries]
    bad = []
    for rep in range(3):
        got = R.rpq_query_batch(gg, nfas, [q.source for q in w.queries])
        assert len(got) == 256
        for i, q in enumerate(w.queries):
            if got[i].tolist() != exp[i]:
                bad.append((rep, i, q.regex, q.source, len(exp[i]) - got[i].size))
    assert not bad, (engine, bad)


@pytest.mark.parametrize("engine,width", [(0, 12), (1, 256)], ids=["slots", "lanes"])
def test_config5_served_stream_every_answer(rmat20, engine, width):
    """The first 512 queries of the 2,000 queries/s Poisson stream, submitted
    at their arrival times into each server engine: every answer equals the
    oracle's."""
    g, gg, og = rmat20
    qs = W.config5(g, rate=2000.0, duration_s=10.0, warmup_s=1.0).queries[:512]
    exp = oracle_answers(og, g.n_labels, [(q.regex, q.source) for q in qs])
    nfas = {}
    for q in qs:
        nfas.setdefault(q.regex, R.rpq_nfa_compile(q.regex, g.n_labels))
    srv = R.Server(gg, max_lanes=width, max_states=16, engine=engine)
    try:
        t0 = time.perf_counter()
        tickets = []
        for q in qs:
            dt = q.arrival_s - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(nfas[q.regex], q.source))
        srv.drain(300000)
        for i, t in enumerate(tickets):
            assert srv.poll(t).tolist() == exp[i], (i, qs[i].regex, qs[i].source)
        assert srv.stats()["completed"] == len(qs)
    finally:
        srv.close()


def test_config2_bench_queries_sampled(rmat20):
    """Ten queries of each rmat20 benchmark template (the first ten sources
    the benchmark draws), one at a time as the benchmark runs them."""
    g, gg, og = rmat20
    qs = W.config2(per_template=10).queries
    exp = oracle_answers(og, g.n_labels, [(q.regex, q.source) for q in qs])
    for q, e in zip(qs, exp):
        got = R.rpq_query(gg, R.rpq_nfa_compile(q.regex, g.n_labels), q.source)
        assert got.tolist() == e, q
