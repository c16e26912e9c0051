"""Serving (continuous batching) against the CPU oracle.

Queries submitted while others are in flight join at the next level step;
each answer must equal the oracle's, and must be the same whether the query
ran alone or in the mix."""

import time

import numpy as np
import pytest

from oracle import oracle as O
from oracle.regex_nfa import Nfa, compile_regex as oracle_compile
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


@pytest.fixture(scope="module")
def setup():
    g = W.rmat_graph(13, 60000, 4, seed=71)
    gg = R.rpq_graph_load(g.n, g.n_labels, g.src, g.dst, g.lab)
    og = O.OracleGraph(g.n, g.n_labels, g.src, g.dst, g.lab)
    return g, gg, og


TEXTS = ["0*", "1/0*", "(0|1)*/2", "^0/1*", "(0/1)*", "0/1/(2|3)*", "(^0|1)+", "3", "2/^2",
         "0/1/2/3/(0|1)*", "(0/1/2)*"]


def run_server(srv, jobs, stagger_s=0.0):
    tickets = []
    for nfa, s in jobs:
        tickets.append(srv.submit(nfa, s))
        if stagger_s:
            time.sleep(stagger_s)
    srv.drain(120000)
    return [srv.poll(t) for t in tickets]


ENGINES = [(0, 8), (1, 64)]  # (engine, slots or lanes)
ENGINE_IDS = ["slots", "lanes"]


@pytest.mark.parametrize("engine,width", ENGINES, ids=ENGINE_IDS)
def test_serve_mixed_and_staggered(setup, engine, width):
    g, gg, og = setup
    srcs = W.below(72, 1, 180, g.n).tolist()
    jobs = [(R.rpq_nfa_compile(TEXTS[i % len(TEXTS)], 4), srcs[i]) for i in range(180)]
    exp = [og.ssr(oracle_compile(TEXTS[i % len(TEXTS)], 4), srcs[i])["answer"].tolist()
           for i in range(180)]
    srv = R.Server(gg, max_lanes=width, max_states=16, engine=engine)
    try:
        got = run_server(srv, jobs)  # 180 queries, fewer slots/lanes: admitted as they free up
        assert [a.tolist() for a in got] == exp
        got = run_server(srv, jobs[:60], stagger_s=0.0005)  # joining mid-flight
        assert [a.tolist() for a in got] == exp[:60]
        st = srv.stats()
        assert st["completed"] == 240 and st["p99_ms"] >= st["p50_ms"]
    finally:
        srv.close()


@pytest.mark.parametrize("engine,width", ENGINES, ids=ENGINE_IDS)
def test_serve_alone_equals_in_mix(setup, engine, width):
    g, gg, og = setup
    srcs = W.below(73, 1, 40, g.n).tolist()
    jobs = [(R.rpq_nfa_compile(TEXTS[(3 * i) % len(TEXTS)], 4), srcs[i]) for i in range(40)]
    srv = R.Server(gg, max_lanes=width, max_states=16, engine=engine)
    try:
        mix = run_server(srv, jobs)
        alone = [run_server(srv, [j])[0] for j in jobs[:12]]
        for a, b in zip(alone, mix[:12]):
            assert a.tolist() == b.tolist()
        single = [R.rpq_query(gg, nfa, s) for nfa, s in jobs[:12]]
        for a, b in zip(single, mix[:12]):
            assert a.tolist() == b.tolist()
    finally:
        srv.close()


@pytest.mark.parametrize("engine,width", ENGINES, ids=ENGINE_IDS)
def test_serve_transition_automata_and_level_cap(setup, engine, width):
    g, gg, og = setup
    autos = [W.tiny_automaton(800 + i, 4, max_states=6, max_trans=12) for i in range(50)]
    srcs = W.below(74, 1, 50, g.n).tolist()
    for cap in (2, 0):
        srv = R.Server(gg, max_lanes=width, max_states=8, max_levels=cap, engine=engine)
        try:
            jobs = [(R.rpq_nfa_from_transitions(S, 4, tr, st, fi), srcs[i])
                    for i, (S, tr, st, fi) in enumerate(autos)]
            got = run_server(srv, jobs)
            for i, (S, tr, st, fi) in enumerate(autos):
                exp = og.ssr(Nfa(S, 4, tr, st, fi), srcs[i], cap)["answer"]
                assert got[i].tolist() == exp.tolist(), (i, cap)
        finally:
            srv.close()


@pytest.mark.parametrize("engine,width", ENGINES, ids=ENGINE_IDS)
def test_serve_queue_limit_and_errors(setup, engine, width):
    g, gg, og = setup
    srv = R.Server(gg, max_lanes=width, max_states=16, queue_capacity=4, engine=engine)
    try:
        nfa = R.rpq_nfa_compile("(0|1|2|3)*", 4)
        accepted, busy = [], 0
        srcs = W.below(75, 1, 400, g.n).tolist()
        for s in srcs:
            try:
                accepted.append((srv.submit(nfa, s), s))
            except R.RpqError as e:
                assert e.status == R.RPQ_ERR_BUSY
                busy += 1
        srv.drain(120000)
        on = oracle_compile("(0|1|2|3)*", 4)
        for t, s in accepted[:40]:
            assert srv.poll(t).tolist() == og.ssr(on, s)["answer"].tolist()
        assert srv.stats()["rejected"] == busy
        with pytest.raises(R.RpqError):
            srv.submit(nfa, g.n)  # source out of range
        if engine == 1:
            with pytest.raises(R.RpqError):
                srv.submit(R.rpq_nfa_compile("/".join(["0"] * 20), 4), 0)  # 21 states > 16 slots
        with pytest.raises(R.RpqError):
            srv.poll(10 ** 9)  # unknown ticket
    finally:
        srv.close()


@pytest.mark.parametrize("engine,width", ENGINES, ids=ENGINE_IDS)
def test_serve_memory_bounded_admission(setup, engine, width):
    """A small memory budget admits fewer queries at once (the device state
    of the admitted queries stays within it) and gives the same answers; a
    query that could never fit is refused at submission."""
    g, gg, og = setup
    srcs = W.below(76, 1, 96, g.n).tolist()
    texts = ["0*", "1/0*", "(0|1)*/2", "^0/1*"]  # DFAs of 1-2 states
    jobs = [(R.rpq_nfa_compile(texts[i % 4], 4), srcs[i]) for i in range(96)]
    exp = [og.ssr(oracle_compile(texts[i % 4], 4), srcs[i])["answer"].tolist() for i in range(96)]
    W64 = (g.n + 63) // 64
    per_query = (4 * 4 * W64 * 8 + 4 * g.n * 4) if engine == 0 else 4 * 2 * ((g.n + 7) // 8)
    free = R.Server(gg, max_lanes=width, max_states=16, engine=engine)
    tight = R.Server(gg, max_lanes=width, max_states=16, engine=engine,
                     memory_budget=2 * per_query)
    try:
        got_free = run_server(free, jobs)
        got_tight = run_server(tight, jobs)
        assert [a.tolist() for a in got_free] == exp
        assert [a.tolist() for a in got_tight] == exp
        st_f, st_t = free.stats(), tight.stats()
        assert st_t["peak_in_flight"] <= 2 and st_t["peak_bytes"] <= 2 * per_query
        assert st_f["peak_in_flight"] > 2  # without the budget more run at once
        big = R.rpq_nfa_compile("/".join(["0"] * 12), 4)  # 13 states: more than the budget
        with pytest.raises(R.RpqError) as e:
            tight.submit(big, srcs[0])
        assert e.value.status == R.RPQ_ERR_OOM
    finally:
        free.close()
        tight.close()
