"""GPU parity of the lane-batched entry point rpq_query_batch against the
CPU oracle: every query of a batch must give exactly the oracle's answer,
whatever the mix of automata and sources sharing the launch."""

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


def load(g):
    return R.rpq_graph_load(g.n, g.n_labels, g.src, g.dst, g.lab)


@pytest.fixture(params=["slots", "lanes", "lanes_pull"], autouse=True)
def engine(request, monkeypatch):
    """Every batch test runs on both engines: concurrent query slots and bit
    lanes -- the latter also with every level pulling and the shortest
    inline rows (the other ends of the lane engine's tuning range)."""
    monkeypatch.setenv("RPQ_BATCH_ENGINE", "slots" if request.param == "slots" else "lanes")
    if request.param == "lanes_pull":
        monkeypatch.setenv("RPQ_LANE_PULL_DIV", "1000000000")
        monkeypatch.setenv("RPQ_LANE_HUB", "32")
    yield request.param


def test_batch_shared_automaton_many_sources():
    """One automaton from many sources (multi-source BFS): every answer equals the oracle's."""
    g = W.rmat_graph(14, 1 << 18, 4, seed=35)
    gg = load(g)
    og = O.OracleGraph(g.n, 4, g.src, g.dst, g.lab)
    srcs = W.below(36, 1, 200, g.n).tolist()
    nfa = R.rpq_nfa_compile("(0|^1)*/2", 4)
    got = R.rpq_query_batch(gg, [nfa] * 200, srcs)
    on = oracle_compile("(0|^1)*/2", 4)
    for i in range(200):
        assert got[i].tolist() == og.ssr(on, srcs[i])["answer"].tolist(), i


def test_batch_tiny_mixed():
    for seed in range(12):
        g = W.tiny_graph(seed + 3000, max_n=16, max_m=40)
        L = g.n_labels
        gg = load(g)
        og = O.OracleGraph(g.n, L, g.src, g.dst, g.lab)
        texts = [W.random_regex(seed * 100 + i, L, 1 + i % 4)[0] for i in range(40)]
        nfas, srcs, exp = [], [], []
        for i, t in enumerate(texts):
            for s in range(0, g.n, max(1, g.n // 3)):
                nfas.append(R.rpq_nfa_compile(t, L))
                srcs.append(s)
                exp.append(og.ssr(oracle_compile(t, L), s)["answer"].tolist())
        got = R.rpq_query_batch(gg, nfas, srcs)
        for i in range(len(exp)):
            assert got[i].tolist() == exp[i], (seed, texts[i // max(1, len(srcs) // len(texts))])


def test_batch_more_than_one_lane_group_and_levels():
    g = W.rmat_graph(12, 30000, 4, seed=31)
    gg = load(g)
    og = O.OracleGraph(g.n, 4, g.src, g.dst, g.lab)
    texts = ["0*", "1/0*", "(0|1)*/2", "^0/1*", "(0/1)*", "0/1/(2|3)*", "(^0|1)+", "3"]
    srcs = W.below(32, 1, 300, g.n).tolist()
    nfas = [R.rpq_nfa_compile(texts[i % len(texts)], 4) for i in range(300)]
    for k in (0, 1, 3):
        got = R.rpq_query_batch(gg, nfas, srcs, max_levels=k)
        for i in range(300):
            exp = og.ssr(oracle_compile(texts[i % len(texts)], 4), srcs[i], k)["answer"]
            assert got[i].tolist() == exp.tolist(), (i, k)


def test_batch_transition_automata_with_hubs():
    """Automata given as transitions (NFAs, several starts) on a graph with a
    20k-edge hub row (split into chunks across warps)."""
    n = 40_000
    rng = W.below(41, 1, 120_000, 1 << 30)
    src = np.concatenate([np.zeros(20_000, np.int32), (rng[:30_000] % n).astype(np.int32)])
    dst = np.concatenate([np.arange(1, 20_001, dtype=np.int32), (rng[30_000:60_000] % n).astype(np.int32)])
    lab = np.concatenate([np.zeros(20_000, np.int32), (rng[60_000:90_000] % 3).astype(np.int32)])
    g = W.Graph("hub", n, 3, src, dst, lab)
    gg = load(g)
    og = O.OracleGraph(n, 3, src, dst, lab)
    autos = [W.tiny_automaton(500 + i, 3, max_states=5, max_trans=10) for i in range(64)]
    srcs = [0 if i % 3 == 0 else int(rng[90_000 + i] % n) for i in range(64)]
    dn = [R.rpq_nfa_from_transitions(S, 3, tr, st, fi) for S, tr, st, fi in autos]
    got = R.rpq_query_batch(gg, dn, srcs)
    for i, (S, tr, st, fi) in enumerate(autos):
        exp = og.ssr(Nfa(S, 3, tr, st, fi), srcs[i])["answer"]
        assert got[i].tolist() == exp.tolist(), i


def test_batch_errors_and_capacity():
    import ctypes

    g = W.config1().graph
    gg = load(g)
    nfas = [R.rpq_nfa_compile("0/1*", 3), R.rpq_nfa_compile("(0|1|2)*", 3)]
    with pytest.raises(R.RpqError):
        R.rpq_query_batch(gg, nfas, [0, 5000])
    handles = (ctypes.c_void_p * 2)(nfas[0].h.value, nfas[1].h.value)
    srcs = np.array([0, 1], np.int32)
    offs = np.zeros(3, np.int64)
    buf = np.zeros(8, np.int32)
    s = R.lib().rpq_query_batch(gg.h, 2, handles, R._ptr(srcs), 0, R._ptr(offs), R._ptr(buf), 8,
                                None, None)
    assert s == R.RPQ_ERR_CAPACITY and offs[2] > 8
    one = R.rpq_query(gg, nfas[0], 0)
    assert offs[1] - offs[0] == one.size
    assert R.rpq_query_batch(gg, [], []) == []


@pytest.mark.parametrize("cap", [0, 64], ids=["buffer_0", "buffer_64"])
def test_batch_with_discovery_buffer_overflow(cap, monkeypatch):
    """Concurrent query kernels (slots engine) whose CTAs' discovery buffers
    overflow on most levels, so that the levels are measured again from the
    visited lists while other queries run beside them: every answer equals
    the oracle's."""
    monkeypatch.setenv("RPQ_DISCOVERY_BUFFER", str(cap))
    g = W.rmat_graph(14, 1 << 18, 4, seed=37)
    gg = load(g)
    og = O.OracleGraph(g.n, 4, g.src, g.dst, g.lab)
    texts = ["0*", "(0|^1)*/2", "1/(0|2)*", "(0/1)*", "^3/(1|2)+", "2/^2"]
    srcs = W.below(38, 1, 96, g.n).tolist()
    nfas = [R.rpq_nfa_compile(texts[i % len(texts)], 4) for i in range(96)]
    got = R.rpq_query_batch(gg, nfas, srcs)
    for i in range(96):
        exp = og.ssr(oracle_compile(texts[i % len(texts)], 4), srcs[i])["answer"]
        assert got[i].tolist() == exp.tolist(), i


def test_fresh_workspaces_on_reused_memory(engine):
    """Device memory freed by an earlier graph comes back, with its old
    contents, as the workspaces of a new graph; those are first used on the
    slot engine's non-blocking streams.  Their clears must be ordered before
    that use: every answer equals the oracle's."""
    junk = W.rmat_graph(18, 1 << 22, 4, seed=43)  # ~50 MB of non-zero ids, then freed
    jg = load(junk)
    del jg
    import gc

    gc.collect()
    g = W.rmat_graph(15, 1 << 19, 4, seed=44)
    gg = load(g)
    og = O.OracleGraph(g.n, 4, g.src, g.dst, g.lab)
    texts = ["0*", "(0|^1)*/2", "1/(0|2)*", "(0/1)*", "^3/(1|2)+", "(0|1|2|3)*"]
    srcs = W.below(45, 1, 48, g.n).tolist()
    nfas = [R.rpq_nfa_compile(texts[i % len(texts)], 4) for i in range(48)]
    got = R.rpq_query_batch(gg, nfas, srcs)
    for i in range(48):
        exp = og.ssr(oracle_compile(texts[i % len(texts)], 4), srcs[i])["answer"]
        assert got[i].tolist() == exp.tolist(), i


def test_lane_autotune_keeps_answers(engine):
    """The lane engine's autotuner picks an inline row length and a pull
    divisor from its candidate sets; the answers do not change."""
    if engine != "lanes":
        pytest.skip("one run is enough")
    g = W.rmat_graph(13, 1 << 17, 4, seed=47)
    gg = load(g)
    og = O.OracleGraph(g.n, 4, g.src, g.dst, g.lab)
    srcs = W.below(48, 1, 64, g.n).tolist()
    nfa = R.rpq_nfa_compile("(0|^1)*/2", 4)
    hub, pdv = R.rpq_graph_autotune_batch(gg, [nfa] * 64, srcs)
    assert hub in (32, 64, 128, 256) and pdv in (0, 2, 4, 8, 16)
    got = R.rpq_query_batch(gg, [nfa] * 64, srcs)
    on = oracle_compile("(0|^1)*/2", 4)
    for i in range(64):
        assert got[i].tolist() == og.ssr(on, srcs[i])["answer"].tolist(), i
