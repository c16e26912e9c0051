"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Answers are sets, so parity is bit-exact set equality (no tolerance).  For
automata given as transition lists (the same automaton on both sides) the
per-query counters of Algorithm 1 -- levels, visited pairs, expanded pairs,
product edges, push-model bytes -- must match exactly as well.
"""

import os

import numpy as np
import pytest

from oracle import oracle as O
from oracle.regex_nfa import Nfa, compile_regex as oracle_compile
from paper_2412_10287_gb300 import rpq as R
from paper_2412_10287_gb300 import workloads as W

from conftest import gpu_available

pytestmark = pytest.mark.gpu

COUNTERS = ("levels", "visited", "expanded", "product_edges", "push_bytes", "answer")
STAT_OF = {"levels": "levels", "visited": "visited_pairs", "expanded": "expanded_pairs",
           "product_edges": "product_edges", "push_bytes": "push_bytes", "answer": "answer_count"}


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2412_10287_gb300 import build as B

    B.build()


def load(g):
    return R.rpq_graph_load(g.n, g.n_labels, g.src, g.dst, g.lab)


def gpu_regex(gg, text, L, source, k=0, stats=False):
    nfa = R.rpq_nfa_compile(text, L)
    return R.rpq_query(gg, nfa, source, k, with_stats=stats)


def check_counters(st, oc):
    for k in COUNTERS:
        assert st[STAT_OF[k]] == oc[k], (k, st, oc)


@pytest.fixture
def pull_mode(request):
    """Force a direction policy through the environment (read per query)."""
    old = {k: os.environ.get(k) for k in ("RPQ_PULL_ALPHA", "RPQ_PULL_MIN")}
    alpha, mn = request.param
    os.environ["RPQ_PULL_ALPHA"] = str(alpha)
    os.environ["RPQ_PULL_MIN"] = str(mn)
    yield request.param
    for k, v in old.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v


MODES = [(0.0, 1 << 30), (1e9, 0), (4.0, 256)]  # push only, pull whenever possible, default
MODE_IDS = ["push", "pull", "auto"]


# ------------------------------------------------------------ graph build --

def test_graph_build_matches_definition():
    g = W.rmat_graph(12, 40000, 5, seed=11)
    gg = load(g)
    trip = np.unique(np.stack([g.lab, g.src, g.dst], 1).astype(np.int64), axis=0)
    assert gg.n_edges() == trip.shape[0]
    for a in range(g.n_labels):
        t = trip[trip[:, 0] == a]
        assert gg.n_edges(a) == t.shape[0]
        off, nbr = R.rpq_graph_export(gg, a, False)
        exp_off = np.zeros(g.n + 1, np.int64)
        np.add.at(exp_off, t[:, 1] + 1, 1)
        assert (off == np.cumsum(exp_off)).all()
        assert (nbr == t[:, 2]).all()  # rows by source, sorted destinations
        tt = t[np.lexsort((t[:, 1], t[:, 2]))]
        off, nbr = R.rpq_graph_export(gg, a, True)
        exp_off = np.zeros(g.n + 1, np.int64)
        np.add.at(exp_off, tt[:, 2] + 1, 1)
        assert (off == np.cumsum(exp_off)).all()
        assert (nbr == tt[:, 1]).all()


def test_graph_build_hypersparse_labels():
    # many labels on a larger vertex set: most labels become hypersparse
    g = W.chung_lu_graph(200_000, 300_000, 2.1, 60, 1.1, seed=5)
    gg = load(g)
    trip = np.unique(np.stack([g.lab, g.src, g.dst], 1).astype(np.int64), axis=0)
    for a in (0, 7, 33, 59):
        t = trip[trip[:, 0] == a]
        off, nbr = R.rpq_graph_export(gg, a, False)
        exp = np.zeros(g.n + 1, np.int64)
        np.add.at(exp, t[:, 1] + 1, 1)
        assert (off == np.cumsum(exp)).all() and (nbr == t[:, 2]).all()


def test_graph_load_rejects_bad_ids():
    with pytest.raises(R.RpqError):
        R.rpq_graph_load(4, 2, [0, 1], [1, 4], [0, 0])
    with pytest.raises(R.RpqError):
        R.rpq_graph_load(4, 2, [0, 1], [1, 2], [0, 2])


# ----------------------------------------------------------- tiny graphs --

@pytest.mark.parametrize("pull_mode", MODES, ids=MODE_IDS, indirect=True)
def test_random_tiny_regex(pull_mode):
    for seed in range(120):
        g = W.tiny_graph(seed + 40, max_n=12, max_m=30)
        L = g.n_labels
        text, _, _ = W.random_regex(seed + 41, L, 1 + seed % 4)
        gg = load(g)
        og = O.OracleGraph(g.n, L, g.src, g.dst, g.lab)
        onfa = oracle_compile(text, L)
        for source in range(g.n):
            for k in (0, 1, 3):
                exp = og.ssr(onfa, source, k)["answer"]
                got = gpu_regex(gg, text, L, source, k)
                assert got.tolist() == exp.tolist(), (seed, text, source, k)


@pytest.mark.parametrize("pull_mode", MODES, ids=MODE_IDS, indirect=True)
def test_random_tiny_automata_counters(pull_mode):
    """Same automaton on both sides: answers and every counter match."""
    for seed in range(150):
        g = W.tiny_graph(seed + 500, max_n=16, max_m=40)
        L = g.n_labels
        S, trans, starts, finals = W.tiny_automaton(seed + 501, L, max_states=6, max_trans=14)
        gg = load(g)
        dn = R.rpq_nfa_from_transitions(S, L, trans, starts, finals)
        on = Nfa(S, L, trans, starts, finals)
        og = O.OracleGraph(g.n, L, g.src, g.dst, g.lab)
        for source in range(0, g.n, max(1, g.n // 4)):
            for k in (0, 2):
                o = og.ssr(on, source, k)
                got, st = R.rpq_query(gg, dn, source, k, with_stats=True)
                assert got.tolist() == o["answer"].tolist(), (seed, source, k)
                check_counters(st, o["counters"])


# ------------------------------------------------- ragged / edge sizes ---

@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 127, 129, 1000, 4097])
def test_ragged_vertex_counts(n):
    g = W.Graph("chain", n, 2, np.arange(n - 1, dtype=np.int32), np.arange(1, n, dtype=np.int32),
                (np.arange(n - 1) % 2).astype(np.int32))
    gg = load(g)
    og = O.OracleGraph(g.n, 2, g.src, g.dst, g.lab)
    for text in ("(0|1)*", "0/1", "(0/1)*", "^(0|1)*", "(0|^1)+"):
        on = oracle_compile(text, 2)
        for source in sorted({0, n // 2, n - 1}):
            assert gpu_regex(gg, text, 2, source).tolist() == og.ssr(on, source)["answer"].tolist()


def test_empty_graph_and_isolated_source():
    g = W.Graph("empty", 100, 3, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))
    gg = load(g)
    assert gpu_regex(gg, "0*", 3, 5).tolist() == [5]
    assert gpu_regex(gg, "0/1", 3, 5).tolist() == []
    g2 = W.config1().graph
    gg2 = load(g2)
    deg = np.bincount(g2.src, minlength=g2.n) + np.bincount(g2.dst, minlength=g2.n)
    iso = int(np.flatnonzero(deg == 0)[0]) if (deg == 0).any() else None
    if iso is not None:
        assert gpu_regex(gg2, "(0|1|2)*", 3, iso).tolist() == [iso]


def test_errors():
    g = W.config1().graph
    gg = load(g)
    with pytest.raises(R.RpqError) as e:
        gpu_regex(gg, "0*", 3, 1000)
    assert e.value.status == R.RPQ_ERR_INVALID
    with pytest.raises(R.RpqError):
        R.rpq_query(gg, R.rpq_nfa_compile("7", 8), 0)  # label beyond the graph's
    # capacity error with the size reported (two-call pattern)
    import ctypes

    nfa = R.rpq_nfa_compile("0/1*", 3)
    buf = np.empty(4, np.int32)
    cnt = ctypes.c_int64()
    s = R.lib().rpq_query(gg.h, nfa.h, 0, 0, R._ptr(buf), 4, ctypes.byref(cnt), None, None)
    assert s == R.RPQ_ERR_CAPACITY and cnt.value > 4


def test_device_and_bitset_outputs():
    import torch

    w = W.config1()
    g = w.graph
    gg = load(g)
    nfa = R.rpq_nfa_compile("0/1*", 3)
    exp = O.ssr(g.n, 3, g.src, g.dst, g.lab, oracle_compile("0/1*", 3), 0)["answer"]
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    cnt = R.rpq_query(gg, nfa, 0, out=out)
    assert out[:cnt].cpu().numpy().tolist() == exp.tolist()
    bits, c2 = R.rpq_query_bitset(gg, nfa, 0)
    assert c2 == exp.size
    got = [v for v in range(g.n) if (int(bits[v >> 6]) >> (v & 63)) & 1]
    assert got == exp.tolist()
    dbits = torch.zeros((g.n + 63) // 64, dtype=torch.int64, device="cuda")
    _, c3 = R.rpq_query_bitset(gg, nfa, 0, out=dbits)
    assert c3 == exp.size
    assert (dbits.cpu().numpy().view(np.uint64) == bits).all()


def test_query_runner_matches_oracle():
    """The prepared call (the bench's timed loop) gives the oracle's answers,
    and its statistics equal those of a plain rpq_query call."""
    import torch

    w = W.config2(per_template=3)
    g = w.graph
    gg = load(g)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    lean = R.QueryRunner(gg, out)
    full = R.QueryRunner(gg, out, with_stats=True)
    og = O.OracleGraph(g.n, g.n_labels, g.src, g.dst, g.lab)
    for q in w.queries:
        nfa = R.rpq_nfa_compile(q.regex, g.n_labels)
        exp = og.ssr(oracle_compile(q.regex, g.n_labels), q.source)["answer"]
        cnt = lean.run(nfa, q.source)
        assert out[:cnt].cpu().numpy().tolist() == exp.tolist(), q
        assert full.run(nfa, q.source) == cnt
        _, st = R.rpq_query(gg, nfa, q.source, out=out, with_stats=True)
        for k in ("levels", "visited_pairs", "expanded_pairs", "product_edges", "push_bytes",
                  "answer_count"):
            assert getattr(full.stats, k) == st[k], (k, q)
    with pytest.raises(R.RpqError):
        lean.run(R.rpq_nfa_compile("0", g.n_labels), g.n)


# ------------------------------------------------------ small workload ---

def test_config1_golden():
    import json

    fx = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "config1_answer.json")))
    w = W.config1()
    gg = load(w.graph)
    got, st = gpu_regex(gg, w.queries[0].regex, 3, w.queries[0].source, stats=True)
    assert got.tolist() == fx["answer"]
    assert st["answer_count"] == len(fx["answer"])


@pytest.mark.parametrize("pull_mode", MODES, ids=MODE_IDS, indirect=True)
def test_hubs_and_long_rows(pull_mode):
    """A hub with 100k out-edges (split across CTAs) and 20k in-edges (long
    pull rows) next to a sparse random part."""
    rng = W.below(77, 1, 400_000, 1 << 30)
    n = 150_000
    hub_out = np.arange(1, 100_001, dtype=np.int32)
    src = np.concatenate([np.zeros(100_000, np.int32), (rng[:50_000] % n).astype(np.int32),
                          np.arange(20_000, 40_000, dtype=np.int32)])
    dst = np.concatenate([hub_out, (rng[50_000:100_000] % n).astype(np.int32),
                          np.full(20_000, 7, np.int32)])
    lab = np.concatenate([np.zeros(100_000, np.int32), (rng[100_000:150_000] % 3).astype(np.int32),
                          np.ones(20_000, np.int32)])
    g = W.Graph("hub", n, 3, src, dst, lab)
    gg = load(g)
    og = O.OracleGraph(n, 3, src, dst, lab)
    for text, s in (("0/1", 0), ("0/(1|2)*", 0), ("(0|1|2)*", 0), ("^1/0*", 7), ("(^0|1)+", 5)):
        exp = og.ssr(oracle_compile(text, 3), s)["answer"]
        assert gpu_regex(gg, text, 3, s).tolist() == exp.tolist(), text


@pytest.mark.parametrize("pull_mode", MODES, ids=MODE_IDS, indirect=True)
def test_rmat_small_workload_counters(pull_mode):
    """R-MAT scale 14 with Zipf labels: several tiles per level, ragged tail;
    template DFAs given as transitions to compare every counter."""
    g = W.rmat_graph(14, 1 << 18, 8, seed=21)
    gg = load(g)
    og = O.OracleGraph(g.n, 8, g.src, g.dst, g.lab)
    L = 8
    autos = [
        (1, [(0, 0, 0)], [0], [0]),                        # a*
        (2, [(0, 1, 1), (1, 0, 1)], [0], [1]),             # b.a*
        (2, [(0, 0, 0), (0, 1, 0), (0, 2, 1)], [0], [1]),  # (a|b)*.c
        (2, [(0, 0 + L, 1), (1, 2, 1)], [0], [1]),         # a^-.c*
        (3, [(0, 0, 1), (1, 1, 2), (2, 0, 1), (0, 3 + L, 2)], [0], [2]),
    ]
    srcs = W.below(22, 1, 12, g.n)
    for S, tr, st_, fi in autos:
        dn = R.rpq_nfa_from_transitions(S, L, tr, st_, fi)
        on = Nfa(S, L, tr, st_, fi)
        for s in srcs.tolist():
            o = og.ssr(on, s)
            got, st = R.rpq_query(gg, dn, s, with_stats=True)
            assert got.tolist() == o["answer"].tolist()
            check_counters(st, o["counters"])


@pytest.mark.slow
def test_config2_sampled_parity():
    """The R-MAT scale-20 workload (2^24 edges, 8 labels) in the launch
    configuration the benchmark times: a sample of its queries against the
    oracle."""
    w = W.config2(per_template=6)
    g = w.graph
    gg = load(g)
    og = O.OracleGraph(g.n, g.n_labels, g.src, g.dst, g.lab)
    for q in w.queries:
        exp = og.ssr(oracle_compile(q.regex, g.n_labels), q.source)["answer"]
        got = gpu_regex(gg, q.regex, g.n_labels, q.source)
        assert got.tolist() == exp.tolist(), q


def test_autotune_keeps_answers():
    """The autotuner only changes the push/pull threshold; answers and the
    algorithm's counters must not change."""
    g = W.rmat_graph(14, 1 << 18, 4, seed=91)
    gg = load(g)
    og = O.OracleGraph(g.n, 4, g.src, g.dst, g.lab)
    texts = ["0*", "1/0*", "(0|1)*/2", "^0/1*"]
    srcs = W.below(92, 1, 8, g.n).tolist()
    nfas = [R.rpq_nfa_compile(texts[i % 4], 4) for i in range(8)]
    alpha, mn, solo = R.rpq_graph_autotune(gg, nfas, srcs)
    assert alpha in (0.0, 1.0, 2.0, 4.0, 8.0, 16.0, 64.0) and mn in (64, 256, 2048)
    assert solo in (-1, 512, 2048, 8192)
    for i in range(8):
        exp = og.ssr(oracle_compile(texts[i % 4], 4), srcs[i])["answer"]
        assert R.rpq_query(gg, nfas[i], srcs[i]).tolist() == exp.tolist()


SOLO = [(-1, 0), (2048, 256), (1 << 30, 1 << 30)]  # never, default, whenever no unit pulls
SOLO_IDS = ["grid_only", "solo_default", "solo_max"]


@pytest.mark.parametrize("solo", SOLO, ids=SOLO_IDS)
@pytest.mark.parametrize("pull_mode", [(1e9, 0), (4.0, 256)], ids=["pull", "auto"], indirect=True)
def test_solo_levels_and_workspace_reuse(solo, pull_mode, monkeypatch):
    """Levels run on the whole grid or on one CTA (with the switches between
    them), and every query leaves its workspace clean for the next: an
    interleaved sequence of queries on one graph, each against the oracle,
    then the first ones again."""
    monkeypatch.setenv("RPQ_SOLO_MASS", str(solo[0]))
    monkeypatch.setenv("RPQ_SOLO_ITEMS", str(solo[1]))
    g = W.rmat_graph(14, 1 << 18, 4, seed=63)
    gg = load(g)
    og = O.OracleGraph(g.n, 4, g.src, g.dst, g.lab)
    texts = ["0*", "1/(0|2)*", "(0|^1)*/2", "^0/1*", "3/3/3", "(0/1)*", "2"]
    srcs = W.below(64, 1, 14, g.n).tolist()
    jobs = [(texts[i % len(texts)], srcs[i]) for i in range(14)]
    exp = [og.ssr(oracle_compile(t, 4), s) for t, s in jobs]
    for (t, s), o in zip(jobs, exp):
        nfa = R.rpq_nfa_compile(t, 4)
        got, st = R.rpq_query(gg, nfa, s, with_stats=True)
        assert got.tolist() == o["answer"].tolist(), (t, s)
        # the counters depend on the automaton: compare with the oracle run
        # on the library's own (minimised) automaton
        e = nfa.export()
        same = Nfa(e["n_states"], 4, list(zip(e["from"].tolist(), e["label"].tolist(),
                                                e["to"].tolist())), e["starts"], e["finals"])
        check_counters(st, og.ssr(same, s)["counters"])
    for (t, s), o in zip(jobs[:5], exp[:5]):
        assert gpu_regex(gg, t, 4, s).tolist() == o["answer"].tolist(), (t, s)
    # bitset outputs go through the grid-wide answer sweep, also when a level
    # cap stops the traversal with a non-empty frontier; list outputs under a
    # cap; then the first queries again on the reused workspaces
    for (t, s) in jobs[:7]:
        for k in (0, 1, 2):
            exp_k = og.ssr(oracle_compile(t, 4), s, k)["answer"].tolist()
            bits = np.zeros((g.n + 63) // 64, np.uint64)
            R.rpq_query_bitset(gg, R.rpq_nfa_compile(t, 4), s, max_levels=k, out=bits)
            ids = np.nonzero(np.unpackbits(bits.view(np.uint8), bitorder="little"))[0]
            assert ids.tolist() == exp_k, (t, s, k)
            assert gpu_regex(gg, t, 4, s, k).tolist() == exp_k, (t, s, k)
    for (t, s), o in zip(jobs[:5], exp[:5]):
        assert gpu_regex(gg, t, 4, s).tolist() == o["answer"].tolist(), (t, s)


@pytest.mark.parametrize("cap", [0, 7, 4096], ids=["buffer_0", "buffer_7", "buffer_default"])
@pytest.mark.parametrize("solo", [SOLO[0], SOLO[2]], ids=["grid_only", "solo_max"])
def test_discovery_buffer_and_list_fallback(cap, solo, monkeypatch):
    """Each CTA measures the pairs it discovered from its own shared-memory
    buffer; when a buffer overflows (forced here with a small limit) the
    level is measured again from the visited lists, by the grid or by CTA 0
    alone.  Answers and counters must equal the oracle's either way."""
    import torch

    monkeypatch.setenv("RPQ_DISCOVERY_BUFFER", str(cap))
    monkeypatch.setenv("RPQ_SOLO_MASS", str(solo[0]))
    monkeypatch.setenv("RPQ_SOLO_ITEMS", str(solo[1]))
    g = W.rmat_graph(14, 1 << 18, 4, seed=67)
    gg = load(g)
    og = O.OracleGraph(g.n, 4, g.src, g.dst, g.lab)
    texts = ["0*", "(0|^1)*/2", "1/(0|2)*", "(0/1)*", "^3/(1|2)+"]
    srcs = W.below(68, 1, 10, g.n).tolist()
    for i, s in enumerate(srcs):
        t = texts[i % len(texts)]
        nfa = R.rpq_nfa_compile(t, 4)
        got, st = R.rpq_query(gg, nfa, s, with_stats=True)
        e = nfa.export()
        same = Nfa(e["n_states"], 4, list(zip(e["from"].tolist(), e["label"].tolist(),
                                                e["to"].tolist())), e["starts"], e["finals"])
        o = og.ssr(same, s)
        assert got.tolist() == o["answer"].tolist(), (t, s)
        check_counters(st, o["counters"])
        dev = torch.empty(g.n, dtype=torch.int32, device="cuda")
        k = R.rpq_query(gg, nfa, s, out=dev)
        assert dev[:k].cpu().numpy().tolist() == o["answer"].tolist(), (t, s)


def test_kernel_launch_counter():
    """Each single query is one cooperative launch of the traversal kernel,
    whatever its answer size or number of levels; a failed argument check
    launches nothing."""
    import torch

    g = W.rmat_graph(13, 1 << 16, 4, seed=69)
    gg = load(g)
    dev = torch.empty(g.n, dtype=torch.int32, device="cuda")
    srcs = W.below(70, 1, 6, g.n).tolist()
    nfa = R.rpq_nfa_compile("(0|^1)*/2", 4)
    a = R.rpq_kernel_launches()
    for s in srcs:
        R.rpq_query(gg, nfa, s, out=dev)
        R.rpq_query(gg, nfa, s)
    assert R.rpq_kernel_launches() - a == 2 * len(srcs)
    a = R.rpq_kernel_launches()
    with pytest.raises(R.RpqError):
        R.rpq_query(gg, nfa, g.n)  # source out of range
    assert R.rpq_kernel_launches() == a


def test_last_answer_two_call_pattern():
    """A host buffer that is too small gets RPQ_ERR_CAPACITY with the full
    count; rpq_last_answer then hands over the whole answer without a second
    traversal.  After a query into device memory there is no host answer."""
    import ctypes

    import torch

    g = W.rmat_graph(13, 60000, 4, seed=81)
    gg = load(g)
    og = O.OracleGraph(g.n, 4, g.src, g.dst, g.lab)
    nfa = R.rpq_nfa_compile("(0|1)*", 4)
    srcs = W.below(82, 1, 6, g.n).tolist()
    for s in srcs:
        exp = og.ssr(oracle_compile("(0|1)*", 4), s)["answer"]
        small = np.zeros(1, np.int32)
        cnt = ctypes.c_int64()
        st = R.lib().rpq_query(gg.h, nfa.h, s, 0, R._ptr(small), 1, ctypes.byref(cnt), None, None)
        assert st == (R.RPQ_OK if exp.size <= 1 else R.RPQ_ERR_CAPACITY)
        assert cnt.value == exp.size
        ptr, n = ctypes.POINTER(ctypes.c_int32)(), ctypes.c_int64()
        assert R.lib().rpq_last_answer(ctypes.byref(ptr), ctypes.byref(n)) == R.RPQ_OK
        got = np.ctypeslib.as_array(ptr, shape=(n.value,)).copy() if n.value else np.empty(0)
        assert got.tolist() == exp.tolist()
        assert R.rpq_query(gg, nfa, s).tolist() == exp.tolist()
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    R.rpq_query(gg, nfa, srcs[0], out=out)
    ptr, n = ctypes.POINTER(ctypes.c_int32)(), ctypes.c_int64()
    assert R.lib().rpq_last_answer(ctypes.byref(ptr), ctypes.byref(n)) == R.RPQ_ERR_INVALID


def test_concurrent_host_threads_share_a_graph():
    """Graphs and automata are shared by host threads: eight threads query
    one graph at once (each call takes its own workspace and stream; host
    answers go through each thread's own pinned buffer)."""
    import threading

    import torch

    g = W.rmat_graph(13, 80000, 4, seed=95)
    gg = load(g)
    og = O.OracleGraph(g.n, 4, g.src, g.dst, g.lab)
    texts = ["0*", "1/(0|2)*", "(0|^1)*/2", "^3/1*", "(0/1)*"]
    nfas = [R.rpq_nfa_compile(t, 4) for t in texts]
    srcs = W.below(96, 1, 64, g.n).tolist()
    exp = {(i % 5, s): og.ssr(oracle_compile(texts[i % 5], 4), s)["answer"].tolist()
           for i, s in enumerate(srcs)}
    errors = []

    def worker(tid):
        try:
            stream = torch.cuda.Stream()
            for k in range(tid, len(srcs), 8):
                key = (k % 5, srcs[k])
                got = R.rpq_query(gg, nfas[k % 5], srcs[k], stream=stream)
                if got.tolist() != exp[key]:
                    errors.append(("host", key))
                out = torch.empty(g.n, dtype=torch.int32, device="cuda")
                c = R.rpq_query(gg, nfas[k % 5], srcs[k], out=out, stream=stream)
                stream.synchronize()
                if out[:c].cpu().tolist() != exp[key]:
                    errors.append(("device", key))
        except Exception as e:  # reported below
            errors.append(("raised", repr(e)))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(8)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors[:5]
