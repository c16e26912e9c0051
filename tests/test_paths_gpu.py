"""GPU parity of the query forms beyond single-source reachability, through
the C ABI, against the CPU oracle:

  * a set of sources V_s (section 2: a 2-RPQ takes a set of starting
    vertices; level 0 = Q_S x V_s) -- rpq_query_multi;
  * single-destination reachability (section 2), computed as the
    single-source query of the reversed automaton (section 4) --
    rpq_query_sdr, checked against the definition {u : v_f in SSR(u)};
  * the level of first reach of every answer vertex -- rpq_query_levels;
  * a shortest witness path -- rpq_query_witness: its length is unique (the
    target's first-reach level) and is compared exactly; the path itself is
    one of possibly many, so it is checked for validity (a 2-path from a
    source to the target whose word the automaton accepts).
"""

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


@pytest.fixture(scope="module")
def rmat14():
    g = W.rmat_graph(14, 1 << 18, 4, seed=35)
    gg = load(g)
    og = O.OracleGraph(g.n, 4, g.src, g.dst, g.lab)
    yield g, gg, og
    og.close()


TEXTS = ["0*", "1/0*", "(0|1)*/2", "^0/1*", "(0/1)*", "0/(1|^2)*/3", "(^0|1)+", "2/^2"]


# ------------------------------------------------------------ source sets --

def test_multi_source_tiny_random():
    for seed in range(60):
        g = W.tiny_graph(seed + 5100, max_n=12, max_m=30)
        S, trans, starts, finals = W.tiny_automaton(seed + 5200, g.n_labels, max_states=5,
                                                    max_trans=10)
        r = W.below(seed, 14, 5, 1 << 20)
        srcs = [int(x % g.n) for x in r[: 1 + seed % 5]]
        og = O.OracleGraph(g.n, g.n_labels, g.src, g.dst, g.lab)
        gg = load(g)
        dn = R.rpq_nfa_from_transitions(S, g.n_labels, trans, starts, finals)
        on = Nfa(S, g.n_labels, trans, starts, finals)
        for k in (0, 1, 2):
            exp = og.query(on, srcs, k)
            got, st = R.rpq_query_multi(gg, dn, srcs, k, with_stats=True)
            assert got.tolist() == exp["answer"].tolist(), (seed, k, srcs)
            assert st["visited_pairs"] == exp["counters"]["visited"]
            assert st["levels"] == exp["counters"]["levels"]
        og.close()


@pytest.mark.parametrize("n_src", [1, 7, 300, 5000])
def test_multi_source_rmat(rmat14, n_src):
    """From 1 up to 5,000 sources (level 0 larger than a CTA's discovery
    buffer), with repeated sources, host and device outputs."""
    import torch

    g, gg, og = rmat14
    srcs = W.below(40 + n_src, 1, n_src, g.n).tolist()
    if n_src > 1:
        srcs += srcs[: n_src // 3]  # repeats
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    for text in TEXTS:
        exp = og.query(oracle_compile(text, 4), srcs)["answer"].tolist()
        nfa = R.rpq_nfa_compile(text, 4)
        assert R.rpq_query_multi(gg, nfa, srcs).tolist() == exp, text
        cnt = R.rpq_query_multi(gg, nfa, srcs, out=out)
        assert out[:cnt].cpu().numpy().tolist() == exp, text


def test_multi_source_edge_cases(rmat14):
    g, gg, og = rmat14
    nfa = R.rpq_nfa_compile("0*", 4)
    assert R.rpq_query_multi(gg, nfa, []).size == 0  # empty V_s: empty answer
    one = R.rpq_query(gg, nfa, 17)
    assert R.rpq_query_multi(gg, nfa, [17]).tolist() == one.tolist()
    assert R.rpq_query_multi(gg, nfa, [17, 17, 17]).tolist() == one.tolist()
    with pytest.raises(R.RpqError) as e:
        R.rpq_query_multi(gg, nfa, [3, g.n])
    assert e.value.status == R.RPQ_ERR_INVALID
    # every vertex a source: a* answers everything
    assert R.rpq_query_multi(gg, nfa, np.arange(g.n)).size == g.n


# ------------------------------------------------------- single destination --

def test_sdr_tiny_every_target():
    """Every target of tiny graphs: the answer equals {u : v_f in SSR(u)}."""
    for seed in range(30):
        g = W.tiny_graph(seed + 6100, max_n=10, max_m=24)
        L = g.n_labels
        text, _, _ = W.random_regex(seed + 6200, L, 1 + seed % 4)
        og = O.OracleGraph(g.n, L, g.src, g.dst, g.lab)
        gg = load(g)
        on = oracle_compile(text, L)
        nfa = R.rpq_nfa_compile(text, L)
        for t in range(g.n):
            assert R.rpq_query_sdr(gg, nfa, t).tolist() == og.sdr(on, t).tolist(), (text, t)
        og.close()


def test_sdr_rmat_sampled_targets(rmat14):
    """Sampled targets on the R-MAT scale-14 graph; the expected answer of
    every target comes from single-source oracle queries from every vertex."""
    g, gg, og = rmat14
    targets = W.below(77, 1, 24, g.n).tolist()
    for text in ("0/1*", "^0/1*", "(0|^3)/2"):
        on = oracle_compile(text, 4)
        hits = {t: [] for t in targets}
        tset = set(targets)
        for u in range(g.n):
            for v in set(og.ssr(on, u)["answer"].tolist()) & tset:
                hits[v].append(u)
        nfa = R.rpq_nfa_compile(text, 4)
        for t in targets:
            assert R.rpq_query_sdr(gg, nfa, t).tolist() == sorted(hits[t]), (text, t)


# -------------------------------------------------------- first-reach level --

def test_levels_tiny_random():
    for seed in range(60):
        g = W.tiny_graph(seed + 7100, max_n=12, max_m=30)
        S, trans, starts, finals = W.tiny_automaton(seed + 7200, g.n_labels, max_states=5,
                                                    max_trans=10)
        srcs = [seed % g.n] if seed % 3 else [seed % g.n, (seed // 3) % g.n]
        og = O.OracleGraph(g.n, g.n_labels, g.src, g.dst, g.lab)
        gg = load(g)
        dn = R.rpq_nfa_from_transitions(S, g.n_labels, trans, starts, finals)
        on = Nfa(S, g.n_labels, trans, starts, finals)
        for k in (0, 2):
            exp = og.query(on, srcs, k, want_first_level=True)
            v, lv = R.rpq_query_levels(gg, dn, srcs, k)
            assert v.tolist() == exp["answer"].tolist(), (seed, k)
            assert lv.tolist() == exp["first_level"][v].tolist(), (seed, k)
        og.close()


def test_levels_rmat_host_and_device(rmat14):
    import ctypes

    import torch

    g, gg, og = rmat14
    srcs = W.below(81, 1, 3, g.n).tolist()
    for text in TEXTS:
        exp = og.query(oracle_compile(text, 4), srcs, want_first_level=True)
        nfa = R.rpq_nfa_compile(text, 4)
        v, lv = R.rpq_query_levels(gg, nfa, srcs)
        assert v.tolist() == exp["answer"].tolist(), text
        assert lv.tolist() == exp["first_level"][v].tolist(), text
        # device outputs, and the levels again after an ordinary query on the
        # same workspace (the pair levels must have been reset)
        R.rpq_query(gg, nfa, srcs[0])
        dv = torch.empty(g.n, dtype=torch.int32, device="cuda")
        dl = torch.empty(g.n, dtype=torch.int32, device="cuda")
        s_arr = np.array(srcs, np.int32)
        cnt = ctypes.c_int64()
        assert R.lib().rpq_query_levels(gg.h, nfa.h, len(srcs), R._ptr(s_arr), 0, R._ptr(dv),
                                        R._ptr(dl), g.n, ctypes.byref(cnt), None) == 0
        assert dv[: cnt.value].cpu().numpy().tolist() == v.tolist()
        assert dl[: cnt.value].cpu().numpy().tolist() == lv.tolist()


# ---------------------------------------------------------------- witness --

def check(g, text, srcs, target, path, exp_level):
    on = oracle_compile(text, g.n_labels)
    if exp_level < 0:
        assert path is None
        return
    assert path is not None
    vs, ws = path
    assert len(ws) == exp_level
    ok, why = O.check_witness(g.n, g.n_labels, g.src, g.dst, g.lab, on.accepts, srcs, target,
                              vs, ws)
    assert ok, why


def test_witness_tiny_every_vertex():
    for seed in range(40):
        g = W.tiny_graph(seed + 8100, max_n=10, max_m=24)
        L = g.n_labels
        text, _, _ = W.random_regex(seed + 8200, L, 1 + seed % 4)
        srcs = [seed % g.n]
        og = O.OracleGraph(g.n, L, g.src, g.dst, g.lab)
        fl = og.query(oracle_compile(text, L), srcs, want_first_level=True)["first_level"]
        og.close()
        gg = load(g)
        nfa = R.rpq_nfa_compile(text, L)
        for t in range(g.n):
            check(g, text, srcs, t, R.rpq_query_witness(gg, nfa, srcs, t), int(fl[t]))


def test_witness_rmat(rmat14):
    g, gg, og = rmat14
    srcs = W.below(91, 1, 2, g.n).tolist()
    for text in TEXTS:
        exp = og.query(oracle_compile(text, 4), srcs, want_first_level=True)
        fl = exp["first_level"]
        nfa = R.rpq_nfa_compile(text, 4)
        ans = exp["answer"]
        picks = ans[:: max(1, ans.size // 6)][:6].tolist() + W.below(92, 1, 2, g.n).tolist()
        for t in picks:
            check(g, text, srcs, t, R.rpq_query_witness(gg, nfa, srcs, t), int(fl[t]))


def test_witness_long_chain_and_capacity():
    """A chain of 3,000 vertices: the witness of the far end has 2,999
    steps (the binding grows its buffer after RPQ_ERR_CAPACITY)."""
    import ctypes

    m = 3000
    src = np.arange(m - 1, dtype=np.int32)
    g = W.Graph("chain", m, 1, src, src + 1, np.zeros(m - 1, np.int32))
    gg = load(g)
    nfa = R.rpq_nfa_compile("0*", 1)
    vs, ws = R.rpq_query_witness(gg, nfa, [0], m - 1)
    assert vs.tolist() == list(range(m)) and ws.tolist() == [0] * (m - 1)
    pv = np.empty(4, np.int32)
    ps = np.empty(4, np.int32)
    ln = ctypes.c_int32()
    s_arr = np.array([0], np.int32)
    st = R.lib().rpq_query_witness(gg.h, nfa.h, 1, R._ptr(s_arr), m - 1, 0, R._ptr(pv), R._ptr(ps),
                                   4, ctypes.byref(ln), None)
    assert st == R.RPQ_ERR_CAPACITY and ln.value == m - 1
    assert R.rpq_query_witness(gg, R.rpq_nfa_compile("^0", 1), [5], 4)[1].tolist() == [1]
    assert R.rpq_query_witness(gg, nfa, [5], 4) is None  # not reachable forwards


# ------------------------------------- Algorithm 2 -> Algorithm 1 hybrid --
# Section 5.1: Algorithm 2 (every step expands the whole visited set, no
# traversal matrix M) while the visited set is small, then Algorithm 1.
# The sets P_k are the same either way (section 4), so answers, levels and
# visited counts equal the oracle's; with Algorithm 2 throughout, the
# expanded-pair counter is the sum of |P_j| over the expanded levels j.

@pytest.mark.parametrize("switch", [1 << 40, 100, 7])
def test_hybrid_tiny_random(switch):
    for seed in range(60):
        g = W.tiny_graph(seed + 9100, max_n=12, max_m=30)
        S, trans, starts, finals = W.tiny_automaton(seed + 9200, g.n_labels, max_states=5,
                                                    max_trans=10)
        og = O.OracleGraph(g.n, g.n_labels, g.src, g.dst, g.lab)
        gg = load(g)
        R.rpq_graph_set_hybrid(gg, switch)
        dn = R.rpq_nfa_from_transitions(S, g.n_labels, trans, starts, finals)
        on = Nfa(S, g.n_labels, trans, starts, finals)
        src = seed % g.n
        for k in (0, 2):
            exp = og.ssr(on, src, k, level_cap=64)
            got, st = R.rpq_query(gg, dn, src, k, with_stats=True)
            assert got.tolist() == exp["answer"].tolist(), (seed, k, switch)
            c = exp["counters"]
            assert (st["levels"], st["visited_pairs"]) == (c["levels"], c["visited"]), (seed, k)
            assert st["expanded_pairs"] >= c["expanded"]
            if switch == 1 << 40 and k == 0:
                sizes = np.cumsum(exp["level_sizes"][: c["levels"] + 1])
                assert st["expanded_pairs"] == int(sizes.sum()), (seed, sizes)
        og.close()


def test_hybrid_rmat_switches_to_algorithm_1(rmat14):
    g, gg, og = rmat14
    srcs = W.below(95, 1, 4, g.n).tolist()
    R.rpq_graph_set_hybrid(gg, 100)
    try:
        for text in TEXTS:
            on = oracle_compile(text, 4)
            nfa = R.rpq_nfa_compile(text, 4)
            for s in srcs:
                # regex automata differ between the two sides (minimised DFA
                # here, Thompson NFA in the oracle), so the counters are
                # compared with Algorithm 1 on the same DFA
                exp = og.ssr(on, s)
                got, st = R.rpq_query(gg, nfa, s, with_stats=True)
                assert got.tolist() == exp["answer"].tolist(), (text, s)
                R.rpq_graph_set_hybrid(gg, 0)
                _, st1 = R.rpq_query(gg, nfa, s, with_stats=True)
                R.rpq_graph_set_hybrid(gg, 100)
                assert st["levels"] == st1["levels"], (text, s)
                assert st["visited_pairs"] == st1["visited_pairs"], (text, s)
                assert st["expanded_pairs"] >= st1["expanded_pairs"], (text, s)
            assert R.rpq_query_multi(gg, nfa, srcs).tolist() == og.query(on, srcs)["answer"].tolist()
    finally:
        R.rpq_graph_set_hybrid(gg, 0)


# ------------------------------------------------------- rare label first --
# Section 5.4-5.5 / section 6: when every accepted word reads a rare label,
# a backward search from that label's edges prunes the forward search.  The
# answer is the query's answer whatever the plan.

def test_rare_plan_tiny_random():
    for seed in range(80):
        g = W.tiny_graph(seed + 9600, max_n=12, max_m=30)
        S, trans, starts, finals = W.tiny_automaton(seed + 9700, g.n_labels, max_states=5,
                                                    max_trans=10)
        og = O.OracleGraph(g.n, g.n_labels, g.src, g.dst, g.lab)
        gg = load(g)
        R.rpq_graph_set_rare_plan(gg, 1 << 40)  # every label counts as rare
        dn = R.rpq_nfa_from_transitions(S, g.n_labels, trans, starts, finals)
        on = Nfa(S, g.n_labels, trans, starts, finals)
        for src in range(0, g.n, max(1, g.n // 4)):
            for k in (0, 2):
                exp = og.ssr(on, src, k)["answer"].tolist()
                assert R.rpq_query(gg, dn, src, k).tolist() == exp, (seed, src, k, trans)
        og.close()


def test_rare_plan_knowledge_base_graph():
    """a/b*/c and a/(b|^c)*/d with a rare last label on a power-law graph of
    500 labels: the same answers as the plain search and the oracle (there
    the rare labels' edges sit in the giant component, so the backward
    search prunes little)."""
    g = W.chung_lu_graph(1_000_000, 10_000_000, 2.1, 500, 1.1, seed=2)
    gg = load(g)
    og = O.OracleGraph(g.n, g.n_labels, g.src, g.dst, g.lab)
    counts = np.bincount(g.lab, minlength=500)
    rare = [int(x) for x in np.flatnonzero((counts > 0) & (counts < 2000))[:6]]
    srcs = W.below(97, 1, 6, g.n).tolist()
    fewer = 0
    for i, c in enumerate(rare):
        for text in (f"0/1*/{c}", f"1/(0|^2)*/{c}", f"(0|1)*/{c}/3"):
            s = srcs[i]
            R.rpq_graph_set_rare_plan(gg, 0)
            plain, st0 = R.rpq_query(gg, R.rpq_nfa_compile(text, 500), s, with_stats=True)
            R.rpq_graph_set_rare_plan(gg, 10000)
            ruled, st1 = R.rpq_query(gg, R.rpq_nfa_compile(text, 500), s, with_stats=True)
            assert ruled.tolist() == plain.tolist(), (text, s)
            assert ruled.tolist() == og.ssr(oracle_compile(text, 500), s)["answer"].tolist()
    og.close()


def test_rare_plan_prunes_a_long_path():
    """0/1*/2 from the head of a 5,000-vertex path of label 1 whose only
    label-2 edge leaves vertex 10: the plain search walks the whole path
    (5,000 levels); rare label first walks back from the one label-2 edge,
    keeps the first 11 path vertices and answers in a dozen levels."""
    m = 5000
    src = np.concatenate([[0], np.arange(1, m, dtype=np.int32), [11]]).astype(np.int32)
    dst = np.concatenate([[1], np.arange(2, m + 1, dtype=np.int32), [m + 1]]).astype(np.int32)
    lab = np.concatenate([[0], np.ones(m - 1, np.int32), [2]]).astype(np.int32)
    g = W.Graph("path", m + 2, 3, src, dst, lab)
    gg = load(g)
    nfa = R.rpq_nfa_compile("0/1*/2", 3)
    plain, st0 = R.rpq_query(gg, nfa, 0, with_stats=True)
    R.rpq_graph_set_rare_plan(gg, 10)
    ruled, st1 = R.rpq_query(gg, nfa, 0, with_stats=True)
    assert plain.tolist() == ruled.tolist() == [m + 1]
    exp = O.ssr(g.n, 3, src, dst, lab, oracle_compile("0/1*/2", 3), 0)["answer"].tolist()
    assert ruled.tolist() == exp
    assert st0["levels"] >= m - 1 and st1["levels"] <= 13
    assert st1["visited_pairs"] < 30 < st0["visited_pairs"]
