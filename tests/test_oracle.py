"""Pins for the CPU oracle (no GPU).

The oracle (oracle/) is checked against things other than itself:
  * brute force straight from the definition of single-source reachability
    (section 2) on tiny random graphs and automata, per word-length bound k
    (section 4: P_k holds the pairs reached by words of length <= k);
  * Algorithm 1 and Algorithm 2 written as dense Boolean matrix products in
    the paper's notation (section 4);
  * closed forms on chains, complete bipartite layers, stars and cycles;
  * invariants of the appendix proof (levels disjoint, P grows strictly while
    M != 0, at most |Q||V| iterations);
  * metamorphic identities: a^- on G equals a on G^T (section 3,
    G^{a^-} = (G^a)^T), Ans(R1|R2) = Ans(R1) u Ans(R2), single-destination
    through the reversed automaton N^- (section 4);
  * the oracle's regex -> NFA construction against Python's ``re`` on all
    words up to length 5.
"""

import itertools
import json
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from oracle.regex_nfa import Nfa, compile_regex, inverse_nfa, RegexError
from paper_2412_10287_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def nfa_from_lists(S, trans, starts, finals, L):
    return Nfa(S, L, list(trans), list(starts), list(finals))


def answer(g, nfa, source, k=0, **kw):
    return O.ssr(g.n, g.n_labels, g.src, g.dst, g.lab, nfa, source, k, **kw)


def as_set(a):
    return set(int(x) for x in a)


# ------------------------------------------------------------ brute force --

@pytest.mark.parametrize("seed", range(60))
def test_oracle_vs_bruteforce_random_automata(seed):
    g = W.tiny_graph(seed)
    S, trans, starts, finals = W.tiny_automaton(seed + 1000, g.n_labels)
    nfa = nfa_from_lists(S, trans, starts, finals, g.n_labels)
    src = seed % g.n
    K = 5
    bf = O.brute_force_levels(g.n, g.n_labels, g.src, g.dst, g.lab, src, nfa.accepts, K)
    for k in range(K + 1):
        got = answer(g, nfa, src, k)["answer"] if k > 0 else None
        if k == 0:
            # max_levels = 0 means unbounded; level 0 alone is Q_S x {v_s}
            exp0 = [src] if set(starts) & set(finals) else []
            assert as_set(bf[0]) == set(exp0)
            continue
        assert as_set(got) == as_set(bf[k]), (k, trans, starts, finals)
    # unbounded answer contains every bounded one and equals the fixpoint
    full = answer(g, nfa, src, 0)
    lv = full["counters"]["levels"]
    assert lv <= S * g.n
    capped = answer(g, nfa, src, max(lv, 1))
    assert as_set(capped["answer"]) == as_set(full["answer"])
    assert as_set(bf[K]) <= as_set(full["answer"])


@pytest.mark.parametrize("seed", range(40))
def test_oracle_vs_bruteforce_random_regex(seed):
    """Random regular expressions: the word-membership test of the brute force
    is Python's ``re`` on a character rendering of the expression, so neither
    the oracle's parser nor its automaton is used on that side."""
    g = W.tiny_graph(seed + 77, max_labels=2)
    L = g.n_labels
    text, pat, chars = W.random_regex(seed, L, depth=2 + seed % 3)
    rx = re.compile(pat)
    accepts = lambda w: rx.fullmatch("".join(chars[s] for s in w)) is not None
    nfa = compile_regex(text, L)
    src = (seed * 7) % g.n
    K = 4
    bf = O.brute_force_levels(g.n, L, g.src, g.dst, g.lab, src, accepts, K)
    for k in range(1, K + 1):
        assert as_set(answer(g, nfa, src, k)["answer"]) == as_set(bf[k]), (text, k)


# ---------------------------------------------------- regex construction --

@pytest.mark.parametrize("seed", range(80))
def test_regex_nfa_language_vs_python_re(seed):
    L = 1 + seed % 3
    text, pat, chars = W.random_regex(seed + 5000, L, depth=1 + seed % 4)
    rx = re.compile(pat)
    nfa = compile_regex(text, L)
    for k in range(0, 6):
        for w in itertools.product(range(2 * L), repeat=k):
            exp = rx.fullmatch("".join(chars[s] for s in w)) is not None
            assert nfa.accepts(w) == exp, (text, pat, w)


def test_regex_syntax_cases():
    L = 3
    acc = lambda t, w: compile_regex(t, L).accepts(w)
    assert acc("0", [0]) and not acc("0", [3])
    assert acc("^0", [3]) and not acc("^0", [0])
    assert acc("^^0", [0])  # (a^-)^- = a
    assert acc("^(0/1)", [4, 3])  # (ab)^- = b^- a^-
    assert acc("0 1", [0, 1]) and acc("0/1", [0, 1]) and acc("0·1", [0, 1])
    assert acc("(0|1)*/2", [1, 0, 1, 2]) and not acc("(0|1)*/2", [1, 0, 1])
    assert acc("0+", [0, 0]) and not acc("0+", [])
    assert acc("0?", []) and acc("0?", [0]) and not acc("0?", [0, 0])
    for bad in ["", "(", "0|", "*", "3", "0/", "a"]:
        with pytest.raises(RegexError):
            compile_regex(bad, L)


# ---------------------------------------------------- dense algorithms -----

@pytest.mark.parametrize("seed", range(40))
def test_oracle_vs_dense_algorithm1_and_2(seed):
    g = W.tiny_graph(seed + 300, max_n=10, max_m=24)
    S, trans, starts, finals = W.tiny_automaton(seed + 400, g.n_labels, max_states=5,
                                                max_trans=12)
    nfa = nfa_from_lists(S, trans, starts, finals, g.n_labels)
    src = seed % g.n
    res = answer(g, nfa, src, 0, want_visited=True)
    P1, ans1, levels1 = O.alg1_dense(g.n, g.n_labels, g.src, g.dst, g.lab, nfa, src)
    P2, ans2 = O.alg2_dense(g.n, g.n_labels, g.src, g.dst, g.lab, nfa, src)
    assert (res["visited"] == P1).all()
    assert (P1 == P2).all()
    assert as_set(res["answer"]) == as_set(np.flatnonzero(ans1)) == as_set(np.flatnonzero(ans2))
    assert res["counters"]["levels"] == levels1
    for k in range(1, 4):
        Pk, _, _ = O.alg1_dense(g.n, g.n_labels, g.src, g.dst, g.lab, nfa, src, k)
        rk = answer(g, nfa, src, k, want_visited=True)
        assert (rk["visited"] == Pk).all()


# -------------------------------------------------------- closed forms -----

def chain(m, label=0, L=1):
    src = np.arange(m - 1, dtype=np.int32)
    return W.Graph("chain", m, L, src, src + 1, np.full(m - 1, label, np.int32))


@pytest.mark.parametrize("m,s", [(1, 0), (2, 0), (10, 0), (10, 4), (257, 3), (1000, 999)])
def test_closed_form_chain(m, s):
    g = chain(m)
    # one-state automaton for a*: exactly one new pair per level
    star = Nfa(1, 1, [(0, 0, 0)], [0], [0])
    r = answer(g, star, s, level_cap=m + 2)
    assert as_set(r["answer"]) == set(range(s, m))
    assert r["counters"]["levels"] == m - 1 - s
    assert (r["level_sizes"][: m - s] == 1).all() and r["level_sizes"][m - s] == 0
    # product edges: every visited pair (0, v) with v < m-1 has one out-edge and
    # one transition; push bytes: 8 + 4 deg per expanded pair with a transition
    c = r["counters"]
    assert c["product_edges"] == m - 1 - s
    assert c["push_bytes"] == 8 * (m - s) + 4 * (m - 1 - s)
    r = answer(g, compile_regex("0*", 1), s)
    assert as_set(r["answer"]) == set(range(s, m))
    r = answer(g, compile_regex("^0*", 1), s)
    assert as_set(r["answer"]) == set(range(0, s + 1))
    r = answer(g, compile_regex("0+", 1), s)
    assert as_set(r["answer"]) == set(range(s + 1, m))
    for k in range(1, 5):
        r = answer(g, compile_regex("0*", 1), s, k)
        assert as_set(r["answer"]) == set(range(s, min(m, s + k + 1)))


def test_closed_form_complete_bipartite():
    A, B, C = list(range(0, 4)), list(range(4, 9)), list(range(9, 12))
    src, dst, lab = [], [], []
    for u in A:
        for v in B:
            src.append(u); dst.append(v); lab.append(0)
    for u in B:
        for v in C:
            src.append(u); dst.append(v); lab.append(1)
    g = W.Graph("bip", 12, 2, np.array(src, np.int32), np.array(dst, np.int32),
                np.array(lab, np.int32))
    q = compile_regex("0/1", 2)
    for s in A:
        assert as_set(answer(g, q, s)["answer"]) == set(C)
    for s in B + C:
        assert as_set(answer(g, q, s)["answer"]) == set()
    # inverse: from c in C, ^1/^0 reaches all of A
    assert as_set(answer(g, compile_regex("^1/^0", 2), 10)["answer"]) == set(A)
    assert as_set(answer(g, compile_regex("^(0/1)", 2), 10)["answer"]) == set(A)


def test_closed_form_star_and_cycle():
    k = 9
    g = W.Graph("star", k + 1, 2, np.zeros(k, np.int32), np.arange(1, k + 1, dtype=np.int32),
                np.zeros(k, np.int32))
    assert as_set(answer(g, compile_regex("0/1*", 2), 0)["answer"]) == set(range(1, k + 1))
    assert as_set(answer(g, compile_regex("0/^0", 2), 3)["answer"]) == set()
    assert as_set(answer(g, compile_regex("^0/0", 2), 3)["answer"]) == set(range(1, k + 1))
    m = 12  # cycle 1..m labelled 1, entered from 0 by label 0
    src = [0] + list(range(1, m + 1))
    dst = [1] + [v % m + 1 for v in range(1, m + 1)]
    lab = [0] + [1] * m
    g = W.Graph("cycle", m + 1, 2, np.array(src, np.int32), np.array(dst, np.int32),
                np.array(lab, np.int32))
    assert as_set(answer(g, compile_regex("0/1*", 2), 0)["answer"]) == set(range(1, m + 1))
    assert as_set(answer(g, compile_regex("0/1/1", 2), 0)["answer"]) == {3}
    assert as_set(answer(g, compile_regex("0/(1/1)*", 2), 0)["answer"]) == set(range(1, m + 1, 2))


def test_empty_and_epsilon_cases():
    g = chain(5)
    # no final state reachable: empty answer
    nfa = Nfa(2, 1, [(0, 0, 1)], [0], [])
    assert answer(g, nfa, 0)["answer"].size == 0
    # start state final: the source answers (zero-length path)
    assert as_set(answer(g, compile_regex("0*", 1), 4)["answer"]) == {4}
    assert as_set(answer(g, compile_regex("0?", 1), 4)["answer"]) == {4}
    # a graph with no edges
    g0 = W.Graph("empty", 3, 1, np.zeros(0, np.int32), np.zeros(0, np.int32),
                 np.zeros(0, np.int32))
    assert as_set(answer(g0, compile_regex("0*", 1), 1)["answer"]) == {1}
    assert as_set(answer(g0, compile_regex("0", 1), 1)["answer"]) == set()
    # a label the graph does not carry contributes nothing
    assert as_set(answer(chain(4, 0, 2), compile_regex("1*/0", 2), 0)["answer"]) == {1}


def test_self_loops_duplicates_multilabel():
    # 0 -0-> 0 (loop), 0 -0-> 1 twice, 0 -1-> 1 (second label on the same edge)
    g = W.Graph("multi", 2, 2, np.array([0, 0, 0, 0], np.int32), np.array([0, 1, 1, 1], np.int32),
                np.array([0, 0, 0, 1], np.int32))
    assert as_set(answer(g, compile_regex("0/0/0", 2), 0)["answer"]) == {0, 1}
    assert as_set(answer(g, compile_regex("1", 2), 0)["answer"]) == {1}
    assert as_set(answer(g, compile_regex("0/^1", 2), 0)["answer"]) == {0}


# ---------------------------------------------------------- invariants -----

@pytest.mark.parametrize("seed", range(20))
def test_level_invariants(seed):
    g = W.tiny_graph(seed + 900, max_n=12, max_m=30)
    S, trans, starts, finals = W.tiny_automaton(seed + 901, g.n_labels, 4, 10)
    nfa = nfa_from_lists(S, trans, starts, finals, g.n_labels)
    src = seed % g.n
    full = answer(g, nfa, src, 0, want_visited=True, level_cap=S * g.n + 2)
    lv = full["counters"]["levels"]
    sizes = full["level_sizes"]
    assert lv <= S * g.n  # termination bound of the appendix
    assert (sizes[1 : lv + 1] > 0).all() and (sizes[lv + 1 :] == 0).all()
    assert full["counters"]["visited"] == sizes.sum() == full["visited"].sum()
    prev_P = None
    prev_ans = set()
    for k in range(1, lv + 2):
        r = answer(g, nfa, src, k, want_visited=True)
        P = r["visited"]
        assert P.sum() == sizes[: k + 1].sum()  # M_k disjoint from P_{k-1}
        if prev_P is not None:
            assert (prev_P <= P).all()  # P_k subset of P_{k+1}
        assert prev_ans <= as_set(r["answer"])
        prev_P, prev_ans = P, as_set(r["answer"])
    assert (prev_P == full["visited"]).all()


# ---------------------------------------------------------- metamorphic ----

@pytest.mark.parametrize("seed", range(20))
def test_inverse_is_transpose(seed):
    """a^- on G gives the same answer as a on G^T (section 3)."""
    g = W.tiny_graph(seed + 1200)
    L = g.n_labels
    text, _, _ = W.random_regex(seed + 1300, L, depth=3)
    gt = W.Graph("T", g.n, L, g.dst, g.src, g.lab)
    # swap every symbol with its inverse in the automaton
    nfa = compile_regex(text, L)
    sw = Nfa(nfa.n_states, L, [(q, a + L if a < L else a - L, r) for q, a, r in nfa.transitions],
             nfa.starts, nfa.finals)
    for s in range(g.n):
        assert as_set(answer(g, nfa, s)["answer"]) == as_set(answer(gt, sw, s)["answer"])


@pytest.mark.parametrize("seed", range(15))
def test_union_identity(seed):
    g = W.tiny_graph(seed + 1500)
    L = g.n_labels
    t1, _, _ = W.random_regex(seed + 1600, L, 3)
    t2, _, _ = W.random_regex(seed + 1700, L, 3)
    s = seed % g.n
    a = as_set(answer(g, compile_regex(t1, L), s)["answer"])
    b = as_set(answer(g, compile_regex(t2, L), s)["answer"])
    c = as_set(answer(g, compile_regex(f"({t1})|({t2})", L), s)["answer"])
    assert c == a | b


@pytest.mark.parametrize("seed", range(15))
def test_single_destination_by_reversed_automaton(seed):
    """SDR(Q) = SSR(Q^-) with N^- (section 4): u answers the single-destination
    query for v_f iff v_f answers the single-source query from u."""
    g = W.tiny_graph(seed + 1800)
    L = g.n_labels
    text, _, _ = W.random_regex(seed + 1900, L, 3)
    nfa = compile_regex(text, L)
    for vf in range(g.n):
        expected = {u for u in range(g.n) if vf in as_set(answer(g, nfa, u)["answer"])}
        got = as_set(answer(g, inverse_nfa(nfa), vf)["answer"])
        assert got == expected


# -------------------------------------------------------------- counters ---

def test_counters_two_state_dfa_on_star():
    """a/b* as a 2-state DFA on a star with k a-leaves each carrying one b-edge
    back to the centre: closed forms for every counter."""
    k = 7
    src = [0] * k + list(range(1, k + 1))
    dst = list(range(1, k + 1)) + [0] * k
    lab = [0] * k + [1] * k
    g = W.Graph("star2", k + 1, 2, np.array(src, np.int32), np.array(dst, np.int32),
                np.array(lab, np.int32))
    dfa = Nfa(2, 2, [(0, 0, 1), (1, 1, 1)], [0], [1])
    c = answer(g, dfa, 0)["counters"]
    # level 0: (0,0); level 1: (1,leaf) x k; level 2: (1,0) via b; level 3: nothing new
    assert c["levels"] == 2
    assert c["visited"] == 1 + k + 1
    assert c["answer"] == k + 1
    # expanded: (0,0) deg_a = k; each (1,leaf) deg_b = 1; (1,0) deg_b = 0
    assert c["expanded"] == 1 + k + 1
    assert c["product_edges"] == k + k + 0
    assert c["push_bytes"] == (8 + 4 * k) + k * (8 + 4) + (8 + 0)


@pytest.mark.parametrize("seed", range(10))
def test_duplicate_edges_change_nothing(seed):
    """E is a set and G^a Boolean: repeating every triple leaves the answer
    and every counter unchanged."""
    g = W.tiny_graph(seed + 2100, max_n=10, max_m=20)
    S, trans, starts, finals = W.tiny_automaton(seed + 2101, g.n_labels, 4, 10)
    nfa = nfa_from_lists(S, trans, starts, finals, g.n_labels)
    g2 = W.Graph("dup", g.n, g.n_labels, np.concatenate([g.src, g.src[::-1]]),
                 np.concatenate([g.dst, g.dst[::-1]]), np.concatenate([g.lab, g.lab[::-1]]))
    for s in range(g.n):
        a, b = answer(g, nfa, s), answer(g2, nfa, s)
        assert a["answer"].tolist() == b["answer"].tolist()
        assert a["counters"] == b["counters"]


# ---------------------------------------------------------------- golden ---

def _load_fixture(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_golden_fixtures():
    for name in sorted(os.listdir(GOLDEN)):
        if not name.endswith(".json") or name.startswith("config"):
            continue
        fx = _load_fixture(name)
        g = W.Graph(name, fx["n"], fx["n_labels"], np.array(fx["src"], np.int32),
                    np.array(fx["dst"], np.int32), np.array(fx["lab"], np.int32))
        for case in fx["cases"]:
            nfa = compile_regex(case["regex"], fx["n_labels"])
            r = answer(g, nfa, case["source"], case.get("max_levels", 0))
            assert as_set(r["answer"]) == set(case["answer"]), (name, case)


def test_golden_config1():
    """The small ER workload: answer written by tests/golden/make_golden.py
    (which calls only the oracle); the generator is bit-identical across
    machines, so the stored answer pins both."""
    fx = _load_fixture("config1_answer.json")
    w = W.config1()
    g = w.graph
    q = w.queries[0]
    r = answer(g, compile_regex(q.regex, g.n_labels), q.source)
    assert r["answer"].tolist() == fx["answer"]
    assert r["counters"] == fx["counters"]


# ------------------------------------------------------ sets of sources ----
# The 2-RPQ of section 2 takes a set of starting vertices V_s; level 0 is
# then Q_S x V_s.

@pytest.mark.parametrize("seed", range(40))
def test_source_set_vs_bruteforce(seed):
    """Brute force from the definition with 2-paths starting anywhere in V_s
    (repeats allowed in the list), per word-length bound k."""
    g = W.tiny_graph(seed + 900)
    S, trans, starts, finals = W.tiny_automaton(seed + 1900, g.n_labels)
    nfa = nfa_from_lists(S, trans, starts, finals, g.n_labels)
    r = W.below(seed, 12, 4, 1 << 20)
    srcs = [int(x % g.n) for x in r[: 1 + seed % 4]]
    og = O.OracleGraph(g.n, g.n_labels, g.src, g.dst, g.lab)
    K = 5
    bf = O.brute_force_levels(g.n, g.n_labels, g.src, g.dst, g.lab, srcs, nfa.accepts, K)
    for k in range(1, K + 1):
        assert as_set(og.query(nfa, srcs, k)["answer"]) == as_set(bf[k]), (k, srcs)
    og.close()


@pytest.mark.parametrize("seed", range(20))
def test_source_set_is_union_of_single_sources(seed):
    """Ans(V_s) = union over v in V_s of Ans(v), at every level bound."""
    g = W.rmat_graph(7, 500, 3, seed=seed + 60)
    text, _, _ = W.random_regex(seed + 61, 3, 3)
    nfa = compile_regex(text, 3)
    og = O.OracleGraph(g.n, 3, g.src, g.dst, g.lab)
    srcs = W.below(seed, 13, 5, g.n).tolist()
    for k in (0, 1, 3):
        union = set()
        for s in srcs:
            union |= as_set(og.ssr(nfa, s, k)["answer"])
        assert as_set(og.query(nfa, srcs, k)["answer"]) == union, (text, k)
    assert og.query(nfa, [], 0)["answer"].size == 0  # no source: nothing is reached
    og.close()


# ------------------------------------------------- level of first reach ----
# The smallest k such that v is in the answer restricted to words of length
# <= k: the length of a shortest accepted word labelling a 2-path to v.

@pytest.mark.parametrize("seed", range(40))
def test_first_level_vs_bruteforce(seed):
    g = W.tiny_graph(seed + 1300)
    S, trans, starts, finals = W.tiny_automaton(seed + 2300, g.n_labels)
    nfa = nfa_from_lists(S, trans, starts, finals, g.n_labels)
    srcs = [seed % g.n] if seed % 2 else [seed % g.n, (seed * 5 + 1) % g.n]
    og = O.OracleGraph(g.n, g.n_labels, g.src, g.dst, g.lab)
    K = 5
    bf = O.brute_force_levels(g.n, g.n_labels, g.src, g.dst, g.lab, srcs, nfa.accepts, K)
    exp = O.first_levels_from(bf, g.n)
    got = og.query(nfa, srcs, 0, want_first_level=True)
    fl = got["first_level"]
    for v in range(g.n):
        if exp[v] >= 0:
            assert fl[v] == exp[v], (v, srcs, trans, starts, finals)
        else:  # not reached within K symbols: later or never
            assert fl[v] == -1 or fl[v] > K, (v, fl[v])
    assert as_set(np.flatnonzero(fl >= 0)) == as_set(got["answer"])
    og.close()


def test_first_level_closed_forms():
    # a* on a chain 0 -> 1 -> ... -> 9 from 3: vertex 3 + i first at level i
    m, s = 10, 3
    src = np.arange(m - 1, dtype=np.int32)
    dst = src + 1
    lab = np.zeros(m - 1, np.int32)
    og = O.OracleGraph(m, 1, src, dst, lab)
    fl = og.ssr(compile_regex("0*", 1), s, want_first_level=True)["first_level"]
    assert fl.tolist() == [-1] * s + list(range(m - s))
    # ^0* from 6 walks the chain backwards
    fl = og.ssr(compile_regex("^0*", 1), 6, want_first_level=True)["first_level"]
    assert fl.tolist() == [6, 5, 4, 3, 2, 1, 0, -1, -1, -1]
    og.close()
    # a* on a directed cycle of length 7 from 2: (v - 2) mod 7
    n = 7
    src = np.arange(n, dtype=np.int32)
    dst = (src + 1) % n
    og = O.OracleGraph(n, 1, src, dst, np.zeros(n, np.int32))
    fl = og.ssr(compile_regex("0*", 1), 2, want_first_level=True)["first_level"]
    assert fl.tolist() == [(v - 2) % n for v in range(n)]
    # (0/0)* on the cycle: even word lengths only, so v is first reached at
    # the smallest even length congruent to (v - 2) mod 7
    fl = og.ssr(compile_regex("(0/0)*", 1), 2, want_first_level=True)["first_level"]
    assert fl.tolist() == [d if d % 2 == 0 else d + 7 for d in ((v - 2) % n for v in range(n))]
    # from the set {0, 4}: the nearer source decides
    fl = og.query(compile_regex("0*", 1), [0, 4], want_first_level=True)["first_level"]
    assert fl.tolist() == [min(v % n, (v - 4) % n) for v in range(n)]
    og.close()


# ------------------------------------------------------------ witnesses ----

def test_check_witness_accepts_valid_and_rejects_broken_paths():
    # edges 0 -a-> 1 -b-> 2, 3 -a-> 2 (a = 0, b = 1, L = 2)
    src, dst, lab = [0, 1, 3], [1, 2, 2], [0, 1, 0]
    acc = compile_regex("0/1/^0", 2).accepts
    ok = lambda vs, ws, t=3, s=(0,): O.check_witness(4, 2, src, dst, lab, acc, s, t, vs, ws)[0]
    assert ok([0, 1, 2, 3], [0, 1, 2])            # a, b, then a backwards from 2 to 3
    assert not ok([0, 1, 2, 3], [0, 1, 0])        # 2 -a-> 3 is not an edge
    assert not ok([1, 2, 3], [1, 2], s=(0,))      # does not start at the source
    assert ok([1, 2, 3], [1, 2], s=(0, 1)) is False  # starts at a source, word not accepted
    assert not ok([0, 1, 2], [0, 1], t=2)         # word a.b not accepted
    assert not ok([0, 1, 2, 3], [0, 1])           # lengths do not pair up
    assert not ok([0, 1, 2, 3], [0, 1, 2], t=2)   # does not end at the target
