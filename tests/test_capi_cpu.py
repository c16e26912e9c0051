"""Host-side checks of librpq.so that need no GPU: the library loads, exports
every function include/rpq.h declares, and its regex compiler (host code)
accepts exactly the language of the oracle's Thompson automaton."""

import itertools
import os
import re

import pytest

from oracle.regex_nfa import compile_regex as oracle_compile
from paper_2412_10287_gb300 import build as B
from paper_2412_10287_gb300 import rpq as R
from paper_2412_10287_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def header_functions():
    text = open(os.path.join(ROOT, "include", "rpq.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rpq_[a-z_]+)\s*\(", text)))


def test_header_symbols_exported():
    names = header_functions()
    assert len(names) >= 20
    assert set(names) == set(R.EXPORTED)
    L = R.lib()
    for n in names:
        assert hasattr(L, n), n


def test_kernel_launch_counter_without_gpu():
    """The launch counter needs no device: compiling automata launches
    nothing, so it does not move."""
    a = R.rpq_kernel_launches()
    R.rpq_nfa_compile("0/1*", 2)
    assert R.rpq_kernel_launches() == a >= 0


def test_version_and_errors():
    assert R.rpq_version().count(".") == 2
    with pytest.raises(R.RpqError) as e:
        R.rpq_nfa_compile("(0|", 2)
    assert e.value.status == R.RPQ_ERR_PARSE
    assert "regex" in R.rpq_last_error()
    with pytest.raises(R.RpqError) as e:
        R.rpq_nfa_compile("5", 2)
    assert e.value.status == R.RPQ_ERR_INVALID
    with pytest.raises(R.RpqError):
        R.rpq_nfa_from_transitions(65, 1, [], [0], [0])
    with pytest.raises(R.RpqError):
        R.rpq_nfa_from_transitions(2, 1, [(0, 2, 1)], [0], [1])  # label 2 >= 2L


@pytest.mark.parametrize("seed", range(60))
def test_compiled_dfa_language_matches_oracle(seed):
    """Language equality with the oracle's Thompson NFA on all words of
    length <= 6 over <= 3 labels and their inverses (<= 5 for 3 labels)."""
    L = 1 + seed % 3
    text, _, _ = W.random_regex(seed + 9000, L, depth=1 + seed % 4)
    dfa = R.rpq_nfa_compile(text, L)
    ref = oracle_compile(text, L)
    S, T, _ = dfa.info()
    assert 1 <= S <= 64
    ex = dfa.export()
    # determinism of the compiled automaton: at most one target per (q, a)
    pairs = list(zip(ex["from"].tolist(), ex["label"].tolist()))
    assert len(pairs) == len(set(pairs))
    assert ex["starts"] == [0]
    maxlen = 6 if L <= 2 else 5
    for k in range(maxlen + 1):
        for w in itertools.product(range(2 * L), repeat=k):
            assert dfa.accepts(w) == ref.accepts(w), (text, w)


def test_compiled_dfa_is_minimal_on_known_cases():
    # a* -> 1 state; a.b* -> 2 states; (a|b)*.c -> 2 states; chain of k -> k+1
    assert R.rpq_nfa_compile("0*", 3).info()[0] == 1
    assert R.rpq_nfa_compile("0/1*", 3).info()[0] == 2
    assert R.rpq_nfa_compile("(0|1)*/2", 3).info()[0] == 2
    assert R.rpq_nfa_compile("0/1/2/0/1", 3).info()[0] == 6
    assert R.rpq_nfa_compile("(0/1)*", 3).info()[0] == 2
    # a finite language of two words, 0.0^-.1 and 0.0^-.2: a chain of three
    # states and one final state reached by either last symbol
    d = R.rpq_nfa_compile("0/^0/(1|2)", 3)
    S, T, _ = d.info()
    assert (S, T) == (4, 4)
    e = d.export()
    assert e["starts"] == [0] and e["finals"] == [3]
    accepted = [w for k in range(5) for w in itertools.product(range(6), repeat=k) if d.accepts(w)]
    assert accepted == [(0, 3, 1), (0, 3, 2)]
    # 0?: the empty word and "0"; both states final
    e = R.rpq_nfa_compile("0?", 1).export()
    assert e["n_states"] == 2 and e["finals"] == [0, 1]
    assert e["from"].tolist() == [0] and e["label"].tolist() == [0] and e["to"].tolist() == [1]


def test_reverse_automaton_language():
    L = 2
    for seed in range(10):
        text, _, _ = W.random_regex(seed + 700, L, 3)
        a = R.rpq_nfa_compile(text, L)
        r = R.rpq_nfa_reverse(a)
        for k in range(5):
            for w in itertools.product(range(2 * L), repeat=k):
                inv = [s + L if s < L else s - L for s in reversed(w)]
                assert r.accepts(w) == a.accepts(inv)


def test_too_many_states_rejected():
    # a chain of 70 labels has 71 states after minimisation
    with pytest.raises(R.RpqError):
        R.rpq_nfa_compile("/".join(["0"] * 70), 1)


def test_answer_copy_small_and_threaded():
    """The binding's copy of a host answer out of the library's buffer: the
    plain copy below the threshold and the threaded one above it return the
    same entries in fresh memory."""
    import ctypes

    import numpy as np

    for n in (0, 1, 1000, R._PARALLEL_COPY_MIN - 1, R._PARALLEL_COPY_MIN,
              3 * R._PARALLEL_COPY_MIN + 7):
        src = np.arange(n, dtype=np.int32)[::-1].copy()
        ptr = src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        got = R._copy_answer(ptr, n)
        assert got.dtype == np.int32 and got.shape == (n,)
        assert (got == src).all()
        if n:
            assert not np.shares_memory(got, src)
