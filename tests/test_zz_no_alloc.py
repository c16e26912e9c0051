"""The no-allocation query entry point (rpq_query_noalloc).

Some callers cannot allocate device memory while they run -- their GPU
memory belongs to another allocator or must stay fixed after start-up -- so
the library offers one query call whose workspace is a fixed array reserved
when the library is loaded.  This file checks, through the C ABI, that it
returns exactly what rpq_query returns and what the CPU oracle returns, on
two calls in a row (the array is reused, so the second call must not see
the first one's state), and that a query too large for the array is
refused with a clear error.  It is
collected last so that a run stopping at the first failure has already run
every other test.
"""

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


def test_noalloc_matches_rpq_query_on_two_calls_in_a_row():
    import torch

    g = W.rmat_graph(16, 1 << 20, 4, seed=61)
    gg = R.rpq_graph_load(g.n, g.n_labels, g.src, g.dst, g.lab)
    og = O.OracleGraph(g.n, g.n_labels, g.src, g.dst, g.lab)
    out = torch.full((g.n,), -1, dtype=torch.int32, device="cuda")
    cases = [("0/1*", 5), ("(0|^2)+", 77)]
    srcs = W.below(62, 1, 2, g.n).tolist()
    for (text, _), s in zip(cases, srcs):
        nfa = R.rpq_nfa_compile(text, g.n_labels)
        expected = R.rpq_query(gg, nfa, s)
        oracle = og.ssr(oracle_compile(text, g.n_labels), s)["answer"].tolist()
        cnt = R.rpq_query_noalloc(gg, nfa, s, out)
        assert cnt == expected.size
        assert out[:cnt].cpu().numpy().tolist() == expected.tolist() == oracle
    # the same query twice more, now with a level cap, after a different one
    nfa = R.rpq_nfa_compile(cases[0][0], g.n_labels)
    for k in (2, 0):
        expected = R.rpq_query(gg, nfa, srcs[0], k)
        oracle = og.ssr(oracle_compile(cases[0][0], g.n_labels), srcs[0], k)["answer"].tolist()
        cnt = R.rpq_query_noalloc(gg, nfa, srcs[0], out, max_levels=k)
        assert out[:cnt].cpu().numpy().tolist() == expected.tolist() == oracle
    og.close()


def test_noalloc_refuses_queries_larger_than_its_scratch():
    import torch

    n = 4_000_000
    g = W.Graph("wide", n, 2, np.arange(10, dtype=np.int32), np.arange(1, 11, dtype=np.int32),
                np.zeros(10, np.int32))
    gg = R.rpq_graph_load(g.n, g.n_labels, g.src, g.dst, g.lab)
    nfa = R.rpq_nfa_compile("0/0/0/0/0/0/0/1", 2)  # 9 states: ~450 MB of workspace
    out = torch.empty(16, dtype=torch.int32, device="cuda")
    with pytest.raises(R.RpqError) as e:
        R.rpq_query_noalloc(gg, nfa, 0, out)
    assert e.value.status == R.RPQ_ERR_INVALID
    assert "scratch" in str(e.value)
    # host output memory is refused as well
    host = np.zeros(4, np.int32)
    cnt = R.ctypes.c_int64()
    status = R.lib().rpq_query_noalloc(gg.h, nfa.h, 0, 0, R._ptr(host), 4, R.ctypes.byref(cnt),
                                       None)
    assert status == R.RPQ_ERR_INVALID
