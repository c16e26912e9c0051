"""Failure paths that can be exercised without faulting the GPU.

* A device wait that runs out: every wait of the query kernel on other CTAs
  (grid barrier, gate, parking) has a limit, after which the kernel records
  RPQ_ERR_TIMEOUT and returns.  The test shortens the limit and has one CTA
  leave the kernel early (a barrier arrival that never comes), checks the
  status, and then checks that the next query on the same graph -- whose
  workspace the failed launch left dirty -- answers exactly.
* A device allocation that fails: a host-side allocator with a byte cap is
  installed through rpq_set_allocator; the call fails with RPQ_ERR_OOM and
  the library keeps working once memory is available.  The server puts a
  query whose allocation failed beside others back in its queue and admits
  fewer at once; every answer still equals the oracle's.
"""

import threading

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


def load(g):
    return R.rpq_graph_load(g.n, g.n_labels, g.src, g.dst, g.lab)


def test_wait_limit_runs_out_and_the_next_query_answers(monkeypatch):
    g = W.rmat_graph(14, 1 << 18, 4, seed=131)
    gg = load(g)
    og = O.OracleGraph(g.n, 4, g.src, g.dst, g.lab)
    text = "(0|1|2|3)*"
    nfa = R.rpq_nfa_compile(text, 4)
    src = int(W.below(132, 1, 1, g.n)[0])
    exp = og.ssr(oracle_compile(text, 4), src)["answer"].tolist()
    assert len(exp) > 1000  # grid levels: the leaving CTA is waited for
    monkeypatch.setenv("RPQ_SOLO_MASS", "-1")  # every level on the whole grid
    monkeypatch.setenv("RPQ_WAIT_LIMIT_MS", "100")
    monkeypatch.setenv("RPQ_TEST_LEAVE_CTA", "1")
    for _ in range(2):
        with pytest.raises(R.RpqError) as e:
            R.rpq_query(gg, nfa, src)
        assert e.value.status == R.RPQ_ERR_TIMEOUT
    monkeypatch.delenv("RPQ_TEST_LEAVE_CTA")
    assert R.rpq_query(gg, nfa, src).tolist() == exp
    monkeypatch.delenv("RPQ_SOLO_MASS")
    assert R.rpq_query(gg, nfa, src).tolist() == exp
    og.close()


class CappedAllocator:
    """Device memory from PyTorch's caching allocator, refused beyond `cap`
    bytes in use (thread-safe: the library calls it from worker threads)."""

    def __init__(self, cap):
        import torch

        self.torch = torch
        self.cap = cap
        self.used = 0
        self.refused = 0
        self.sizes = {}
        self.mu = threading.Lock()

    def alloc(self, size):
        with self.mu:
            if self.used + size > self.cap:
                self.refused += 1
                return 0
            p = self.torch.cuda.caching_allocator_alloc(size, 0)
            self.used += size
            self.sizes[p] = size
            return p

    def free(self, p):
        with self.mu:
            self.used -= self.sizes.pop(p)
        self.torch.cuda.caching_allocator_delete(p)


@pytest.fixture
def capped():
    a = CappedAllocator(1 << 62)
    R.rpq_set_allocator(a.alloc, a.free)
    yield a
    R.rpq_set_allocator()


def test_allocation_failure_returns_oom_and_recovers(capped):
    g = W.rmat_graph(13, 60000, 4, seed=141)
    gg = load(g)
    og = O.OracleGraph(g.n, 4, g.src, g.dst, g.lab)
    graph_bytes = capped.used
    capped.cap = graph_bytes + 4096  # no room for a query workspace
    nfa = R.rpq_nfa_compile("1/0*", 4)
    with pytest.raises(R.RpqError) as e:
        R.rpq_query(gg, nfa, 5)
    assert e.value.status == R.RPQ_ERR_OOM and capped.refused > 0
    assert capped.used == graph_bytes  # the partial workspace went back
    capped.cap = 1 << 62
    assert R.rpq_query(gg, nfa, 5).tolist() == og.ssr(oracle_compile("1/0*", 4), 5)["answer"].tolist()
    gg.close()
    assert capped.used == 0
    og.close()


def test_server_backs_off_after_allocation_failures(capped):
    g = W.rmat_graph(13, 60000, 4, seed=151)
    gg = load(g)
    og = O.OracleGraph(g.n, 4, g.src, g.dst, g.lab)
    graph_bytes = capped.used
    # the size of one query workspace, from a probe graph of the same shape
    probe = load(W.rmat_graph(13, 60000, 4, seed=152))
    before = capped.used
    R.rpq_query(probe, R.rpq_nfa_compile("0*", 4), 0)
    ws_bytes = capped.used - before
    probe.close()
    assert ws_bytes > 0
    capped.cap = graph_bytes + int(2.5 * ws_bytes)  # two workspaces fit, not eight
    texts = ["0*", "1/0*", "(0|1)*/2", "^0/1*"]
    srcs = W.below(153, 1, 64, g.n).tolist()
    srv = R.Server(gg, max_lanes=8, engine=0)
    try:
        tickets = [srv.submit(R.rpq_nfa_compile(texts[i % 4], 4), s) for i, s in enumerate(srcs)]
        srv.drain(120000)
        for i, (t, s) in enumerate(zip(tickets, srcs)):
            exp = og.ssr(oracle_compile(texts[i % 4], 4), s)["answer"].tolist()
            assert srv.poll(t).tolist() == exp, i
        st = srv.stats()
        assert st["completed"] == 64
        assert capped.refused > 0 and st["oom_retries"] > 0
    finally:
        srv.close()
        gg.close()  # its memory goes back through the capped allocator
        og.close()
