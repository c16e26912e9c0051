"""Multi-rank host logic of the benchmark on CPU ranks (gloo, world size 2).

Queries are independent, so N GPUs run N query sets with no collective on
the data path (weak scaling): rank 0 runs the workload's own queries, every
other rank an equally sized set of its own.  The job's time is the slowest
rank's, taken by one all-reduce.  Each rank here answers its set with the
oracle and the parent checks what was gathered."""

import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _graph():
    from paper_2412_10287_gb300 import workloads as W

    return W.rmat_graph(10, 6000, 8, seed=5)


def _answers(g, qs):
    from oracle import oracle as O
    from oracle.regex_nfa import compile_regex

    og = O.OracleGraph(g.n, g.n_labels, g.src, g.dst, g.lab)
    return [[q.regex, q.source, og.ssr(compile_regex(q.regex, g.n_labels), q.source)["answer"].tolist()]
            for q in qs]


def _rank_main(rank, world, port, outdir):
    import sys

    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        g = _graph()
        qs = bench.rank_queries(g, "rmat20", 2, rank)
        mine = _answers(g, qs)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        slowest = bench.max_over_ranks(0.25 + rank, dist)
        with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
            json.dump({"gathered": gathered, "slowest": slowest}, f)
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks_shard_queries_and_take_the_slowest_time(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    import bench
    from paper_2412_10287_gb300 import workloads as W

    g = _graph()
    sets = [bench.rank_queries(g, "rmat20", 2, r) for r in range(world)]
    # rank 0 runs the workload's own queries; rank 1 a different set of the same size
    own = W.make_queries(g, W.TEMPLATES_SMALL, 2, seed=1, zipf_s=1.0)
    assert [(q.regex, q.source) for q in sets[0]] == [(q.regex, q.source) for q in own]
    assert len(sets[1]) == len(sets[0])
    assert [(q.regex, q.source) for q in sets[1]] != [(q.regex, q.source) for q in sets[0]]
    expect = [_answers(g, qs) for qs in sets]
    for r in range(world):
        with open(tmp_path / f"rank{r}.json") as f:
            got = json.load(f)
        assert got["gathered"] == expect  # every rank sees every rank's answers
        assert got["slowest"] == pytest.approx(0.25 + world - 1)
