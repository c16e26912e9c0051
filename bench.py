#!/usr/bin/env python
"""Benchmark: single-source 2-RPQ queries/s on one GB300 (or N replicas).

Default workload ``kb20m``, the largest single-GPU configuration: a
knowledge-base-shaped Chung-Lu graph (20,000,000 vertices, 200,000,000
edges, out-degree exponent 2.1, 500 labels with Zipf(1.1) frequencies,
seed 2) and 200 single-source queries (8 templates x 25 random sources with
non-zero degree: a.b*.c, (a|b^-)+, a*.b*, chains, (a.b)*, a.(b|c^-)*.d),
run one at a time as in the paper's evaluation (section 5.3: data
preloaded, sequential isolated queries).

One step = those 200 queries.  ``value`` = queries/s with the graph and the
outputs resident on the device (rpq_query with a device output buffer,
CUDA events on the launching stream around each step, L2 flushed between
steps).  ``e2e`` = the same queries through the public API with host
output buffers and regex compilation inside the timed region.  The roofline
object refers to the traversal kernel (one cooperative launch per query).

The same line carries, under ``extras``, the other configurations on the
R-MAT scale-20 graph: 400 single queries one at a time (``rmat20``), 256
mixed queries per rpq_query_batch call against the same queries one at a
time (``batch``), and a Poisson stream of 2,000 queries/s through the
server against the unbatched served loop (``serve``).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload kb20m|rmat20|batch|serve] [--no-extras]
"""

from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

HBM_FALLBACK_GBS = 6800.0
PROFILE_JSON = os.path.join(ROOT, "profiles", "rpq_query_kernel_kb20m.json")
KERNEL_SOURCE = os.path.join(ROOT, "paper_2412_10287_gb300", "csrc", "query.cu")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--per-template", type=int, default=None,
                    help="sources per template (default: 25 on kb20m, 100 on rmat20)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="CPU work budget of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="kb20m", choices=["kb20m", "rmat20", "batch", "serve"],
                    help="kb20m: single queries on the 20M-vertex knowledge-base graph (the "
                         "default line); rmat20: single queries on the R-MAT scale-20 graph; "
                         "batch: 256 mixed queries per launch; serve: Poisson arrivals through "
                         "the server")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave out the rmat20 / batch / serve figures of the default line")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--one-query", default=None,
                    help="profiling case: run this regex once for warm-up and once more "
                         "(with --source) on the workload's graph, print its counters, exit")
    ap.add_argument("--source", type=int, default=0)
    ap.add_argument("--kb-size", default=None, metavar="N,M",
                    help="with --one-query: a knowledge-base graph of N vertices and M edges "
                         "(same generator and seed as kb20m) instead of the workload's graph")
    ap.add_argument("--profile-sample", type=int, default=0, metavar="N",
                    help="profiling case: run the workload's queries once, then again only "
                         "the N with the most algorithmic bytes (the launches to capture), "
                         "and write their algorithmic bytes to --sample-out; exit")
    ap.add_argument("--sample-out", default="gpurun_out/profile_sample.json")
    ap.add_argument("--sample-json", default=None,
                    help="with --write-profile: the --profile-sample file of the capture")
    ap.add_argument("--write-profile", default=None, metavar="NCU_CSV",
                    help="read an ncu CSV of traversal-kernel launches taken with --metrics "
                         "dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum and "
                         "write the per-launch DRAM traffic file of --workload, then exit")
    return ap.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def sha256(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def profile_traffic(alg_bytes_per_launch=None):
    """Per-launch DRAM bytes of the traversal kernel from the committed ncu
    summary, or None if absent or taken on a different kernel source.  A
    summary taken on a sample of launches holds their DRAM bytes per
    algorithmic byte; that ratio times `alg_bytes_per_launch` (this run's
    mean) is the traffic of a mean launch."""
    try:
        with open(PROFILE_JSON) as f:
            pj = json.load(f)
        if pj.get("kernel_source_sha256") != sha256(KERNEL_SOURCE):
            return None
        ratio = pj.get("dram_per_algorithmic_byte")
        if ratio is not None and alg_bytes_per_launch is not None:
            return ratio * alg_bytes_per_launch
        return pj.get("dram_bytes_per_launch")
    except Exception:
        return None


UNIT_SCALE = {"": 1.0, "k": 1e3, "K": 1e3, "M": 1e6, "G": 1e9, "T": 1e12,
              "n": 1e-9, "u": 1e-6, "m": 1e-3}


def ncu_value(unit, value):
    """A metric value of an ncu CSV in base units (bytes, seconds)."""
    v = float(str(value).replace(",", ""))
    u = unit.strip()
    for base in ("byte", "second", "s"):
        if u.endswith(base):
            return v * UNIT_SCALE.get(u[: -len(base)], 1.0)
    return v


def write_profile(csv_path, workload_name, sample_json=None):
    """Per-launch DRAM bytes and ncu durations of the traversal kernel, from an
    ncu CSV, written beside the kernel source's hash so that a later change
    to the kernel voids the figure.  With `sample_json` (written by
    --profile-sample: the algorithmic bytes of each captured launch, in
    launch order) the summary also holds DRAM bytes per algorithmic byte
    over the sample, which scales the traffic to any run's mean launch."""
    import csv

    launches = {}
    with open(csv_path, newline="") as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for row in csv.DictReader(lines):
        if "rpq_query_kernel" not in row.get("Kernel Name", ""):
            continue
        d = launches.setdefault(row["ID"], {})
        d[row["Metric Name"]] = ncu_value(row.get("Metric Unit", ""), row["Metric Value"])
    ids = sorted(launches, key=lambda k: int(k))
    per = [launches[k] for k in ids
           if "dram__bytes_read.sum" in launches[k] and "dram__bytes_write.sum" in launches[k]]
    if not per:
        raise SystemExit(f"no rpq_query_kernel launches with DRAM metrics in {csv_path}")
    rd = sum(d["dram__bytes_read.sum"] for d in per) / len(per)
    wr = sum(d["dram__bytes_write.sum"] for d in per) / len(per)
    dur = [d["gpu__time_duration.sum"] for d in per if "gpu__time_duration.sum" in d]
    out = {
        "kernel": "rpq_query_kernel", "workload": workload_name, "launches": len(per),
        "kernel_source_sha256": sha256(KERNEL_SOURCE),
        "dram_bytes_per_launch": rd + wr, "dram_read_bytes_per_launch": rd,
        "dram_write_bytes_per_launch": wr,
        "ncu_ms_per_launch": (sum(dur) / len(dur) * 1e3) if dur else None,
        "note": "ncu flushes caches before each profiled launch: cold-cache figures",
    }
    if sample_json:
        with open(sample_json) as f:
            sj = json.load(f)
        alg = sj["algorithmic_bytes"]
        if len(alg) != len(per):
            raise SystemExit(f"{len(per)} captured launches, {len(alg)} sample queries")
        dram = [d["dram__bytes_read.sum"] + d["dram__bytes_write.sum"] for d in per]
        out["sample"] = sj.get("sample")
        out["sample_algorithmic_bytes_per_launch"] = sum(alg) / len(alg)
        out["sample_push_bytes_per_launch"] = sum(sj["push_bytes"]) / len(alg)
        out["dram_per_algorithmic_byte"] = sum(dram) / sum(alg)
        out["dram_per_push_byte"] = sum(dram) / max(1, sum(sj["push_bytes"]))
    path = os.path.join(ROOT, "profiles", f"rpq_query_kernel_{workload_name}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out))


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.remove(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def workload(per_template, name="kb20m"):
    from paper_2412_10287_gb300 import workloads as W

    if name == "kb20m":
        return W.config3(per_template=per_template)
    return W.config2(per_template=per_template)


# query templates, seed and label skew of each single-query workload
QUERY_SPECS = {"rmat20": ("TEMPLATES_SMALL", 1, 1.0), "kb20m": ("TEMPLATES_KB", 2, 1.1)}
# sources per template of each single-query workload (one step)
PER_TEMPLATE = {"rmat20": 100, "kb20m": 25}


def per_template_for(name, requested=None):
    return requested if requested else PER_TEMPLATE[name]


def rank_queries(g, name, per_template, rank):
    """The queries rank `rank` runs (weak scaling: every rank its own units).
    Rank 0 runs the workload's own queries; rank r > 0 an equally sized set
    drawn the same way with its own seed."""
    from paper_2412_10287_gb300 import workloads as W

    tpl, seed, zipf = QUERY_SPECS[name]
    return W.make_queries(g, getattr(W, tpl), per_template,
                          seed=seed if rank == 0 else seed + 7919 * rank, zipf_s=zipf)


def max_over_ranks(seconds, dist, device=None):
    """The slowest rank's time (the job's time), through one all-reduce."""
    import torch

    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_config(w, n_queries, extra=None):
    if w.name == "kb20m":
        desc = ("kb20m: Chung-Lu power-law graph, 20,000,000 vertices, 200,000,000 edges "
                "(out-degree exponent 2.1), 500 labels Zipf(1.1), seed 2; "
                f"{n_queries} single-source queries (a/b*/c, (a|^b)+, a*/b*, chains, (a/b)*, "
                "a/(b|^c)*/d), one at a time")
    else:
        desc = ("rmat20: R-MAT scale 20 (1,048,576 vertices, 2^24 edge samples, "
                "a=0.57 b=c=0.19), 8 labels Zipf(1.0), seed 1; "
                f"{n_queries} single-source queries (a*, a.b*, (a|b)*.c, a^-.b*), "
                "one at a time")
    c = {"workload": desc,
         "n_vertices": w.graph.n, "n_edge_samples": w.graph.m, "n_labels": w.graph.n_labels,
         "queries_per_step": n_queries,
         "l2": "flushed between steps (256 MiB write)",
         "timing": ("value, ms_per_step and latencies from the timed steps, queries without "
                    "per-query statistics; roofline, product edges and bytes from as many "
                    "further steps of the same queries with the library's statistics (CUDA "
                    "events around every launch)"),
         "parallelism": "replicas (query-sharded, no collective)"}
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------- CPU oracle ----

def autotune(R, gg, g, name):
    """The push/pull threshold picked by the library's autotuner on a sample
    of queries drawn apart from the timed ones (other seed), before timing."""
    from paper_2412_10287_gb300 import workloads as W

    tpl = W.TEMPLATES_KB if name == "kb20m" else W.TEMPLATES_SMALL
    sample = W.make_queries(g, tpl, 4, seed=99, zipf_s=1.1 if name == "kb20m" else 1.0)
    alpha, mn, solo = R.rpq_graph_autotune(gg, [R.rpq_nfa_compile(q.regex, g.n_labels)
                                                 for q in sample], [q.source for q in sample])
    return {"pull_alpha": alpha, "pull_min": mn, "solo_mass": solo,
            "sample": f"{len(sample)} queries of the same templates, seed 99"}


def oracle_graph(w):
    from oracle import oracle as O

    g = w.graph
    return O.OracleGraph(g.n, g.n_labels, g.src, g.dst, g.lab)


def oracle_sample(w, seconds_budget, og=None, max_threads=None, offset=0):
    """Times the CPU oracle (as it stands) on a bounded sample of the
    workload's queries, on the host cores (one query per thread).  The
    sample walks the queries in a fixed interleaved order (every template
    in turn), starting at `offset`; a query is submitted only while the
    elapsed time is under `seconds_budget` (the first one always), so the
    wall time is the budget plus at most the queries still running then.  Returns queries/s over
    the queries done and what the sample was."""
    from oracle.regex_nfa import compile_regex

    g = w.graph
    own = og is None
    if own:
        og = oracle_graph(w)
    threads = max_threads or len(os.sched_getaffinity(0))
    qs = w.queries
    # interleaved order: query k of template 0, of template 1, ... then k+1
    by_tpl = {}
    for q in qs:
        by_tpl.setdefault(q.template, []).append(q)
    order = [lst[k] for k in range(max(len(v) for v in by_tpl.values()))
             for lst in by_tpl.values() if k < len(lst)]
    order = order[offset % len(order):] + order[:offset % len(order)]
    done = []
    t0 = time.perf_counter()

    def run(q):
        og.ssr(compile_regex(q.regex, g.n_labels), q.source)
        return q

    it = iter(order)
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        running = set()
        while True:
            while len(running) < threads and (time.perf_counter() - t0 < seconds_budget
                                              or not (done or running)):
                q = next(it, None)
                if q is None:
                    break
                running.add(ex.submit(run, q))
            if not running:
                break
            fin, running = cf.wait(running, return_when=cf.FIRST_COMPLETED)
            done.extend(f.result() for f in fin)
    wall = time.perf_counter() - t0
    if own:
        og.close()
    return {"value": len(done) / wall, "unit": "queries/s", "cores": threads, "kind": "oracle",
            "queries": len(done), "wall_s": wall,
            "sample": f"{len(done)} of the {len(qs)} queries (templates interleaved, from "
                      f"position {offset % len(order)}), {threads} threads, one query per "
                      f"thread; adjacency lists built before timing; {wall:.1f} s wall"}


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on the same workload,
    metric and unit as the GPU line, each step a bounded sample."""
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    name = args.workload if args.workload in QUERY_SPECS else "kb20m"
    w = workload(per_template_for(name, args.per_template), name)
    og = oracle_graph(w)
    per_step = max(2.0, min(20.0, 100.0 / max(1, args.steps + args.warmup)))
    vals = []
    offset = 0
    for i in range(args.warmup + args.steps):
        r = oracle_sample(w, per_step, og=og, offset=offset)
        offset += r["queries"]
        if i >= args.warmup:
            vals.append(r)
    og.close()
    nq = sum(r["queries"] for r in vals)
    wall = sum(r["wall_s"] for r in vals)
    v = nq / wall
    line = {"impl": "reference", "metric": "rpq_queries_per_s", "value": v, "unit": "queries/s",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * wall / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": workload_config(w, len(w.queries),
                                      {"note": "CPU oracle; each step a bounded sample of the "
                                               f"workload's queries ({per_step:.0f} s budget); "
                                               "ms_per_step is the wall time of the samples run"}),
            "cpu_baseline": {"value": v, "unit": "queries/s", "cores": vals[-1]["cores"],
                             "kind": "oracle",
                             "sample": f"{nq} queries over {len(vals)} timed steps; last step: "
                                       + vals[-1]["sample"]},
            "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------ batch / serve ----

def run_batch(args, R, torch, g=None, gg=None):
    """256 mixed queries (2-12 DFA states) per rpq_query_batch call against
    the same 256 queries run one at a time.  Returns the figures."""
    import ctypes

    from paper_2412_10287_gb300 import workloads as W

    g = g or W.config2_graph()
    w = W.config4(g, 256)
    gg = gg or R.rpq_graph_load(g.n, g.n_labels, g.src, g.dst, g.lab)
    # the lane engine's tuning (inline row length, pull divisor) on a sample
    # drawn apart from the timed queries: one automaton from 64 sources of
    # another seed (the shared-automaton batches lanes serve)
    tune_srcs = W.below(33, 1, 64, g.n).tolist()
    lane_hub, lane_pull = R.rpq_graph_autotune_batch(
        gg, [R.rpq_nfa_compile("0*", g.n_labels)] * 64, tune_srcs)
    nfas = [R.rpq_nfa_compile(q.regex, g.n_labels) for q in w.queries]
    srcs = [q.source for q in w.queries]
    states = [n.info()[0] for n in nfas]
    res = R.rpq_query_batch(gg, nfas, srcs)  # warm-up, sizes the output
    total = sum(a.size for a in res)
    out = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
    offs = np.zeros(len(nfas) + 1, np.int64)
    handles = (ctypes.c_void_p * len(nfas))(*[x.h.value for x in nfas])
    src_arr = np.array(srcs, np.int32)
    stream = torch.cuda.current_stream()

    def batch_once():
        s = R.lib().rpq_query_batch(gg.h, len(nfas), handles, R._ptr(src_arr), 0, R._ptr(offs),
                                    R._ptr(out), out.numel(), None,
                                    ctypes.c_void_p(stream.cuda_stream))
        assert s == 0, R.rpq_last_error()

    one = torch.empty(g.n, dtype=torch.int32, device="cuda")

    def seq_once():
        for nfa, s in zip(nfas, srcs):
            R.rpq_query(gg, nfa, s, out=one, stream=stream)

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        batch_once()
        seq_once()
    tb, ts = [], []
    batch_launches = 0
    for _ in range(args.steps):
        for fn, acc in ((batch_once, tb), (seq_once, ts)):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k0 = R.rpq_kernel_launches()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if fn is batch_once:
                batch_launches += R.rpq_kernel_launches() - k0
            acc.append(e0.elapsed_time(e1) / 1000.0)
    qb = len(nfas) * args.steps / sum(tb)
    qs = len(nfas) * args.steps / sum(ts)
    # the same batch forced onto bit lanes, and a shared-automaton batch (one
    # automaton from 256 sources: the multi-source BFS case lanes are made for)
    extra = {}
    shared = [R.rpq_nfa_compile("0*", g.n_labels)] * len(srcs)
    sh_handles = (ctypes.c_void_p * len(shared))(*[x.h.value for x in shared])
    for label, env, jobs in (("mixed_on_lanes", "lanes", None),
                             ("mixed_on_lanes_push_only", "lanes_push", None),
                             ("shared_automaton_lanes", None, "shared"),
                             ("shared_automaton_sequential", None, "shared_seq")):
        old_env = os.environ.get("RPQ_BATCH_ENGINE")
        if env:
            os.environ["RPQ_BATCH_ENGINE"] = "lanes"
        if env == "lanes_push":
            os.environ["RPQ_LANE_PULL_DIV"] = "0"
        try:
            if jobs is None:
                fn = batch_once
            else:
                sh_res = R.rpq_query_batch(gg, shared, srcs)
                sh_out = torch.empty(max(1, sum(a.size for a in sh_res)), dtype=torch.int32,
                                     device="cuda")
                if jobs == "shared":
                    def fn():
                        st_ = R.lib().rpq_query_batch(gg.h, len(shared), sh_handles,
                                                      R._ptr(src_arr), 0, R._ptr(offs),
                                                      R._ptr(sh_out), sh_out.numel(), None,
                                                      ctypes.c_void_p(stream.cuda_stream))
                        assert st_ == 0, R.rpq_last_error()
                else:
                    def fn():
                        for s_ in srcs:
                            R.rpq_query(gg, shared[0], s_, out=one, stream=stream)
            fn()
            ts_ = []
            for _ in range(args.steps):
                flush.fill_(1)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                fn()
                torch.cuda.synchronize()
                ts_.append(time.perf_counter() - t0)
            extra[label] = len(srcs) * args.steps / sum(ts_)
        finally:
            os.environ.pop("RPQ_LANE_PULL_DIV", None)
            if env:
                if old_env is None:
                    os.environ.pop("RPQ_BATCH_ENGINE", None)
                else:
                    os.environ["RPQ_BATCH_ENGINE"] = old_env
    return {"workload": "rmat20_batch: the rmat20 graph; 256 mixed queries per rpq_query_batch "
                        f"call (DFA states {min(states)}-{max(states)}); seed 3",
            "queries_per_s": qb, "ms_per_step": 1000.0 * sum(tb) / args.steps,
            "sequential_single_queries_per_s": qs, "batch_speedup": qb / qs,
            "engine": os.environ.get("RPQ_BATCH_ENGINE", "auto (slots for mixed automata)"),
            "other_engines_queries_per_s": extra,
            "lane_autotuned": {"lane_hub": lane_hub, "pull_div": lane_pull,
                               "sample": "one automaton (0*) from 64 sources of another seed"},
            "answer_vertices_per_step": int(total), "gpu_launches": batch_launches,
            "l2": "flushed between steps (256 MiB write)"}


def run_serve(args, R, torch, g=None, gg=None):
    """Poisson arrivals (2,000 q/s) replayed in real time into the server, and
    into a one-at-a-time served loop; then both at saturation.  Returns the
    figures."""
    from paper_2412_10287_gb300 import workloads as W

    g = g or W.config2_graph()
    w = W.config5(g, rate=2000.0, duration_s=args.serve_seconds, warmup_s=1.0)
    gg = gg or R.rpq_graph_load(g.n, g.n_labels, g.src, g.dst, g.lab)
    nfas = {}
    for q in w.queries:
        if q.regex not in nfas:
            nfas[q.regex] = R.rpq_nfa_compile(q.regex, g.n_labels)
    qs = w.queries
    engines = {"slots": dict(max_lanes=8, engine=0), "lanes": dict(max_lanes=256, max_states=16,
                                                                    engine=1)}
    for cfg in engines.values():  # warm-up burst
        srv = R.Server(gg, **cfg)
        for q in qs[:256]:
            srv.submit(nfas[q.regex], q.source)
        srv.drain(600000)
        srv.close()

    def served(server):
        t0 = time.perf_counter()
        tickets = []
        for q in qs:
            dt = q.arrival_s - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets.append(server.submit(nfas[q.regex], q.source))
        server.drain(600000)
        st = server.stats()
        for t in tickets:
            server.poll(t)
        return st

    served_stats = {}
    for name, cfg in engines.items():
        srv = R.Server(gg, **cfg)
        k0 = R.rpq_kernel_launches()
        served_stats[name] = served(srv)
        served_stats[name]["gpu_launches"] = R.rpq_kernel_launches() - k0
        srv.close()
    st_srv = served_stats["slots"]

    # unbatched served loop: one query at a time in arrival order
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    lat = []
    t0 = time.perf_counter()
    for q in qs:
        now = time.perf_counter() - t0
        if q.arrival_s > now:
            time.sleep(q.arrival_s - now)
        R.rpq_query(gg, nfas[q.regex], q.source, out=out, stream=stream)
        lat.append((time.perf_counter() - t0 - q.arrival_s) * 1000.0)
    span = time.perf_counter() - t0
    lat.sort()
    unb = {"qps": len(qs) / span, "p50_ms": lat[len(lat) // 2],
           "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))]}

    # saturation: everything submitted at once
    sat_n = min(len(qs), 4096)
    sat = {}
    for name, cfg in engines.items():
        srv = R.Server(gg, **cfg)
        t0 = time.perf_counter()
        tickets = [srv.submit(nfas[q.regex], q.source) for q in qs[:sat_n]]
        srv.drain(600000)
        sat[name] = sat_n / (time.perf_counter() - t0)
        for t in tickets:
            srv.poll(t)
        srv.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for q in qs[:sat_n]:
        R.rpq_query(gg, nfas[q.regex], q.source, out=out, stream=stream)
    sat_seq = sat_n / (time.perf_counter() - t0)
    return {"workload": f"rmat20_serve: Poisson arrivals at 2,000 q/s for "
                        f"{args.serve_seconds + 1.0:.0f} s ({len(qs)} queries, mixed templates "
                        "of 1-12 DFA states); server engine 0 = 8 concurrent query slots "
                        "(queries_per_s), engine 1 = 256 bit lanes",
            "queries_per_s": st_srv["qps"], "p50_ms": st_srv["p50_ms"],
            "p99_ms": st_srv["p99_ms"], "gpu_launches": st_srv["gpu_launches"],
            "engines": {k: {"qps": v["qps"], "p50_ms": v["p50_ms"], "p99_ms": v["p99_ms"],
                            "gpu_launches": v["gpu_launches"]}
                        for k, v in served_stats.items()},
            "unbatched_served_loop": unb,
            "saturation_queries_per_s": {"server_slots": sat["slots"],
                                         "server_lanes": sat["lanes"],
                                         "one_at_a_time": sat_seq, "queries": sat_n}}


# ------------------------------------------------------------- GPU path ---

def measure_single(R, torch, w, gg, nfas, srcs, steps, warmup, stream, clock_dev=None,
                   dist=None):
    """Times `steps` steps of the workload's queries run one at a time with
    device outputs and no per-query statistics (CUDA events around each step
    on the launching stream, L2 flushed in between; the host latency of
    every call), then `steps` more steps of the same queries with the
    library's statistics, whose CUDA events around every launch give the
    kernel's device time and whose counters give the algorithmic bytes.
    Returns the step times and latencies of the first, the statistics
    records of the second, the launches counted in the first and the clocks
    over both."""
    out = torch.empty(w.graph.n, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    lean = R.QueryRunner(gg, out, stream)
    full = R.QueryRunner(gg, out, stream, with_stats=True)
    states = [nfa.info()[0] for nfa in nfas]
    pc = time.perf_counter

    def lean_step(lat):
        run = lean.run
        for nfa, s in zip(nfas, srcs):
            t0 = pc()
            run(nfa, s)
            lat.append(pc() - t0)

    def stats_step(recs):
        run, st = full.run, full.stats
        for nfa, s, S in zip(nfas, srcs, states):
            run(nfa, s)
            recs.append((st.as_dict(), S))

    def timed(body, sink):
        flush.fill_(1)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        k0 = R.rpq_kernel_launches()
        e0.record(stream)
        body(sink)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), R.rpq_kernel_launches() - k0

    for _ in range(warmup):
        lean_step([])
        stats_step([])
    torch.cuda.synchronize()
    step_ms, lat, recs, k_timed = [], [], [], 0
    clk = ClockSampler(clock_dev) if clock_dev is not None else None
    if clk:
        clk.__enter__()
    try:
        for _ in range(steps):
            ms, k = timed(lean_step, lat)
            step_ms.append(ms)
            k_timed += k
        for _ in range(steps):
            timed(stats_step, recs)
    finally:
        if clk:
            clk.__exit__(None, None, None)
    return {"step_ms": step_ms, "lat": lat, "recs": recs, "launches": k_timed,
            "clocks": clk.summary() if clk else None}


def latency_summary(lat_s):
    lat = sorted(x * 1000.0 for x in lat_s)
    return lat[len(lat) // 2], lat[min(len(lat) - 1, int(0.99 * len(lat)))]


def algorithmic_bytes(recs, W_words):
    """Push-model bytes and the dense formulation's bitset sweeps (3 x S x W
    x 8 bytes per expanded level) of the recorded queries."""
    push = sum(r[0]["push_bytes"] for r in recs)
    sweep = sum(3 * r[1] * W_words * 8 * (r[0]["levels"] + 1) for r in recs)
    return push, sweep


def run_rmat20_extra(args, R, torch, g, gg):
    """The rmat20 single-query figures (400 queries one at a time) for the
    default line's extras."""
    from paper_2412_10287_gb300 import workloads as W

    qs = W.make_queries(g, W.TEMPLATES_SMALL, 100, seed=1, zipf_s=1.0)
    nfas = [R.rpq_nfa_compile(q.regex, g.n_labels) for q in qs]
    srcs = [q.source for q in qs]
    stream = torch.cuda.current_stream()
    m = measure_single(R, torch, W.Workload("rmat20", g, qs), gg, nfas, srcs, args.steps,
                       args.warmup, stream)
    total_s = sum(m["step_ms"]) / 1000.0
    p50, p99 = latency_summary(m["lat"])
    push, sweep = algorithmic_bytes(m["recs"], (g.n + 63) // 64)
    launch_s = sum(r[0]["device_ms"] for r in m["recs"]) / len(m["recs"]) / 1000.0
    peak, _ = measured_peak()
    ach = (push + sweep) / len(m["recs"]) / launch_s / 1e9
    return {"workload": "rmat20: R-MAT scale 20, 8 labels Zipf(1.0), seed 1; 400 single-source "
                        "queries (a*, a.b*, (a|b)*.c, a^-.b*), one at a time",
            "queries_per_s": len(qs) * args.steps / total_s, "p50_ms": p50, "p99_ms": p99,
            "ms_per_step": 1000.0 * total_s / args.steps,
            "product_edges_per_s": sum(r[0]["product_edges"] for r in m["recs"]) / total_s,
            "roofline": {"achieved": ach, "frac": ach / peak, "unit": "GB/s",
                         "avg_launch_ms": launch_s * 1000.0,
                         "achieved_push_bytes_only": push / len(m["recs"]) / launch_s / 1e9},
            "gpu_launches": m["launches"]}


RARE_MAX = 200_000  # edges: labels at or below this count as rare for the rare-first plan


def rare_queries(g, count=48, seed=7):
    """Queries whose last label is rare: a/b*/c and a/(b|^d)*/c with a, b, d
    among the 10 most frequent labels and c among the labels with at most
    RARE_MAX edges (the long tail of the Zipf label distribution)."""
    from paper_2412_10287_gb300 import workloads as W

    counts = np.bincount(g.lab, minlength=g.n_labels)
    order = np.argsort(-counts)
    freq = order[:10]
    tail = np.flatnonzero((counts > 0) & (counts <= RARE_MAX))
    if tail.size == 0:
        return []
    r = W.below(seed, 1, 5 * count, 1 << 30)
    deg = np.bincount(g.src, minlength=g.n) + np.bincount(g.dst, minlength=g.n)
    cand = np.flatnonzero(deg > 0)
    qs = []
    for i in range(count):
        a, b, d = (int(freq[r[5 * i + k] % freq.size]) for k in range(3))
        c = int(tail[r[5 * i + 3] % tail.size])
        text = f"{a}/{b}*/{c}" if i % 2 == 0 else f"{a}/({b}|^{d})*/{c}"
        qs.append(W.Query(text, int(cand[r[5 * i + 4] % cand.size]), "rare-last"))
    return qs


def run_rare_plan(args, R, torch, w, gg):
    """Rare label first against the plain search, on queries whose last
    label is rare and on the workload's own queries; answers compared."""
    g = w.graph
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(qs, nfas, plan):
        R.rpq_graph_set_rare_plan(gg, RARE_MAX if plan else 0)
        answers = []
        for rep_ in range(2):  # warm-up pass, then the timed one
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cnts = [R.rpq_query(gg, nfa, q.source, out=out, stream=stream)
                    for nfa, q in zip(nfas, qs)]
            e1.record(stream)
            torch.cuda.synchronize()
        for nfa, q in zip(nfas, qs[:16]):
            answers.append(R.rpq_query(gg, nfa, q.source).tolist())
        R.rpq_graph_set_rare_plan(gg, 0)
        return len(qs) / (e0.elapsed_time(e1) / 1000.0), cnts, answers

    res = {"rare_max_edges": RARE_MAX}
    for name, qs in (("rare_last_label", rare_queries(g)), ("workload", w.queries)):
        if not qs:
            continue
        nfas = [R.rpq_nfa_compile(q.regex, g.n_labels) for q in qs]
        q0, c0, a0 = timed(qs, nfas, False)
        q1, c1, a1 = timed(qs, nfas, True)
        res[name] = {"queries": len(qs), "plain_queries_per_s": q0, "rare_first_queries_per_s": q1,
                     "speedup": q1 / q0, "answers_equal": c0 == c1 and a0 == a1}
    return res


def run_extras(args, R, torch):
    """rmat20, batch and serve figures on the R-MAT scale-20 graph."""
    from paper_2412_10287_gb300 import workloads as W

    g = W.config2_graph()
    gg = R.rpq_graph_load(g.n, g.n_labels, g.src, g.dst, g.lab)
    out = {"rmat20": run_rmat20_extra(args, R, torch, g, gg),
           "batch": run_batch(args, R, torch, g, gg),
           "serve": run_serve(args, R, torch, g, gg)}
    gg.close()
    return out


def run_profile_sample(args):
    """The launches an ncu DRAM capture takes: every query of the workload
    once (skipped by the capture: `-s` = the number of queries), then the
    `--profile-sample` queries with the longest device time again (they
    dominate the mean launch), whose algorithmic and push-model bytes go to
    `--sample-out`.  The push/pull
    setting is the library's default or the RPQ_PULL_* / RPQ_SOLO_*
    environment variables (no autotuning launches before the capture)."""
    import torch

    torch.cuda.set_device(0)
    import __graft_entry__

    __graft_entry__.build()
    from paper_2412_10287_gb300 import rpq as R

    name = args.workload
    w = workload(per_template_for(name, args.per_template), name)
    g = w.graph
    gg = R.rpq_graph_load(g.n, g.n_labels, g.src, g.dst, g.lab)
    W_words = (g.n + 63) // 64
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    nfas = [R.rpq_nfa_compile(q.regex, g.n_labels) for q in w.queries]
    alg = []
    for nfa, q in zip(nfas, w.queries):
        _, st = R.rpq_query(gg, nfa, q.source, out=out, stream=stream, with_stats=True)
        S = nfa.info()[0]
        alg.append((st["push_bytes"] + 3 * S * W_words * 8 * (st["levels"] + 1), st["push_bytes"],
                    st["device_ms"]))
    pick = sorted(range(len(alg)), key=lambda i: -alg[i][2])[:args.profile_sample]
    for i in pick:
        R.rpq_query(gg, nfas[i], w.queries[i].source, out=out, stream=stream)
    torch.cuda.synchronize()
    rec = {"workload": name, "skip_launches": len(nfas),
           "queries": [[w.queries[i].regex, w.queries[i].source] for i in pick],
           "algorithmic_bytes": [alg[i][0] for i in pick],
           "push_bytes": [alg[i][1] for i in pick],
           "device_ms": [alg[i][2] for i in pick],
           "sample": f"the {len(pick)} of the {len(nfas)} {name} queries with the longest "
                     "device time, captured after one pass over all of them"}
    os.makedirs(os.path.dirname(os.path.abspath(args.sample_out)), exist_ok=True)
    with open(args.sample_out, "w") as f:
        json.dump(rec, f)
    print(json.dumps(rec))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.write_profile:
        write_profile(args.write_profile, args.workload, args.sample_json)
        return
    if args.profile_sample:
        run_profile_sample(args)
        return
    if args.one_query is not None:
        import torch

        torch.cuda.set_device(0)
        import __graft_entry__

        __graft_entry__.build()
        from paper_2412_10287_gb300 import rpq as R
        from paper_2412_10287_gb300 import workloads as W

        if args.kb_size:
            n_, m_ = (int(x) for x in args.kb_size.split(","))
            g = W.config3_graph(n_, m_)
        else:
            g = W.config3_graph() if args.workload == "kb20m" else W.config2_graph()
        gg = R.rpq_graph_load(g.n, g.n_labels, g.src, g.dst, g.lab)
        nfa = R.rpq_nfa_compile(args.one_query, g.n_labels)
        for _ in range(2):
            _, st = R.rpq_query(gg, nfa, args.source, with_stats=True)
        print(json.dumps({"query": args.one_query, "source": args.source, "stats": st}))
        return
    if args.workload in ("batch", "serve"):
        import torch

        torch.cuda.set_device(0)
        import __graft_entry__

        __graft_entry__.build()
        from paper_2412_10287_gb300 import rpq as R

        r = (run_batch if args.workload == "batch" else run_serve)(args, R, torch)
        metric = "rpq_queries_per_s" if args.workload == "batch" else "rpq_served_queries_per_s"
        line = {"metric": metric, "value": r["queries_per_s"], "unit": "queries/s", "n_gpus": 1,
                "steps": args.steps if args.workload == "batch" else 1,
                "warmup": args.warmup if args.workload == "batch" else 1,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                "data": "synthetic", "config": {"workload": r["workload"]}}
        line.update({k: v for k, v in r.items() if k not in ("workload", "queries_per_s")})
        print(json.dumps(line), flush=True)
        return
    import torch

    ws, rank, local = dist_info()
    dist = None
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    import __graft_entry__

    __graft_entry__.build()
    from paper_2412_10287_gb300 import rpq as R

    name = args.workload
    per_template = per_template_for(name, args.per_template)
    w = workload(per_template, name)
    if rank > 0:
        w.queries = rank_queries(w.graph, name, per_template, rank)
    g = w.graph
    gg = R.rpq_graph_load(g.n, g.n_labels, g.src, g.dst, g.lab)
    tuned = autotune(R, gg, g, name)
    nfas = [R.rpq_nfa_compile(q.regex, g.n_labels) for q in w.queries]
    srcs = [q.source for q in w.queries]
    nq = len(srcs)
    stream = torch.cuda.current_stream()
    W_words = (g.n + 63) // 64
    global PROFILE_JSON
    PROFILE_JSON = os.path.join(ROOT, "profiles", f"rpq_query_kernel_{name}.json")

    m = measure_single(R, torch, w, gg, nfas, srcs, args.steps, args.warmup, stream,
                       clock_dev=dev, dist=dist)
    recs = m["recs"]
    total_s = sum(m["step_ms"]) / 1000.0
    if ws > 1:
        total_s = max_over_ranks(total_s, dist, "cuda")
    value = ws * nq * args.steps / total_s
    p50, p99 = latency_summary(m["lat"])
    kern_ms = [r[0]["device_ms"] for r in recs]
    push_bytes, sweep_bytes = algorithmic_bytes(recs, W_words)
    prod_edges = sum(r[0]["product_edges"] for r in recs)
    alg_bytes_per_launch = (push_bytes + sweep_bytes) / len(recs)
    avg_launch_s = sum(kern_ms) / len(kern_ms) / 1000.0
    achieved = alg_bytes_per_launch / avg_launch_s / 1e9
    peak, peak_kind = measured_peak()

    # end to end through the public API: compile + query with host outputs.
    # The bytes each step moves come from one untimed pass with statistics;
    # the timed steps make the calls a user makes, without them.
    h2d, d2h = 0, 0
    for q in w.queries:
        nfa = R.rpq_nfa_compile(q.regex, g.n_labels)
        _, st = R.rpq_query(gg, nfa, q.source, stream=stream, with_stats=True)
        h2d += st["h2d_bytes"]
        d2h += st["d2h_bytes"]
    e2e_steps = []
    for k in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for q in w.queries:
            nfa = R.rpq_nfa_compile(q.regex, g.n_labels)
            ans = R.rpq_query(gg, nfa, q.source, stream=stream)
        e2e_steps.append(time.perf_counter() - t0)
    e2e_s = sum(e2e_steps)
    if ws > 1:
        e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    e2e_value = ws * nq * args.steps / e2e_s
    # per-launch DRAM traffic: the committed ncu sample's DRAM bytes per
    # algorithmic byte, scaled to this run's algorithmic bytes per launch
    traffic = profile_traffic(alg_bytes_per_launch)

    extras = None
    if ws == 1 and not args.no_extras:
        rare = run_rare_plan(args, R, torch, w, gg) if name == "kb20m" else None
        gg.close()  # the R-MAT graph takes its place on the device
        extras = run_extras(args, R, torch)
        if rare:
            extras["rare_first"] = rare

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(w, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": "rpq_queries_per_s", "value": value, "unit": "queries/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": workload_config(w, nq, {"autotuned": tuned}),
            "p50_ms": p50, "p99_ms": p99,
            "product_edges_per_s": ws * prod_edges / total_s,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "rpq_query_kernel",
                         "peak_kind": f"{peak_kind} copy bandwidth",
                         "algorithmic_bytes_per_launch": alg_bytes_per_launch,
                         "achieved_push_bytes_only": push_bytes / len(recs) / avg_launch_s / 1e9,
                         "avg_launch_ms": avg_launch_s * 1000.0},
            "e2e": {"value": e2e_value, "unit": "queries/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": m["launches"],
            "clocks": m["clocks"],
        }
        if cpu:
            line["cpu_baseline"] = cpu
        if extras:
            line["extras"] = extras
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
