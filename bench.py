#!/usr/bin/env python
"""Benchmark: single-source 2-RPQ queries/s on one GB300 (or N replicas).

Workload (default ``rmat20``): R-MAT scale 20 (1,048,576 vertices, 2^24 edge
samples, a=0.57 b=c=0.19), 8 labels with Zipf(1.0) frequencies, seed 1; 400
queries = templates a*, a.b*, (a|b)*.c, a^-.b* x 100 random sources with
non-zero degree; queries run one at a time, as in the paper's evaluation
(section 5.3: data preloaded, sequential isolated queries).

One step = those 400 queries.  ``value`` = queries/s with the graph and the
outputs resident on the device (rpq_query with a device output buffer,
CUDA events on the launching stream around each step, L2 flushed between
steps).  ``e2e`` = the same queries through the public API with host
output buffers and regex compilation inside the timed region.  The roofline
line refers to the traversal kernel (one cooperative launch per query).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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
PROFILE_JSON = os.path.join(ROOT, "profiles", "rpq_query_kernel_rmat20.json")
KERNEL_SOURCE = os.path.join(ROOT, "paper_2412_10287_gb300", "csrc", "query.cu")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--per-template", type=int, default=100)
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="CPU work budget of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="rmat20", choices=["rmat20", "kb20m", "batch", "serve"],
                    help="rmat20: single queries (the default line); kb20m: single queries on "
                         "the 20M-vertex knowledge-base graph; batch: 256 mixed queries per "
                         "launch; serve: Poisson arrivals through the server")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--one-query", default=None,
                    help="profiling case: run this regex once for warm-up and once more "
                         "(with --source) on the workload's graph, print its counters, exit")
    ap.add_argument("--source", type=int, default=0)
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


def profile_traffic():
    """Per-launch DRAM bytes of the traversal kernel from the committed ncu
    summary, or None if absent or taken on a different kernel source."""
    try:
        with open(PROFILE_JSON) as f:
            pj = json.load(f)
        if pj.get("kernel_source_sha256") != sha256(KERNEL_SOURCE):
            return None
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


def write_profile(csv_path, workload_name):
    """Per-launch DRAM bytes and ncu durations of the traversal kernel, from an
    ncu CSV, written beside the kernel source's hash so that a later change
    to the kernel voids the figure."""
    import csv

    launches = {}
    with open(csv_path, newline="") as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for row in csv.DictReader(lines):
        if "rpq_query_kernel" not in row.get("Kernel Name", ""):
            continue
        d = launches.setdefault(row["ID"], {})
        d[row["Metric Name"]] = ncu_value(row.get("Metric Unit", ""), row["Metric Value"])
    per = [d for d in launches.values()
           if "dram__bytes_read.sum" in d and "dram__bytes_write.sum" in d]
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


def workload(per_template, name="rmat20"):
    from paper_2412_10287_gb300 import workloads as W

    if name == "kb20m":
        return W.config3(per_template=per_template)
    return W.config2(per_template=per_template)


# query templates, seed and label skew of each single-query workload
QUERY_SPECS = {"rmat20": ("TEMPLATES_SMALL", 1, 1.0), "kb20m": ("TEMPLATES_KB", 2, 1.1)}


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


def oracle_sample(w, seconds_budget, max_threads=None):
    """Times the CPU oracle (as it stands) on a stratified sample of the
    workload's queries, on the host cores (one query per thread)."""
    from oracle import oracle as O
    from oracle.regex_nfa import compile_regex

    g = w.graph
    og = O.OracleGraph(g.n, g.n_labels, g.src, g.dst, g.lab)
    threads = max_threads or len(os.sched_getaffinity(0))
    qs = w.queries
    # estimate the per-query cost on a small probe, then size the sample
    probe = [qs[i] for i in range(0, len(qs), max(1, len(qs) // 8))][:8]
    t0 = time.perf_counter()
    for q in probe:
        og.ssr(compile_regex(q.regex, g.n_labels), q.source)
    per_q = (time.perf_counter() - t0) / max(1, len(probe))
    n_sample = int(max(threads, min(len(qs), seconds_budget / max(per_q, 1e-6))))
    stride = max(1, len(qs) // n_sample)
    sample = qs[::stride][:n_sample]
    nfas = [compile_regex(q.regex, g.n_labels) for q in sample]

    def run(i):
        return og.ssr(nfas[i], sample[i].source)["counters"]["answer"]

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(run, range(len(sample))))
    wall = time.perf_counter() - t0
    og.close()
    return {"value": len(sample) / wall, "unit": "queries/s", "cores": threads, "kind": "oracle",
            "sample": f"{len(sample)} of the {len(qs)} queries (every {stride}th), "
                      f"{threads} threads, one query per thread; adjacency lists built before "
                      f"timing; {wall:.1f} s wall"}


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    w = workload(args.per_template)
    per_step_budget = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    vals = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample(w, per_step_budget * 4)
        if i >= args.warmup:
            vals.append(r)
    v = statistics.median([r["value"] for r in vals])
    line = {"impl": "reference", "metric": "rpq_queries_per_s", "value": v, "unit": "queries/s",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * len(w.queries) / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": workload_config(w, len(w.queries),
                                      {"note": "CPU oracle timed on a bounded sample per step"}),
            "cpu_baseline": {"value": v, "unit": "queries/s", "cores": vals[-1]["cores"],
                             "kind": "oracle", "sample": vals[-1]["sample"]},
            "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------ batch / serve ----

def run_batch(args, R, torch):
    """256 mixed queries (2-12 DFA states) per rpq_query_batch launch against
    the same 256 queries run one at a time."""
    from paper_2412_10287_gb300 import workloads as W

    g = W.config2_graph()
    w = W.config4(g, 256)
    gg = R.rpq_graph_load(g.n, g.n_labels, g.src, g.dst, g.lab)
    nfas = [R.rpq_nfa_compile(q.regex, g.n_labels) for q in w.queries]
    srcs = [q.source for q in w.queries]
    states = [n.info()[0] for n in nfas]
    res = R.rpq_query_batch(gg, nfas, srcs)  # warm-up, sizes the output
    total = sum(a.size for a in res)
    out = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
    offs = np.zeros(len(nfas) + 1, np.int64)
    import ctypes

    handles = (ctypes.c_void_p * len(nfas))(*[x.h.value for x in nfas])
    src_arr = np.array(srcs, np.int32)
    stream = torch.cuda.current_stream()

    def batch_once():
        s = R.lib().rpq_query_batch(gg.h, len(nfas), handles, R._ptr(src_arr), 0, R._ptr(offs),
                                    R._ptr(out), out.numel(), None,
                                    ctypes.c_void_p(stream.cuda_stream))
        assert s == 0, R.rpq_last_error()

    def seq_once():
        one = torch.empty(g.n, dtype=torch.int32, device="cuda")
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
    for label, env, jobs in (("mixed_on_lanes", "lanes", None),
                             ("shared_automaton_lanes", None, "shared"),
                             ("shared_automaton_sequential", None, "shared_seq")):
        old_env = os.environ.get("RPQ_BATCH_ENGINE")
        if env:
            os.environ["RPQ_BATCH_ENGINE"] = env
        try:
            if jobs is None:
                fn = batch_once
            else:
                shared = [R.rpq_nfa_compile("0*", g.n_labels)] * len(srcs)
                sh_handles = (ctypes.c_void_p * len(shared))(*[x.h.value for x in shared])
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
                        one = torch.empty(g.n, dtype=torch.int32, device="cuda")
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
            if env:
                if old_env is None:
                    os.environ.pop("RPQ_BATCH_ENGINE", None)
                else:
                    os.environ["RPQ_BATCH_ENGINE"] = old_env
    line = {"metric": "rpq_queries_per_s", "value": qb, "unit": "queries/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * sum(tb) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "rmat20_batch: the rmat20 graph; 256 mixed queries per "
                                   f"rpq_query_batch call (DFA states {min(states)}-{max(states)}); "
                                   "seed 3",
                       "l2": "flushed between steps (256 MiB write)"},
            "sequential_single_queries_per_s": qs, "batch_speedup": qb / qs,
            "engine": os.environ.get("RPQ_BATCH_ENGINE", "auto (slots for mixed automata)"),
            "other_engines_queries_per_s": extra,
            "answer_vertices_per_step": int(total), "gpu_launches": batch_launches}
    print(json.dumps(line), flush=True)


def run_serve(args, R, torch):
    """Poisson arrivals (2,000 q/s) replayed in real time into the server, and
    into a one-at-a-time served loop; then both at saturation."""
    import threading

    from paper_2412_10287_gb300 import workloads as W

    g = W.config2_graph()
    w = W.config5(g, rate=2000.0, duration_s=args.serve_seconds, warmup_s=1.0)
    gg = R.rpq_graph_load(g.n, g.n_labels, g.src, g.dst, g.lab)
    nfas = {}
    for q in w.queries:
        if q.regex not in nfas:
            nfas[q.regex] = R.rpq_nfa_compile(q.regex, g.n_labels)
    qs = w.queries
    engines = {"slots": dict(max_lanes=12, engine=0), "lanes": dict(max_lanes=256, max_states=16,
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

    line = {"metric": "rpq_served_queries_per_s", "value": st_srv["qps"], "unit": "queries/s",
            "n_gpus": 1, "steps": 1, "warmup": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"rmat20_serve: Poisson arrivals at 2,000 q/s for "
                                   f"{args.serve_seconds + 1.0:.0f} s ({len(qs)} queries, mixed "
                                   "templates of 1-12 DFA states); server engine 0 = 12 "
                                   "concurrent query slots (value), engine 1 = 256 bit lanes"},
            "p50_ms": st_srv["p50_ms"], "p99_ms": st_srv["p99_ms"],
            "gpu_launches": st_srv["gpu_launches"],
            "engines": {k: {"qps": v["qps"], "p50_ms": v["p50_ms"], "p99_ms": v["p99_ms"],
                            "gpu_launches": v["gpu_launches"]}
                        for k, v in served_stats.items()},
            "unbatched_served_loop": unb,
            "saturation_queries_per_s": {"server_slots": sat["slots"],
                                         "server_lanes": sat["lanes"],
                                         "one_at_a_time": sat_seq, "queries": sat_n}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- GPU path ---

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.write_profile:
        write_profile(args.write_profile, args.workload)
        return
    if args.one_query is not None:
        import torch

        torch.cuda.set_device(0)
        import __graft_entry__

        __graft_entry__.build()
        from paper_2412_10287_gb300 import rpq as R
        from paper_2412_10287_gb300 import workloads as W

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

        (run_batch if args.workload == "batch" else run_serve)(args, R, torch)
        return
    import torch

    ws, rank, local = dist_info()
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

    per_template = args.per_template if args.workload == "rmat20" else min(args.per_template, 25)
    w = workload(per_template, args.workload)
    if rank > 0:
        w.queries = rank_queries(w.graph, args.workload, per_template, rank)
    g = w.graph
    gg = R.rpq_graph_load(g.n, g.n_labels, g.src, g.dst, g.lab)
    tuned = autotune(R, gg, g, args.workload)
    nfas = [R.rpq_nfa_compile(q.regex, g.n_labels) for q in w.queries]
    srcs = [q.source for q in w.queries]
    nq = len(srcs)
    stream = torch.cuda.current_stream()
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    W_words = (g.n + 63) // 64
    if args.workload == "kb20m":
        global PROFILE_JSON
        PROFILE_JSON = os.path.join(ROOT, "profiles", "rpq_query_kernel_kb20m.json")

    def one_step(collect):
        res = []
        for nfa, s in zip(nfas, srcs):
            t0 = time.perf_counter()
            cnt, st = R.rpq_query(gg, nfa, s, out=out, stream=stream, with_stats=True)
            if collect:
                res.append((time.perf_counter() - t0, st, nfa.info()[0]))
        return res

    for _ in range(args.warmup):
        one_step(False)
    torch.cuda.synchronize()

    step_ms, recs = [], []
    k_timed = 0
    with ClockSampler(dev) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            if ws > 1:
                torch.distributed.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            k0 = R.rpq_kernel_launches()
            e0.record(stream)
            recs.extend(one_step(True))
            e1.record(stream)
            torch.cuda.synchronize()
            k_timed += R.rpq_kernel_launches() - k0
            step_ms.append(e0.elapsed_time(e1))
    clocks = clk.summary()
    total_s = sum(step_ms) / 1000.0
    if ws > 1:
        total_s = max_over_ranks(total_s, torch.distributed, "cuda")
    value = ws * nq * args.steps / total_s

    lat = sorted(r[0] * 1000.0 for r in recs)
    p50 = lat[len(lat) // 2]
    p99 = lat[min(len(lat) - 1, int(0.99 * len(lat)))]
    kern_ms = [r[1]["device_ms"] for r in recs]
    push_bytes = sum(r[1]["push_bytes"] for r in recs)
    sweep_bytes = sum(3 * r[2] * W_words * 8 * (r[1]["levels"] + 1) for r in recs)
    prod_edges = sum(r[1]["product_edges"] for r in recs)
    alg_bytes_per_launch = (push_bytes + sweep_bytes) / len(recs)
    avg_launch_s = sum(kern_ms) / len(kern_ms) / 1000.0
    achieved = alg_bytes_per_launch / avg_launch_s / 1e9
    peak, peak_kind = measured_peak()

    # end to end through the public API: compile + query with host outputs
    e2e_steps, h2d, d2h = [], 0, 0
    for k in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for q in w.queries:
            nfa = R.rpq_nfa_compile(q.regex, g.n_labels)
            ans, st = R.rpq_query(gg, nfa, q.source, stream=stream, with_stats=True)
            if k == 0:
                h2d += st["h2d_bytes"]
                d2h += st["d2h_bytes"]
        e2e_steps.append(time.perf_counter() - t0)
    e2e_s = sum(e2e_steps)
    if ws > 1:
        e2e_s = max_over_ranks(e2e_s, torch.distributed, "cuda")
    e2e_value = ws * nq * args.steps / e2e_s

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
            "product_edges_per_s": ws * prod_edges / (total_s if ws == 1 else total_s),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": profile_traffic(),
                         "kernel": "rpq_query_kernel",
                         "peak_kind": f"{peak_kind} copy bandwidth",
                         "algorithmic_bytes_per_launch": alg_bytes_per_launch,
                         "achieved_push_bytes_only": push_bytes / len(recs) / avg_launch_s / 1e9,
                         "avg_launch_ms": avg_launch_s * 1000.0},
            "e2e": {"value": e2e_value, "unit": "queries/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": k_timed,
            "clocks": clocks,
        }
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
