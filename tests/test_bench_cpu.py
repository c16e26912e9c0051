"""Host logic of bench.py that its JSON line depends on, on CPU: ncu CSV
units, the per-launch DRAM summary written beside the kernel source's hash
and read back for the roofline's `traffic`, the measured-peak lookup and the
clock-sample summary that decides whether a run is kept."""

import csv
import io
import json
import os

import pytest

import bench

NCU_HEADER = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream",
              "Block Size", "Grid Size", "Device", "CC", "Section Name", "Metric Name",
              "Metric Unit", "Metric Value"]


def ncu_csv(rows):
    """An ncu --csv log: a banner line, then quoted CSV rows."""
    buf = io.StringIO()
    buf.write("==PROF== Connected to process 1\n")
    w = csv.writer(buf, quoting=csv.QUOTE_ALL, lineterminator="\n")
    w.writerow(NCU_HEADER)
    for launch, kernel, metric, unit, value in rows:
        w.writerow([launch, "1", "python", "host", kernel, "1", "7", "(256, 1, 1)", "(456, 1, 1)",
                    "0", "10.3", "Command line profiler metrics", metric, unit, value])
    return buf.getvalue()


def test_ncu_units_to_base():
    assert bench.ncu_value("byte", "1,024") == 1024.0
    assert bench.ncu_value("Kbyte", "2") == 2000.0
    assert bench.ncu_value("Mbyte", "1.5") == 1.5e6
    assert bench.ncu_value("Gbyte", "2") == 2e9
    assert bench.ncu_value("nsecond", "1500") == pytest.approx(1.5e-6)
    assert bench.ncu_value("usecond", "2") == pytest.approx(2e-6)
    assert bench.ncu_value("msecond", "3") == pytest.approx(3e-3)
    assert bench.ncu_value("", "7") == 7.0
    assert bench.ncu_value("%", "12.5") == 12.5


def test_write_profile_means_and_hash(tmp_path, monkeypatch):
    """Means over the traversal kernel's launches only, other kernels
    ignored, stored with the kernel source's sha256; traffic is read back
    only while that hash matches."""
    k = "rpq::<unnamed>::rpq_query_kernel(rpq::<unnamed>::KParams)"
    rows = [("1", k, "dram__bytes_read.sum", "byte", "1,000,000"),
            ("1", k, "dram__bytes_write.sum", "Kbyte", "10"),
            ("1", k, "gpu__time_duration.sum", "nsecond", "100,000"),
            ("2", k, "dram__bytes_read.sum", "Mbyte", "3"),
            ("2", k, "dram__bytes_write.sum", "byte", "30000"),
            ("2", k, "gpu__time_duration.sum", "usecond", "300"),
            ("3", "rpq::<unnamed>::radix_scatter_kernel", "dram__bytes_read.sum", "Gbyte", "9")]
    src = tmp_path / "ncu.csv"
    src.write_text(ncu_csv(rows))
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    bench.write_profile(str(src), "unit")
    out = json.loads((tmp_path / "profiles" / "rpq_query_kernel_unit.json").read_text())
    assert out["launches"] == 2
    assert out["dram_read_bytes_per_launch"] == pytest.approx(2e6)
    assert out["dram_write_bytes_per_launch"] == pytest.approx(2e4)
    assert out["dram_bytes_per_launch"] == pytest.approx(2.02e6)
    assert out["ncu_ms_per_launch"] == pytest.approx(0.2)
    assert out["kernel_source_sha256"] == bench.sha256(bench.KERNEL_SOURCE)

    monkeypatch.setattr(bench, "PROFILE_JSON", str(tmp_path / "profiles" / "rpq_query_kernel_unit.json"))
    assert bench.profile_traffic() == pytest.approx(2.02e6)
    other = tmp_path / "kernel_copy.cu"
    other.write_text(open(bench.KERNEL_SOURCE).read() + "\n// changed\n")
    monkeypatch.setattr(bench, "KERNEL_SOURCE", str(other))
    assert bench.profile_traffic() is None  # taken on another kernel source
    monkeypatch.setattr(bench, "PROFILE_JSON", str(tmp_path / "missing.json"))
    assert bench.profile_traffic() is None


def test_write_profile_rejects_a_csv_without_the_kernel(tmp_path, monkeypatch):
    src = tmp_path / "ncu.csv"
    src.write_text(ncu_csv([("1", "other_kernel", "dram__bytes_read.sum", "byte", "5")]))
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    with pytest.raises(SystemExit):
        bench.write_profile(str(src), "unit")


def test_measured_peak_file_or_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak() == (bench.HBM_FALLBACK_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6773.2}))
    assert bench.measured_peak() == (6773.2, "measured")


def clock_rows(tmp_path, rows):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        for r in rows:
            f.write(", ".join(r) + "\n")
    return s.summary()


def test_clock_summary_median_max_and_reasons(tmp_path):
    idle = ["Not Active"] * 4
    rows = [["2070", "2070", "900.1", "0x0"] + idle,
            ["2055", "2070", "1100.0", "0x0"] + idle,
            ["2070", "2070", "1390.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"]]
    out = clock_rows(tmp_path, rows)
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    rows.append(["1500", "2070", "1400.0", "0x8", "Active", "Not Active", "Active", "Not Active"])
    out = clock_rows(tmp_path, rows)
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert not os.path.exists(str(tmp_path / "clocks.csv"))  # the sample file is removed


def test_clock_summary_without_samples(tmp_path):
    out = clock_rows(tmp_path, [])
    assert out == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}


def test_write_profile_sample_ratio_scales_traffic(tmp_path, monkeypatch):
    """A capture of a few sample launches stores DRAM bytes per algorithmic
    byte; the traffic of a run's mean launch is that ratio times the run's
    algorithmic bytes per launch."""
    k = "rpq::<unnamed>::rpq_query_kernel(rpq::<unnamed>::KParams)"
    rows = [("7", k, "dram__bytes_read.sum", "byte", "3,000"),
            ("7", k, "dram__bytes_write.sum", "byte", "1,000"),
            ("9", k, "dram__bytes_read.sum", "byte", "5,000"),
            ("9", k, "dram__bytes_write.sum", "byte", "1,000")]
    src = tmp_path / "ncu.csv"
    src.write_text(ncu_csv(rows))
    sj = tmp_path / "sample.json"
    sj.write_text(json.dumps({"algorithmic_bytes": [2000, 3000], "push_bytes": [500, 500],
                              "sample": "two launches"}))
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    bench.write_profile(str(src), "unit", str(sj))
    out = json.loads((tmp_path / "profiles" / "rpq_query_kernel_unit.json").read_text())
    assert out["dram_per_algorithmic_byte"] == pytest.approx(10000 / 5000)
    assert out["dram_per_push_byte"] == pytest.approx(10.0)
    monkeypatch.setattr(bench, "PROFILE_JSON", str(tmp_path / "profiles" / "rpq_query_kernel_unit.json"))
    assert bench.profile_traffic(1e6) == pytest.approx(2e6)
    assert bench.profile_traffic() == pytest.approx(5000.0)  # the sample's own mean
    sj.write_text(json.dumps({"algorithmic_bytes": [2000], "push_bytes": [500]}))
    with pytest.raises(SystemExit):  # launches and sample queries must pair up
        bench.write_profile(str(src), "unit", str(sj))


def test_oracle_sample_is_bounded_and_counts_what_ran():
    from paper_2412_10287_gb300 import workloads as W

    g = W.rmat_graph(10, 6000, 8, seed=5)
    qs = W.make_queries(g, W.TEMPLATES_SMALL, 5, seed=1, zipf_s=1.0)
    w = W.Workload("rmat10", g, qs)
    r = bench.oracle_sample(w, 0.0, max_threads=2)  # no time: one round of submissions
    assert 1 <= r["queries"] <= 2 and r["cores"] == 2 and r["kind"] == "oracle"
    r = bench.oracle_sample(w, 30.0, max_threads=2)
    assert r["queries"] == len(qs) and r["value"] == pytest.approx(r["queries"] / r["wall_s"])


def test_rare_queries_end_in_a_rare_label():
    import numpy as np

    from paper_2412_10287_gb300 import workloads as W

    g = W.chung_lu_graph(200_000, 2_000_000, 2.1, 500, 1.1, seed=2)
    counts = np.bincount(g.lab, minlength=500)
    qs = bench.rare_queries(g, 12)
    assert len(qs) == 12
    for q in qs:
        last = int(q.regex.rsplit("/", 1)[1])
        assert 0 < counts[last] <= bench.RARE_MAX
        assert 0 <= q.source < g.n
