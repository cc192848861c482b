"""Host logic of bench.py, no GPU: the ncu launch-list summary (launches and
time per call of the forward and backward kernels, foreign kernels left out),
the traffic file built from one-kernel captures (bytes per launch with unit
conversion, per call, per unit), its stale-hash rule, and the roofline
arithmetic against hand-computed figures."""
import csv
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402  (parses its arguments in main() only)

HEADER = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
          "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]


def _launch(rows, i, name, ns, rd, wr):
    base = [str(i), "1", "python", "h", name, "1", "7", "(256, 1, 1)", "(1, 1, 1)", "0", "10.3", "Command line"]
    rows.append(base + ["gpu__time_duration.sum", "nsecond", f"{ns:,}"])
    rows.append(base + ["dram__bytes_read.sum", "byte", f"{rd:,}"])
    rows.append(base + ["dram__bytes_write.sum", "byte", f"{wr:,}"])


def _write_list(path, rows):
    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(HEADER)
        w.writerows(rows)


def _write_raw(path, launches):
    """Raw page of an ncu report: header, units, one row per launch."""
    h = ["ID", "Kernel Name", "dram__bytes_read.sum", "dram__bytes_write.sum", "gpu__time_duration.sum"]
    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(h)
        w.writerow(["", "", launches[0][2], launches[0][4], "nsecond"])
        for i, (name, rd, _, wr, _) in enumerate(launches):
            w.writerow([str(i), name, f"{rd:,}", f"{wr:,}", "1,000"])


PRE = "void gs::preprocess_kernel<1, false>(const gs_camera *, GaussIn, Ws)"
MERGE = "gs::merge_pass_kernel(Ws, int)"
BLEND = "void gs::blend_persistent_kernel<2, 1>(const gs_camera *, Ws, OutPtrs)"
BWD = "void gs::blend_backward_kernel<2, 1>(const gs_camera *, Ws, const float *)"


def _two_forwards_one_backward(rows):
    i = 0
    for call in range(2):  # two forwards: two merge passes each; one backward
        for name, ns in ((PRE, 2000), (MERGE, 300), (MERGE, 300), (BLEND, 3000)):
            _launch(rows, i, name, ns, 0, 0)
            i += 1
    _launch(rows, i, BWD, 5000, 0, 0)
    _launch(rows, i + 1, "void at::native::vectorized_elementwise_kernel<4>(int)", 9000, 1, 1)  # not ours


def test_ncu_summary_per_call(tmp_path):
    rows = []
    _two_forwards_one_backward(rows)
    p = tmp_path / "launches.csv"
    _write_list(p, rows)
    kern = bench.ncu_summary(str(p))
    assert kern["merge_pass_kernel"]["launches_per_call"] == 2
    assert kern["preprocess_kernel"]["launches_per_call"] == 1
    assert kern["blend_persistent_kernel"]["ms_per_call_under_ncu"] == pytest.approx(0.003)
    assert kern["blend_backward_kernel"]["ms_per_call_under_ncu"] == pytest.approx(0.005)  # one backward call
    assert "vectorized_elementwise_kernel" not in kern


def test_ncu_traffic_from_one_kernel_captures(tmp_path):
    """Bytes per launch from each kernel's own capture (units converted),
    launches per call from the time-only list, bytes per unit from the
    captured run's counts; the file carries the sources' hash."""
    rows = []
    _two_forwards_one_backward(rows)
    lst = tmp_path / "launches.csv"
    _write_list(lst, rows)
    _write_raw(tmp_path / "pre.csv", [(PRE, 1.5, "Kbyte", 500, "byte")])  # 1500 + 500 bytes
    _write_raw(tmp_path / "merge.csv", [(MERGE, 10, "byte", 10, "byte"), (MERGE, 20, "byte", 0, "byte"),
                                        (MERGE, 30, "byte", 20, "byte")])  # 30 bytes per launch
    _write_raw(tmp_path / "bwd.csv", [(BWD, 2, "Mbyte", 1, "Mbyte")])
    line = {"config": {"gaussians_per_gpu": 100}, "stats": {"records": 100, "pairs": 30, "visible": 25}}
    sj = tmp_path / "small.json"
    sj.write_text("log line\n" + json.dumps(line) + "\n")
    out = tmp_path / "traffic.json"
    kern = bench.ncu_traffic(str(lst), [str(tmp_path / x) for x in ("pre.csv", "merge.csv", "bwd.csv")], "cmd",
                             stats_json=str(sj), out_path=str(out))
    assert kern["preprocess_kernel"]["dram_bytes_per_call"] == pytest.approx(2000.0)
    assert kern["preprocess_kernel"]["unit"] == "gaussians"
    assert kern["preprocess_kernel"]["bytes_per_unit"] == pytest.approx(20.0)
    assert kern["merge_pass_kernel"]["captured_launches"] == 3
    assert kern["merge_pass_kernel"]["dram_bytes_per_launch"] == pytest.approx(30.0)
    assert kern["merge_pass_kernel"]["dram_bytes_per_call"] == pytest.approx(60.0)  # two passes per call
    assert kern["merge_pass_kernel"]["bytes_per_unit"] == pytest.approx(2.0)  # over 30 pairs
    assert kern["blend_backward_kernel"]["dram_bytes_per_call"] == pytest.approx(3e6)
    assert "blend_persistent_kernel" not in kern  # not captured
    t = json.loads(out.read_text())
    assert t["source_hash"] == bench.source_hash() and t["kernels"] == kern and t["command"] == "cmd"


def test_traffic_file_is_ignored_once_sources_change(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    t = {"source_hash": bench.source_hash(), "kernels": {"preprocess_kernel": {"dram_bytes_per_call": 5.0}}}
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(t))
    assert bench.dram_traffic()["preprocess_kernel"]["dram_bytes_per_call"] == 5.0
    monkeypatch.setattr(bench, "source_hash", lambda: "0000000000000000")
    assert bench.dram_traffic() == {}


def test_rooflines_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: (1000.0, "measured"))  # 1000 GB/s
    monkeypatch.setattr(bench, "dram_traffic", lambda: {"preprocess_kernel": {"dram_bytes_per_call": 123.0}})
    N = R = 1_000_000
    nvis, P = 250_000, 1_000_000
    stats = {"n_records": R, "n_visible": nvis, "n_pairs": P}
    stage_ms = {"preprocess": 1.0, "scatter": 0.5, "sort": 0.25, "merge": 0.25, "blend": 2.0,
                "blend_backward": 4.0, "preprocess_backward": 1.0}
    roof, per = bench.rooflines(stats, stage_ms, n_eval_fwd=10**9, n_eval_bwd=5 * 10**8, n_pix=1, N=N,
                                sm_count=100, sm_mhz=2000.0, exp_rate=1e12)
    pre = 12 * N + R // 8 + nvis * (28 + 4 + 96 + 48 + 64)
    assert per["preprocess"]["algorithmic"] == pre
    assert per["preprocess"]["achieved"] == pytest.approx(pre / 1e-3 / 1e9)
    assert per["preprocess"]["frac"] == pytest.approx(pre / 1e-3 / 1e9 / 1000.0)
    assert per["preprocess"]["traffic"] == 123.0 and per["scatter"]["traffic"] is None
    assert per["sort"]["ms"] == 0.5 and per["sort"]["algorithmic"] == 16 * P  # chunks + merge passes
    assert per["preprocess_backward"]["algorithmic"] == R // 8 + nvis * (12 + 28 + 4 + 96 + 64 + 236)
    alu = 100 * 128 * 2000e6 / 1e12  # T lane-ops/s
    assert per["blend"]["peak"] == pytest.approx(alu)
    assert per["blend"]["unit"] == per["blend_backward"]["unit"] == "T lane-ops/s"  # an FMA counts once
    assert per["preprocess"]["unit"] == "GB/s"
    assert per["blend"]["achieved"] == pytest.approx(bench.OPS_PER_EVAL_FWD * 1e9 / 2e-3 / 1e12)
    assert per["blend_backward"]["achieved"] == pytest.approx(bench.OPS_PER_EVAL_BWD * 5e8 / 4e-3 / 1e12)
    assert per["blend"]["exp2"]["frac"] == pytest.approx(1e9 / 2e-3 / 1e12)
    assert per["blend_backward"]["also_writes_bytes"] == 236 * N
    assert roof["kernel"] == "blend_backward"  # the longest stage


def test_traffic_scaled_by_units(tmp_path, monkeypatch):
    """A capture of a small case carries over to the bench workload as bytes
    per unit: preprocess per Gaussian, the pair stages per pair, the
    preprocess backward per visible record."""
    rows = []
    SC = "gs::scatter_kernel(const gs_camera *, Ws)"
    PB = "gs::preprocess_backward_kernel<1, true>(const gs_camera *, GaussInB, Ws, GradOut)"
    for i, name in enumerate((PRE, SC, PB, BWD)):
        _launch(rows, i, name, 1000, 0, 0)
    lst = tmp_path / "launches.csv"
    _write_list(lst, rows)
    for f, name, b in (("a.csv", PRE, 1000), ("b.csv", SC, 300), ("c.csv", PB, 100)):
        _write_raw(tmp_path / f, [(name, b, "byte", 0, "byte")])
    line = {"config": {"gaussians_per_gpu": 100}, "stats": {"records": 100, "pairs": 30, "visible": 25}}
    sj = tmp_path / "small.json"
    sj.write_text("log line\n" + json.dumps(line) + "\n")
    out = tmp_path / "traffic.json"
    kern = bench.ncu_traffic(str(lst), [str(tmp_path / f) for f in ("a.csv", "b.csv", "c.csv")], "cmd",
                             stats_json=str(sj), out_path=str(out))
    assert kern["preprocess_kernel"]["unit"] == "gaussians" and kern["preprocess_kernel"]["bytes_per_unit"] == 10.0
    assert kern["scatter_kernel"]["bytes_per_unit"] == 10.0  # 300 bytes over 30 pairs
    assert kern["preprocess_backward_kernel"]["bytes_per_unit"] == 4.0  # 100 bytes over 25 visible
    monkeypatch.setattr(bench, "peaks", lambda: (1000.0, "measured"))
    monkeypatch.setattr(bench, "dram_traffic", lambda: kern)
    stats = {"n_records": 1000, "n_visible": 200, "n_pairs": 500}
    _, per = bench.rooflines(stats, {"preprocess": 1.0, "scatter": 1.0, "preprocess_backward": 1.0}, n_eval_fwd=1,
                             n_eval_bwd=1, n_pix=1, N=1000, sm_count=1, sm_mhz=1000.0)
    assert per["preprocess"]["traffic"] == pytest.approx(10.0 * 1000)
    assert per["scatter"]["traffic"] == pytest.approx(10.0 * 500)
    assert per["preprocess_backward"]["traffic"] == pytest.approx(4.0 * 200)


def test_ncu_table_from_raw_pages(tmp_path, capsys):
    """The kernel summary's table: units converted (us -> us, Gbyte -> MB),
    SM active over elapsed, stall ratios, blank cells for missing metrics."""
    h = ["ID", "Kernel Name", "gpu__time_duration.sum", "dram__bytes_read.sum", "sm__cycles_active.avg",
         "sm__cycles_elapsed.avg", "smsp__average_warps_issue_stalled_wait_per_issue_active.ratio"]
    p = tmp_path / "raw_k.csv"
    with open(p, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(h)
        w.writerow(["", "", "us", "Gbyte", "cycle", "cycle", ""])
        w.writerow(["0", "void k(int)", "545.7", "1.25", "50", "200", "1.5"])
    lines = bench.ncu_table([str(p)])
    assert lines[0] == "| metric | k |"
    rows = {ln.split(" | ")[0].lstrip("| "): ln.split(" | ")[1].rstrip(" |") for ln in lines[2:]}
    assert rows["duration (us, serialised)"] == "545.7"
    assert rows["DRAM read (MB)"] == "1250.0"
    assert rows["SM cycles active / elapsed"] == "0.25"
    assert rows["stall wait (per issue)"] == "1.50"
    assert rows["DRAM write (MB)"] == ""  # not in the report
