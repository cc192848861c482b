"""Host logic of bench.py, no GPU: the ncu launch-list summary (per-call DRAM
bytes of the forward and backward kernels, unit conversion, foreign kernels left
out), the stale-hash rule of the traffic file, and the roofline arithmetic
against hand-computed figures."""
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


def test_ncu_summary_bytes_per_call(tmp_path):
    rows, i = [], 0
    for call in range(2):  # two forwards: two merge passes each; one backward
        for name, ns, rd, wr in (("void gs::preprocess_kernel<1, false>(const gs_camera *, GaussIn, Ws)", 2000, 100, 50),
                                 ("gs::merge_pass_kernel(Ws, int)", 300, 10, 10),
                                 ("gs::merge_pass_kernel(Ws, int)", 300, 20, 0),
                                 ("void gs::blend_persistent_kernel<2, 1>(const gs_camera *, Ws, OutPtrs)", 3000, 40, 4)):
            _launch(rows, i, name, ns, rd, wr)
            i += 1
    _launch(rows, i, "void gs::blend_backward_kernel<2, 1>(const gs_camera *, Ws, const float *)", 5000, 7, 1000)
    i += 1
    _launch(rows, i, "void at::native::vectorized_elementwise_kernel<4>(int)", 9000, 1, 1)  # not ours
    p = tmp_path / "launches.csv"
    with open(p, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(HEADER)
        w.writerows(rows)
    out = tmp_path / "traffic.json"
    kern = bench.ncu_summary(str(p), "ncu ... python bench.py", out_path=str(out))
    assert kern["preprocess_kernel"]["dram_bytes_per_call"] == 150
    assert kern["merge_pass_kernel"]["launches_per_call"] == 2
    assert kern["merge_pass_kernel"]["dram_bytes_per_call"] == 40
    assert kern["blend_persistent_kernel"]["ms_per_call_under_ncu"] == pytest.approx(0.003)
    assert kern["blend_backward_kernel"]["dram_bytes_per_call"] == 1007  # one backward call
    assert "vectorized_elementwise_kernel" not in kern
    t = json.loads(out.read_text())
    assert t["source_hash"] == bench.source_hash() and t["kernels"] == kern


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
    _launch(rows, 0, "void gs::preprocess_kernel<1, false>(const gs_camera *, GaussIn, Ws)", 2000, 600, 400)
    _launch(rows, 1, "gs::scatter_kernel(const gs_camera *, Ws)", 500, 100, 200)
    _launch(rows, 2, "gs::preprocess_backward_kernel<1, true>(const gs_camera *, GaussInB, Ws, GradOut)", 900, 50, 50)
    _launch(rows, 3, "void gs::blend_backward_kernel<2, 1>(const gs_camera *, Ws, const float *)", 500, 1, 1)
    p = tmp_path / "launches.csv"
    with open(p, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(HEADER)
        w.writerows(rows)
    line = {"config": {"gaussians_per_gpu": 100}, "stats": {"records": 100, "pairs": 30, "visible": 25}}
    sj = tmp_path / "small.json"
    sj.write_text("log line\n" + json.dumps(line) + "\n")
    out = tmp_path / "traffic.json"
    kern = bench.ncu_summary(str(p), "cmd", out_path=str(out), stats_json=str(sj))
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
