#!/usr/bin/env python
"""Throughput of batched RGB-D Gaussian-splatting rendering on GB300.

Workload (one step): 64 environments, each its own synthetic indoor room of
U[300k, 1.5M] Gaussians (uneven), one 256x256 RGB-D camera per env at a random
pose; forward (EWA projection + SH-3 colour, binning, per-tile sort, blending)
and backward (gradients w.r.t. all Gaussian parameters) in one captured CUDA
graph, SH stored in FP16, blending by a persistent grid, tile size and batch
depth chosen by the autotuner.  The paper measures its renderer inside
Habitat-Lab at 256x256 with 300K-7M Gaussians (Sec. 4.5, Table 6); its scans
are not available, the synthetic rooms stand in for them.

Prints one JSON line (rank 0).  value = env-frames/s of the whole job
(forward + backward), with the forward alone, the plain per-env FP32 path, the
live per-stage timing of the dominant kernel against its roofline, the
end-to-end number through the public API with host buffers, the clocks seen
during the timed region and the FP64 CPU oracle on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RGB-D frames/s at 64 envs (fwd, fwd+bwd) vs plain per-env path; % roofline"
UNIT = "env-frames/s"
N_ENVS, W, H = 64, 256, 256
N_MIN, N_MAX = 300_000, 1_500_000
# (tile_w, tile_h, batch_depth, pixels per thread x, y)
TILE_CANDIDATES = [(16, 16, 256, 1, 1), (16, 16, 256, 2, 2), (16, 16, 128, 2, 2), (16, 16, 128, 2, 1),
                   (16, 8, 128, 1, 1), (16, 8, 128, 2, 1), (16, 8, 64, 2, 2), (16, 8, 128, 2, 2), (8, 8, 64, 1, 1),
                   (8, 8, 128, 1, 1), (8, 8, 64, 2, 1), (32, 16, 256, 2, 2)]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def smi_index(local: int) -> int:
    """nvidia-smi index of the local CUDA device (CUDA_VISIBLE_DEVICES remaps)."""
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [x.strip() for x in vis.split(",") if x.strip()]
    if local < len(ids) and ids[local].isdigit():
        return int(ids[local])
    return local


def dist_init():
    import torch

    from paper_2604_12626_gb300 import shard

    return shard.init("nccl" if torch.cuda.is_available() else "gloo")


def barrier(ws):
    from paper_2604_12626_gb300 import shard

    shard.barrier(ws)


def max_over_ranks(x, ws):
    from paper_2604_12626_gb300 import shard

    return shard.max_over_ranks(x, ws)


# ---------------------------------------------------------------------------
# CPU oracle baseline (test infrastructure; timed as it stands)
# ---------------------------------------------------------------------------
def oracle_step(env_ids, seed0, budget_s=None, scale=1.0):
    """FP64 oracle forward + backward of whole envs; returns (envs done, seconds)."""
    import oracle
    from paper_2604_12626_gb300 import synth

    oracle.build()
    sizes = synth.batch_sizes(max(env_ids) + 1, N_MIN, N_MAX, seed0, scale)
    done, t_total = 0, 0.0
    rng = np.random.default_rng(0)
    for e in env_ids:
        g = synth.room_scene(sizes[e], seed=seed0 + e)
        cam = synth.room_camera(seed0 + e, W, H)
        d_rgb = rng.standard_normal((3, H, W))
        d_depth = rng.standard_normal((H, W)) * 0.1
        t0 = time.perf_counter()
        oracle.render(g, cam, W, H)
        oracle.render_backward(g, cam, W, H, d_rgb, d_depth)
        t_total += time.perf_counter() - t0
        done += 1
        if budget_s is not None and t_total >= budget_s:
            break
    return done, t_total


def oracle_configs(seed0=0):
    """The FP64 oracle on the other configurations, on the host cores, at 1
    thread and at all cores (OpenMP over image row bands): forward of the
    5k-Gaussian box at 128x128, of a 1M-Gaussian room at 640x480 and of env 0
    of the 64-env batch at 256x256; the adjoint (1 thread) of that env; and one
    of the 16 views of the training step (500k room + 2 posed avatars, 512x512)
    forward + adjoint, scaled to the 16-view step."""
    import oracle
    from paper_2604_12626_gb300 import synth

    oracle.build()
    cores = os.cpu_count() or 1
    out = {"cores": cores}

    def t_of(fn):
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    def both(name, g, cam, Wc, Hc):
        t1 = t_of(lambda: oracle.render(g, cam, Wc, Hc, nthreads=1))
        tn = t_of(lambda: oracle.render(g, cam, Wc, Hc, nthreads=0))
        out[name] = {"fwd_frames_per_s_1_thread": 1.0 / t1, f"fwd_frames_per_s_{cores}_cores": 1.0 / tn,
                     "gaussians": int(g["means"].shape[0]), "width": Wc, "height": Hc}

    both("box_5k_128px", synth.box_scene(5000, seed=0), synth.identity_camera(128, 128), 128, 128)
    both("room_1M_640x480", synth.room_scene(1_000_000, seed=1), synth.room_camera(1, 640, 480), 640, 480)
    n0 = synth.batch_sizes(1, N_MIN, N_MAX, seed0)[0]
    g0, cam0 = synth.room_scene(n0, seed=seed0), synth.room_camera(seed0, W, H)
    both("batch_env0_256px", g0, cam0, W, H)
    rng = np.random.default_rng(0)
    tb = t_of(lambda: oracle.render_backward(g0, cam0, W, H, rng.standard_normal((3, H, W)),
                                              rng.standard_normal((H, W))))
    out["batch_env0_256px"]["bwd_frames_per_s_1_thread"] = 1.0 / tb
    wl = synth.training_scene(seed=0)
    av = wl["avatars"]
    pm, pc = oracle.lbs(av["means"], av["log_scales"], av["quats"], av["joint_ids"].astype(np.int32), av["weights"],
                        av["avatar_of"], wl["G"].astype(np.float64))
    room, ns, m = wl["room"], wl["room"]["means"].shape[0], av["means"].shape[0]
    g = dict(means=np.concatenate([room["means"].astype(np.float64), pm]),
             log_scales=np.concatenate([room["log_scales"], np.zeros((m, 3), np.float32)]),
             quats=np.concatenate([room["quats"], np.tile(np.float32([1, 0, 0, 0]), (m, 1))]),
             opacity_logits=np.concatenate([room["opacity_logits"], av["opacity_logits"]]),
             sh=np.concatenate([room["sh"], av["sh"]]), cov3d=np.concatenate([np.zeros((ns, 6)), pc]),
             use_cov=np.concatenate([np.zeros(ns, np.uint8), np.ones(m, np.uint8)]))
    cam = wl["cams"][0]
    tf = t_of(lambda: oracle.render(g, cam, 512, 512, nthreads=0))
    tb = t_of(lambda: oracle.render_backward(g, cam, 512, 512, np.ones((3, 512, 512)), np.zeros((512, 512))))
    nv = wl["cams"].shape[0]
    out["training_16x512px"] = {"step_s_estimate": nv * (tf + tb), "view_frames_per_s": 1.0 / (tf + tb),
                                "sample": f"view 0 of {nv}: forward on {cores} cores {tf:.2f} s + adjoint on 1 "
                                          f"thread {tb:.2f} s, scaled to {nv} views"}
    return out


def run_reference(args, ws, rank):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    envs_per_step = 1
    for _ in range(args.warmup):
        oracle_step([0], 0, scale=args.scale)
    t = 0.0
    n = 0
    for k in range(args.steps):
        d, s = oracle_step([(k * envs_per_step + i) % N_ENVS for i in range(envs_per_step)], 0, scale=args.scale)
        n += d
        t += s
    value = n / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "FP64 CPU oracle, forward+backward of one 256x256 room env (300k-1.5M "
                                   "Gaussians) per step, env k at step k"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n} env(s) of the 64-env batch, forward (OpenMP) + backward (1 thread)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def tune_fwd_bwd(api, rend, G, cams, candidates, N, dev, reps=2):
    """The autotuner on the whole step: gs_autotune times the forward per
    candidate; the backward is timed here with the same CUDA events, and the
    candidate with the fastest forward + backward wins."""
    import torch

    outs = rend.alloc_outputs()
    d_rgb = torch.zeros((rend.batch.n_views, 3, rend.height, rend.width), device=dev)
    d_depth = torch.zeros((rend.batch.n_views, rend.height, rend.width), device=dev)
    grads = dict(means=torch.empty((N, 3), device=dev), log_scales=torch.empty((N, 3), device=dev),
                 quats=torch.empty((N, 4), device=dev), opacity_logits=torch.empty((N,), device=dev),
                 sh=torch.empty((N, 16, 3), device=dev))
    best, best_ms = None, None
    base = api.GsRenderConfig.from_buffer_copy(rend.cfg)
    for cand in candidates:
        rend.cfg = api.GsRenderConfig.from_buffer_copy(base)
        try:
            (_, fwd_ms) = rend.autotune(G, cams, [cand], reps=reps, out=outs)
        except api.GsError:
            continue
        rend.backward(G, cams, d_rgb, d_depth, grads=grads)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            rend.forward(G, cams, out=outs)
            rend.backward(G, cams, d_rgb, d_depth, grads=grads)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        if best_ms is None or ms < best_ms:
            best, best_ms = list(cand), ms
    rend.cfg = api.GsRenderConfig.from_buffer_copy(base)
    rend.cfg.tile_w, rend.cfg.tile_h, rend.cfg.batch_depth, rend.cfg.pix_x, rend.cfg.pix_y = best
    return best, best_ms

# Algorithmic work per unit: bytes for the memory-bound stages (rooflines()),
# FP32 lane operations per evaluation for the two blend kernels.
OPS_PER_EVAL_FWD = 17   # offset, quadratic form, exp, alpha clamp / skip, T update, 3 colours + depth
OPS_PER_EVAL_BWD = 40   # recomputed alpha, T_prev, dL/dalpha, conic / centre / colour / depth terms
# the kernels of each stage (the blend at 2x1 pixels per thread is the quarter-list kernel)
KERNELS_OF_STAGE = {"preprocess": ("preprocess_kernel",), "scan": ("scan_bins_kernel",),
                    "scatter": ("scatter_kernel",), "sort": ("sort_chunks_kernel", "sort_small_kernel", "merge_pass_kernel"),
                    "blend": ("blend_persistent_kernel", "blendq_persistent_kernel"),
                    "blend_backward": ("blend_backward_kernel",), "preprocess_backward": ("preprocess_backward_kernel",)}
CSRC = os.path.join(ROOT, "paper_2604_12626_gb300", "csrc")


def source_hash():
    import hashlib

    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(CSRC, name), "rb") as f:
                h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def dram_traffic():
    """Per-launch DRAM bytes of each kernel from the committed ncu summary, or
    {} once the kernel sources have changed since it was taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            t = json.load(f)
    except Exception:
        return {}
    if t.get("source_hash") != source_hash():
        return {}
    return t.get("kernels", {})


FWD_KERNELS = ("setup_kernel", "preprocess_kernel", "scan_bins_kernel", "scatter_kernel", "sort_chunks_kernel",
               "sort_small_kernel", "merge_pass_kernel", "blend_persistent_kernel", "blendq_persistent_kernel")
BWD_KERNELS = ("clear_record_grads_kernel", "blend_backward_kernel", "preprocess_backward_kernel")


# the unit each kernel's DRAM traffic scales with, for carrying bytes measured
# on a small capture over to the bench workload: the blend backward's bytes are
# mostly the dense gradient clear (per Gaussian), the pair stages' per pair
UNIT_OF_KERNEL = {"setup_kernel": "gaussians", "preprocess_kernel": "gaussians", "scan_bins_kernel": "pairs",
                  "scatter_kernel": "pairs", "sort_chunks_kernel": "pairs", "sort_small_kernel": "pairs",
                  "merge_pass_kernel": "pairs", "blend_persistent_kernel": "pairs", "blendq_persistent_kernel": "pairs",
                  "clear_record_grads_kernel": "visible", "blend_backward_kernel": "gaussians",
                  "preprocess_backward_kernel": "visible"}


def _units(stats_line):
    st = stats_line.get("stats", {})
    return {"gaussians": stats_line.get("config", {}).get("gaussians_per_gpu") or st.get("records"),
            "pairs": st.get("pairs"), "visible": st.get("visible")}


def _kernel_name(full):
    import re

    m = re.match(r"(?:void )?(?:gs::)?([A-Za-z_0-9]+)", full)
    return m.group(1) if m else full[:40]


def _launch_list(csv_path):
    """Per-kernel launches, ms and DRAM bytes (where captured) of an ncu --csv
    launch list, and the number of forward and backward calls in it (launches
    of the preprocess and of the blend backward)."""
    import collections
    import csv

    with open(csv_path) as f:
        rows = [r for r in csv.reader(f) if len(r) > 10]
    h, rows = rows[0], rows[1:]
    iK, iM, iV, iID, iU = (h.index(x) for x in ("Kernel Name", "Metric Name", "Metric Value", "ID", "Metric Unit"))
    per, names = collections.defaultdict(dict), {}
    to_ms = {"nsecond": 1e-6, "ns": 1e-6, "usecond": 1e-3, "us": 1e-3, "msecond": 1.0, "ms": 1.0, "second": 1e3}
    for r in rows:
        v = float(r[iV].replace(",", ""))
        if r[iM] == "gpu__time_duration.sum":
            v *= to_ms.get(r[iU], 1e-6)
        per[r[iID]][r[iM]] = v
        names[r[iID]] = _kernel_name(r[iK])
    agg = collections.OrderedDict()
    for i, d in per.items():
        a = agg.setdefault(names[i], dict(launches=0, ms=0.0, rd=0.0, wr=0.0))
        a["launches"] += 1
        a["ms"] += d.get("gpu__time_duration.sum", 0.0)
        a["rd"] += d.get("dram__bytes_read.sum", 0.0)
        a["wr"] += d.get("dram__bytes_write.sum", 0.0)
    n_fwd = max(agg.get("preprocess_kernel", {}).get("launches", 0), 1)
    n_bwd = max(agg.get("blend_backward_kernel", {}).get("launches", 0), 1)
    return agg, n_fwd, n_bwd


def ncu_summary(csv_path):
    """Prints the per-kernel table of an ncu --csv launch list of this bench
    (launches, time, share of this repository's kernels; DRAM bytes where the
    list has them) and returns per kernel its launches and ms per call."""
    agg, n_fwd, n_bwd = _launch_list(csv_path)
    ours = {k: a for k, a in agg.items() if k in FWD_KERNELS + BWD_KERNELS}
    tot = sum(a["ms"] for a in ours.values())
    kern = {}
    print(f"{'kernel':28s} {'launches':>8s} {'total ms':>9s} {'share':>6s} {'ms/launch':>9s} {'DRAM MB/launch':>14s}")
    for k, a in sorted(ours.items(), key=lambda x: -x[1]["ms"]):
        calls = n_fwd if k in FWD_KERNELS else n_bwd
        kern[k] = {"launches_per_call": a["launches"] / calls, "ms_per_call_under_ncu": a["ms"] / calls}
        print(f"{k:28s} {a['launches']:8d} {a['ms']:9.3f} {100 * a['ms'] / tot:5.1f}% {a['ms'] / a['launches']:9.4f} "
              f"{(a['rd'] + a['wr']) / a['launches'] / 1e6:14.1f}")
    rest = [a for k, a in agg.items() if k not in ours]
    print(f"(other kernels: {sum(a['launches'] for a in rest)} launches, {sum(a['ms'] for a in rest):.3f} ms; "
          f"{n_fwd} forward and {n_bwd} backward calls)")
    return kern


def _raw_dram(csv_path):
    """(kernel, DRAM bytes) of each launch in the raw page of an ncu report
    (`ncu -i REPORT --page raw --csv`)."""
    import csv

    with open(csv_path) as f:
        rows = list(csv.reader(f))
    h, unit_row, data = rows[0], rows[1], rows[2:]
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12}
    iK = h.index("Kernel Name")
    cols = [h.index("dram__bytes_read.sum"), h.index("dram__bytes_write.sum")]
    out = []
    for r in data:
        if len(r) != len(h):
            continue
        b = sum(float(r[i].replace(",", "")) * scale[unit_row[i]] for i in cols)
        out.append((_kernel_name(r[iK]), b))
    return out


# rows of the full-capture table: (label, metric, scale); None = SM active / elapsed
NCU_TABLE = (
    ("duration (us, serialised)", "gpu__time_duration.sum", 1e-3),
    ("warp instructions (M)", "smsp__inst_executed.sum", 1e-6),
    ("issue slots busy (% of active)", "smsp__issue_active.avg.pct_of_peak_sustained_active", 1.0),
    ("warps active (% of peak)", "sm__warps_active.avg.pct_of_peak_sustained_active", 1.0),
    ("registers per thread", "launch__registers_per_thread", 1.0),
    ("ALU pipe (% active)", "sm__inst_executed_pipe_alu.avg.pct_of_peak_sustained_active", 1.0),
    ("FMA pipe (% active)", "sm__inst_executed_pipe_fma.avg.pct_of_peak_sustained_active", 1.0),
    ("XU pipe (% active)", "sm__inst_executed_pipe_xu.avg.pct_of_peak_sustained_active", 1.0),
    ("LSU pipe (% active)", "sm__inst_executed_pipe_lsu.avg.pct_of_peak_sustained_active", 1.0),
    ("DRAM read (MB)", "dram__bytes_read.sum", 1e-6),
    ("DRAM write (MB)", "dram__bytes_write.sum", 1e-6),
    ("DRAM throughput (% of peak)", "gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed", 1.0),
    ("shared bank conflicts (M)", "l1tex__data_bank_conflicts_pipe_lsu_mem_shared.sum", 1e-6),
    ("SM cycles active / elapsed", None, 1.0),
)
NCU_STALLS = ("long_scoreboard", "short_scoreboard", "wait", "barrier", "not_selected", "math_pipe_throttle",
              "mio_throttle", "lg_throttle")


def _raw_first(csv_path):
    """{metric: value in base units} of the first launch in the raw page of
    an ncu report (`ncu -i REPORT --page raw --csv`): times in ns, bytes in
    bytes."""
    import csv

    with open(csv_path) as f:
        rows = list(csv.reader(f))
    h, unit_row, vals = rows[0], rows[1], rows[2]
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1.0, "ns": 1.0, "usecond": 1e3,
             "us": 1e3, "msecond": 1e6, "ms": 1e6}
    out = {}
    for k, u, v in zip(h, unit_row, vals):
        try:
            out[k] = float(v.replace(",", "")) * scale.get(u, 1.0)
        except ValueError:
            pass
    return out


def ncu_table(raw_csvs):
    """Markdown table of the figures the kernel summary quotes, one column per
    report (raw-page CSVs of `ncu --set full` captures, one launch each)."""
    ds = [_raw_first(p) for p in raw_csvs]
    names = [os.path.basename(p).replace("raw_", "").replace(".csv", "") for p in raw_csvs]
    lines = ["| metric | " + " | ".join(names) + " |", "|---" * (len(names) + 1) + "|"]

    def cell(x, fmt):
        return "" if x is None else format(x, fmt)

    for label, key, sc in NCU_TABLE:
        if key is None:
            cells = [cell(d["sm__cycles_active.avg"] / d["sm__cycles_elapsed.avg"]
                          if d.get("sm__cycles_elapsed.avg") else None, ".2f") for d in ds]
        else:
            cells = [cell(d[key] * sc if key in d else None, ".1f") for d in ds]
        lines.append(f"| {label} | " + " | ".join(cells) + " |")
    for st in NCU_STALLS:
        key = f"smsp__average_warps_issue_stalled_{st}_per_issue_active.ratio"
        lines.append(f"| stall {st} (per issue) | " + " | ".join(cell(d.get(key), ".2f") for d in ds) + " |")
    print("\n".join(lines))
    return lines


def ncu_traffic(launch_csv, raw_csvs, command, stats_json=None, out_path=None):
    """profiles/dram_traffic.json (or out_path) from one-kernel captures: each
    kernel's DRAM bytes per launch from its own report (raw-page CSVs; a kernel
    launched several times per call is captured over the launches of one whole
    call), its launches per call from a time-only launch list of the same launch
    shape whose calls all ran to the end, and -- with stats_json, the captured
    run's JSON line -- its bytes per unit (UNIT_OF_KERNEL), which the bench
    multiplies by its own counts.  Tagged with the kernel sources' hash."""
    import collections

    agg, n_fwd, n_bwd = _launch_list(launch_csv)
    units = None
    if stats_json:
        with open(stats_json) as f:
            units = _units(json.loads(f.read().strip().splitlines()[-1]))
    per = collections.defaultdict(list)
    for p in raw_csvs:
        for k, b in _raw_dram(p):
            per[k].append(b)
    kern = {}
    for k in sorted(per):
        if k not in FWD_KERNELS + BWD_KERNELS or k not in agg:
            continue
        lpc = agg[k]["launches"] / (n_fwd if k in FWD_KERNELS else n_bwd)
        bpl = sum(per[k]) / len(per[k])
        kern[k] = {"dram_bytes_per_launch": bpl, "captured_launches": len(per[k]), "launches_per_call": lpc,
                   "dram_bytes_per_call": bpl * lpc}
        if units and units.get(UNIT_OF_KERNEL.get(k)):
            kern[k]["unit"] = UNIT_OF_KERNEL[k]
            kern[k]["bytes_per_unit"] = kern[k]["dram_bytes_per_call"] / units[UNIT_OF_KERNEL[k]]
        print(f"{k:28s} {len(per[k]):3d} launches captured  {bpl / 1e6:10.1f} MB/launch  x {lpc:.2f} per call"
              + (f"  {kern[k]['bytes_per_unit']:8.1f} B per {kern[k]['unit']}" if "unit" in kern[k] else ""))
    out = {"source_hash": source_hash(),
           "what": "DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of each kernel per gs_render / "
                   "gs_render_backward call: bytes per launch from a capture of that kernel alone, times its "
                   "launches per call; stale once the kernel sources change (source_hash over csrc/)",
           "command": command, "units_of_capture": units, "kernels": kern}
    with open(out_path or os.path.join(ROOT, "profiles", "dram_traffic.json"), "w") as f:
        json.dump(out, f, indent=1)
    return kern


def exp2_rate(api, torch, dev, stream, sm_count):
    """Measured exp2 throughput of the special-function unit (gs_exp2_rate):
    8 CTAs of 256 threads per SM, 4096 steps of 8 chains each."""
    out = torch.empty(sm_count * 8 * 256, device=dev)
    api.exp2_rate(sm_count * 8, 64, out, stream)  # warm-up
    ops = sm_count * 8 * 256 * 4096 * 8
    ms = _event_ms(torch, stream, lambda: api.exp2_rate(sm_count * 8, 4096, out, stream), reps=3)
    return ops / (ms * 1e-3)


def rooflines(stats, stage_ms, n_eval_fwd, n_eval_bwd, n_pix, N, sm_count, sm_mhz, exp_rate=None):
    """Achieved vs peak per kernel, from live CUDA-event stage times."""
    hbm, peak_kind = peaks()
    mhz = sm_mhz or 2070.0
    alu_peak = sm_count * 128 * mhz * 1e6 / 1e12  # FP32 lanes x clock, T lane-ops/s
    R, nvis, P = stats["n_records"], stats["n_visible"], stats["n_pairs"]
    traffic = dram_traffic()
    # algorithmic bytes per launch (FP16 SH storage; one view per env, so a
    # visible record is one seen Gaussian)
    mem = {
        # means of every Gaussian, the visibility bits; per visible record its
        # scales + rotation, opacity logit, SH, the 48-byte record and the
        # 64-byte gradient row it clears
        "preprocess": 12 * N + R // 8 + nvis * (28 + 4 + 96 + 48 + 64),
        "scatter": nvis * 20 + 12 * P,
        "sort": 16 * P,
        # the visibility bits; per seen Gaussian its parameters (means, scales +
        # rotation, opacity logit, SH), its 64-byte gradient row and its
        # 236-byte parameter gradient
        "preprocess_backward": R // 8 + nvis * (12 + 28 + 4 + 96 + 64 + 236),
    }
    ops = {"blend": OPS_PER_EVAL_FWD * n_eval_fwd, "blend_backward": OPS_PER_EVAL_BWD * n_eval_bwd}
    ms = dict(stage_ms)
    if "sort" in ms:
        ms["sort"] = ms["sort"] + ms.get("merge", 0.0)
    out = {}
    for k, b in mem.items():
        if k in ms and ms[k] > 0:
            a = b / (ms[k] * 1e-3) / 1e9
            out[k] = {"bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm,
                      "algorithmic": b, "ms": ms[k], "peak_kind": peak_kind}
    for k, f in ops.items():
        if k in ms and ms[k] > 0:
            a = f / (ms[k] * 1e-3) / 1e12
            out[k] = {"bound": "alu", "achieved": a, "peak": alu_peak, "unit": "T lane-ops/s", "frac": a / alu_peak,
                      "algorithmic": f, "ms": ms[k],
                      "peak_kind": f"derived: {sm_count} SMs x 128 FP32 lanes x {mhz:.0f} MHz"}
    live = {"gaussians": N, "pairs": P, "visible": nvis}
    for k, v in out.items():
        # bytes per unit from the capture times this run's units (else the
        # captured call's bytes, when the capture was of this workload)
        tb = [traffic[x]["bytes_per_unit"] * live[traffic[x]["unit"]] if "bytes_per_unit" in traffic[x]
              else traffic[x]["dram_bytes_per_call"] for x in KERNELS_OF_STAGE[k] if x in traffic]
        v["traffic"] = float(sum(tb)) if tb else None
    for k, n_ev in (("blend", n_eval_fwd), ("blend_backward", n_eval_bwd)):
        if exp_rate and k in out:
            # one exp per evaluation, against the measured exp2 rate
            a = n_ev / (out[k]["ms"] * 1e-3)
            out[k]["exp2"] = {"achieved_gops": a / 1e9, "peak_gops": exp_rate / 1e9, "frac": a / exp_rate}
    if "blend_backward" in out:
        # the persistent backward also clears the dense parameter gradients
        # (236 bytes per Gaussian; the preprocess backward then writes the seen rows)
        out["blend_backward"]["also_writes_bytes"] = 236 * N
    dom = max(out, key=lambda k: out[k]["ms"])
    roof = dict(out[dom], kernel=dom)
    return roof, out


def _event_ms(torch, stream, fn, reps=10):
    with torch.cuda.stream(stream):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def avatar_and_composite_rows(api, synth, torch, dev, stream, outs, hbm_peak):
    """CUDA-event times of the kernels outside the headline step: LBS deform
    and its adjoint (100 B per avatar Gaussian forward: 64 B of canonical
    parameters, weights and joint ids read, 36 B of posed mean and covariance
    written), keyframe
    interpolation + forward kinematics of 256 avatars, and the composite of two
    64 x 256 x 256 RGB-D layers (48 B per pixel)."""
    n_av, n_per, n_frames = 256, 50_000, 30
    base = [synth.avatar_canonical(n_per, k) for k in range(8)]  # 8 distinct avatars, tiled over 32 envs
    cat = {k: np.concatenate([base[a % 8][k] for a in range(n_av)]) for k in base[0]}
    m = n_av * n_per
    T = lambda x, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(x)).to(dev, dt)  # noqa: E731
    av = api.Avatars(T(cat["means"]), T(cat["log_scales"]), T(cat["quats"]), T(cat["joint_ids"].view(np.int16),
                     torch.int16), T(cat["weights"]), T(np.repeat(np.arange(n_av), n_per).astype(np.int32), torch.int32),
                     n_av, synth.N_JOINTS)
    del cat
    rng = np.random.default_rng(7)
    frames = T(np.stack([np.stack([synth.random_pose(17 * a + f % 4) for f in range(n_frames)])
                         for a in range(n_av)]).astype(np.float32))
    t = T(rng.uniform(0, n_frames - 1, n_av).astype(np.float32))
    from scipy.spatial.transform import Rotation

    local = T(Rotation.from_rotvec(rng.normal(0, 0.3, (n_av * synth.N_JOINTS, 3))).as_matrix()
              .reshape(n_av, synth.N_JOINTS, 3, 3).astype(np.float32))
    root = T(np.tile(np.hstack([np.eye(3), [[1.0], [2.0], [0.9]]]).astype(np.float32), (n_av, 1, 1)))
    rest = T(synth.REST_JOINTS.astype(np.float32))
    G = torch.empty((n_av, synth.N_JOINTS, 3, 4), device=dev)
    om, oc = torch.empty((m, 3), device=dev), torch.empty((m, 6), device=dev)
    gr = dict(means=torch.zeros((m, 3), device=dev), log_scales=torch.zeros((m, 3), device=dev),
              quats=torch.zeros((m, 4), device=dev), G=torch.zeros_like(G))
    interp_ms = _event_ms(torch, stream, lambda: api.interpolate_joints(frames, t, out=G, stream=stream))
    fk_ms = _event_ms(torch, stream, lambda: api.forward_kinematics(local, root, rest, synth.PARENTS, out=G,
                                                                   stream=stream))
    # proxy capsules of the posed avatars (8 per env over 32 envs) and the two
    # avatar queries for 4096 candidate steps per env
    radius = T(np.full(synth.N_JOINTS, 0.08, np.float32))
    caps = torch.empty((n_av, synth.N_JOINTS, 8), device=dev)
    caps_ms = _event_ms(torch, stream, lambda: api.avatar_capsules(G, rest, synth.PARENTS, radius, out=caps,
                                                                  stream=stream))
    n_qenv, n_q = 32, 32 * 4096
    cap_off = torch.arange(0, n_av * synth.N_JOINTS + 1, (n_av // n_qenv) * synth.N_JOINTS, device=dev,
                           dtype=torch.int64)
    q_env = T(np.repeat(np.arange(n_qenv), n_q // n_qenv).astype(np.int32), torch.int32)
    q0 = T(np.stack([rng.uniform(0, 3, n_q), rng.uniform(0, 4, n_q), rng.uniform(0.1, 1.8, n_q)], 1).astype(np.float32))
    q1 = q0 + T(rng.normal(0, 0.25, (n_q, 3)).astype(np.float32))
    q_out = (torch.empty(n_q, device=dev), torch.empty(n_q, dtype=torch.int32, device=dev), torch.empty(n_q, device=dev),
             torch.empty(n_q, dtype=torch.uint8, device=dev))
    query_ms = _event_ms(torch, stream, lambda: api.capsule_query(caps.view(-1, 8), cap_off, q_env, q0, q1, 0.1,
                                                                 out=q_out, stream=stream))
    q_blocked = float(q_out[3].float().mean().item())
    deform_ms = _event_ms(torch, stream, lambda: api.deform(av, G, om, oc, stream=stream))
    dmean, dcov = torch.ones_like(om), torch.ones_like(oc)
    deform_bwd_ms = _event_ms(torch, stream, lambda: api.deform_backward(av, G, dmean, dcov, gr, stream=stream), 5)
    fwd_bytes = 100 * m
    bwd_bytes = m * (12 + 12 + 16 + 8 + 16 + 4 + 12 + 24 + 40)  # inputs, upstream grads, canonical grads (RMW excluded)
    del av, om, oc, gr, dmean, dcov, frames
    # composite of the bench frames with a second layer of the same shape
    V, _, H, W = outs[0].shape
    rgb_b = torch.rand_like(outs[0])
    dep_b = torch.rand_like(outs[1]) * 8.0
    rgb_o, dep_o = torch.empty_like(outs[0]), torch.empty_like(outs[1])
    comp_ms = _event_ms(torch, stream, lambda: api.composite_nearest(outs[0], outs[1], rgb_b, dep_b,
                                                                    out=(rgb_o, dep_o), stream=stream))
    comp_bytes = 48 * V * H * W
    # the mesh layer of a mixed scene: each env's room mesh, one view per env
    meshes = [synth.room_mesh(e % 8, n_boxes=12, grid=16) for e in range(V)]
    tri_off = np.cumsum([0] + [mm["triangles"].shape[0] for mm in meshes])
    v_off = np.cumsum([0] + [mm["vertices"].shape[0] for mm in meshes])
    mesh = api.Mesh.from_numpy(dict(vertices=np.concatenate([mm["vertices"] for mm in meshes]),
                                    colors=np.concatenate([mm["colors"] for mm in meshes]),
                                    triangles=np.concatenate([mm["triangles"] + v_off[k]
                                                              for k, mm in enumerate(meshes)])), device=dev)
    mbatch = api.Batch(tri_off)
    cams_m = api.cameras_tensor(np.stack([synth.room_camera(e, W, H) for e in range(V)]), dev)
    mout = (torch.empty_like(outs[0]), torch.empty_like(outs[1]))
    mws = torch.empty(int(tri_off[-1]) * 96 + 16, dtype=torch.uint8, device=dev)
    mesh_ms = _event_ms(torch, stream, lambda: api.render_mesh(mesh, mbatch, cams_m, W, H, out=mout, workspace=mws,
                                                               stream=stream))

    def hbm(b, ms):
        a = b / (ms * 1e-3) / 1e9
        return {"ms": ms, "achieved_gbs": a, "frac": a / hbm_peak, "algorithmic_bytes": b}

    return {"lbs_deform": dict(hbm(fwd_bytes, deform_ms), avatars=n_av, gaussians=m),
            "lbs_deform_backward": dict(hbm(bwd_bytes, deform_bwd_ms), avatars=n_av, gaussians=m,
                                        note="joint gradients summed per warp by joint-owner lanes, one atomic per (CTA, joint, entry)"),
            "keyframe_interpolation": {"ms": interp_ms, "avatars": n_av, "frames": n_frames},
            "forward_kinematics": {"ms": fk_ms, "avatars": n_av, "joints": synth.N_JOINTS},
            "avatar_capsules": {"ms": caps_ms, "avatars": n_av, "capsules": n_av * synth.N_JOINTS},
            "capsule_query": {"ms": query_ms, "queries": n_q, "envs": n_qenv,
                              "capsules_per_env": (n_av // n_qenv) * synth.N_JOINTS, "blocked_fraction": q_blocked,
                              "what": "distance to the nearest capsule, blocked flag and first-contact fraction "
                                      "of a 0.1 m sphere per candidate step"},
            "composite": dict(hbm(comp_bytes, comp_ms), views=V, width=W, height=H),
            "mesh_layer": {"ms": mesh_ms, "views": V, "triangles_per_view": int(tri_off[-1]) // V, "width": W,
                           "height": H}}


def _graph_ms(torch, stream, fn, k=20, warm=3):
    """fn captured in a CUDA graph on ``stream``; mean CUDA-event time of k replays."""
    with torch.cuda.stream(stream):
        fn()
    torch.cuda.synchronize()
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gr, stream=stream):
        fn()
    return _event_ms(torch, stream, gr.replay, k)


def single_view_rows(api, synth, torch, dev, stream):
    """The single-view configurations: a 5k-Gaussian box scene at 128x128 and
    a 1M-Gaussian room at 640x480, each forward and forward + backward in a
    CUDA graph (FP32 SH, 16x16 tiles, batch depth 256)."""
    rows = {}
    for name, g, cam, Wc, Hc in (
            ("box_5k_128px", synth.box_scene(5000, seed=0), synth.identity_camera(128, 128), 128, 128),
            ("room_1M_640x480", synth.room_scene(1_000_000, seed=1), synth.room_camera(1, 640, 480), 640, 480)):
        n = g["means"].shape[0]
        G = api.Gaussians.from_numpy(g, device=dev)
        r = api.Renderer(api.Batch(np.array([0, n])), Wc, Hc, device=dev, grad_overwrite=True)
        ct = api.cameras_tensor(cam[None], dev)
        out = r.alloc_outputs()
        grads = dict(means=torch.empty((n, 3), device=dev), log_scales=torch.empty((n, 3), device=dev),
                     quats=torch.empty((n, 4), device=dev), opacity_logits=torch.empty((n,), device=dev),
                     sh=torch.empty((n, 16, 3), device=dev))
        d_rgb = torch.ones((1, 3, Hc, Wc), device=dev)
        d_dep = torch.zeros((1, Hc, Wc), device=dev)
        fwd = _graph_ms(torch, stream, lambda: r.forward(G, ct, out=out, stream=stream))

        def fb():
            r.forward(G, ct, out=out, stream=stream)
            r.backward(G, ct, d_rgb, d_dep, grads=grads, stream=stream)

        fbm = _graph_ms(torch, stream, fb)
        rows[name] = {"gaussians": n, "width": Wc, "height": Hc, "fwd_ms": fwd, "fwd_frames_per_s": 1e3 / fwd,
                      "fwd_bwd_ms": fbm, "fwd_bwd_frames_per_s": 1e3 / fbm}
    return rows


def training_row(api, synth, torch, dev, stream):
    """The training step: one 500k-Gaussian room + 2 avatars of 50k Gaussians
    (24 joints), 16 views at 512x512, L1 loss (RGB and depth, mean) against a
    target rendered from perturbed parameters, gradients of every parameter and
    of the joint transforms (api.AvatarScene: deform, render, loss gradient,
    backward in overwrite mode, deform backward) in one CUDA graph; FP32 and
    FP16 SH storage, and with FP16 SH the fused path (the avatars posed inside
    gs_render_avatars and gs_render_avatars_backward)."""
    wl = synth.training_scene(seed=0)
    T = lambda x, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(x)).to(dev, dt)  # noqa: E731
    room, av = wl["room"], wl["avatars"]
    n_views, Hc, Wc = wl["cams"].shape[0], 512, 512
    cams = api.cameras_tensor(wl["cams"], dev)
    Gj = T(wl["G"])
    kw = dict(tile=(16, 16), batch_depth=128, pix=(2, 1), persistent=True)
    out = {"workload": f"1 room x {room['means'].shape[0]} + {wl['G'].shape[0]} avatars x 50k Gaussians, "
                       f"{n_views} views {Wc}x{Hc}, L1 loss vs perturbed target, fwd+bwd incl. joint gradients",
           "tile": [16, 16], "batch_depth": 128, "pixels_per_thread": [2, 1]}
    for shd, name, fused in ((torch.float32, "f32_sh", False), (torch.float16, "f16_sh", False),
                             (torch.float16, "f16_sh_fused", True)):
        def scene(perturbed):
            rm, rsh, am, ash = room["means"], room["sh"], av["means"], av["sh"]
            if perturbed:
                rm, rsh = rm + wl["d_room_means"], rsh + wl["d_room_sh"]
                am, ash = am + wl["d_av_means"], ash + wl["d_av_sh"]
            sc = dict(means=T(rm), log_scales=T(room["log_scales"]), quats=T(room["quats"]),
                      opacity_logits=T(room["opacity_logits"]), sh=T(rsh))
            avs = dict(means=T(am), log_scales=T(av["log_scales"]), quats=T(av["quats"]),
                       opacity_logits=T(av["opacity_logits"]), sh=T(ash),
                       joint_ids=T(av["joint_ids"].view(np.int16), torch.int16), weights=T(av["weights"]),
                       avatar_of=T(av["avatar_of"], torch.int32))
            return api.AvatarScene(sc, avs, wl["G"].shape[0], synth.N_JOINTS, Wc, Hc, n_views, sh_dtype=shd,
                                   device=dev, fused=fused and not perturbed, **kw)
        tgt = scene(True)
        with torch.cuda.stream(stream):
            t_rgb, t_dep = (x.clone() for x in tgt.forward(Gj, cams, stream=stream)[:2])
        torch.cuda.synchronize()
        del tgt
        sc = scene(False)
        d_rgb, d_dep = torch.empty_like(t_rgb), torch.empty_like(t_dep)
        loss = torch.zeros((), device=dev)

        def step():
            rgb, dep = sc.forward(Gj, cams, stream=stream)[:2]
            torch.sub(rgb, t_rgb, out=d_rgb)
            torch.sub(dep, t_dep, out=d_dep)
            torch.add(d_rgb.abs().mean(), d_dep.abs().mean(), out=loss)
            d_rgb.sign_().mul_(1.0 / d_rgb.numel())
            d_dep.sign_().mul_(1.0 / d_dep.numel())
            sc.backward(Gj, cams, d_rgb, d_dep, stream=stream)

        ms = _graph_ms(torch, stream, step, k=10)
        torch.cuda.synchronize()
        assert sc.renderer.status() == 0
        out[name] = {"ms_per_step": ms, "view_frames_per_s": n_views / (ms * 1e-3), "loss": float(loss)}
        del sc
    return out


def fused_avatar_row(api, synth, torch, dev, stream):
    """Forward of 32 envs, each a 1M-Gaussian room plus 8 avatars of 50k
    Gaussians posed per frame, 256x256: LBS fused into the preprocess
    (gs_render_avatars) against gs_deform_avatars + gs_render."""
    n_envs, n_room, n_av, n_per = 32, 1_000_000, 8, 50_000
    g, offs, cams = synth.batched_rooms(n_envs, n_room, n_room, W, H, seed0=900)
    base = [synth.avatar_canonical(n_per, k) for k in range(n_av)]
    per_env = n_room + n_av * n_per
    keys = ("means", "log_scales", "quats", "opacity_logits", "sh")
    cat = {k: np.concatenate([np.concatenate([g[k][e * n_room:(e + 1) * n_room]] + [base[a][k] for a in range(n_av)])
                              for e in range(n_envs)]) for k in keys}
    del g
    av = {k: np.concatenate([base[a][k] for _ in range(n_envs) for a in range(n_av)]) for k in base[0]}
    m = n_envs * n_av * n_per
    avatar_of = np.repeat(np.arange(n_envs * n_av), n_per).astype(np.int32)
    dest = np.concatenate([e * per_env + n_room + np.arange(n_av * n_per) for e in range(n_envs)]).astype(np.int64)
    Gj = np.stack([synth.random_pose(3 * e + a) for e in range(n_envs) for a in range(n_av)]).astype(np.float32)
    for e in range(n_envs):  # the avatars stand in front of the env's camera
        fwd, C = cams[e][6:9], cams[e][9:12]
        for a in range(n_av):
            k = e * n_av + a
            root = C + fwd * (1.5 + 0.4 * a) + np.array([0.3 * (a % 3 - 1), 0.0, -0.3])
            Gj[k, :, :, 3] += (root - Gj[k, 0, :, 3]).astype(np.float32)
    T = lambda x, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(x)).to(dev, dt)  # noqa: E731
    sh16 = T(cat.pop("sh")).to(torch.float16)
    G = {k: T(v) for k, v in cat.items()}
    del cat
    cov = torch.zeros((n_envs * per_env, 6), device=dev)
    means_posed = G["means"].clone()
    A_unf = api.Avatars(T(av["means"]), T(av["log_scales"]), T(av["quats"]), T(av["joint_ids"].view(np.int16),
                        torch.int16), T(av["weights"]), T(avatar_of, torch.int32), n_envs * n_av, synth.N_JOINTS,
                        dest=T(dest, torch.int64))
    A_fus = api.Avatars(*A_unf.t[:6], n_envs * n_av, synth.N_JOINTS)
    Gjt = T(Gj)
    batch = api.Batch(np.arange(n_envs + 1) * per_env, env_cov3d_begin=np.arange(n_envs) * per_env + n_room)
    g_unf = api.Gaussians(means_posed, G["log_scales"], G["quats"], G["opacity_logits"], sh16, cov3d=cov)
    g_fus = api.Gaussians(G["means"], G["log_scales"], G["quats"], G["opacity_logits"], sh16)
    kw = dict(tile=(8, 8), batch_depth=64, pix=(2, 1), persistent=True)
    r1 = api.Renderer(batch, W, H, device=dev, **kw)
    r2 = api.Renderer(batch, W, H, device=dev, **kw)
    ct = api.cameras_tensor(cams, dev)
    o1, o2 = r1.alloc_outputs(), r2.alloc_outputs()

    def unfused():
        api.deform(A_unf, Gjt, means_posed, cov, stream=stream)
        r1.forward(g_unf, ct, out=o1, stream=stream)

    def fused():
        r2.forward_avatars(g_fus, A_fus, Gjt, ct, out=o2, stream=stream)

    ms_unf = _event_ms(torch, stream, unfused, 5)
    ms_fus = _event_ms(torch, stream, fused, 5)
    torch.cuda.synchronize()
    same = all(bool(torch.equal(x, y)) for x, y in zip(o1, o2))
    return {"workload": f"{n_envs} envs x (1M room + {n_av} avatars x 50k), {W}x{H}, forward", "gaussians": n_envs * per_env,
            "avatar_gaussians": m, "unfused_ms": ms_unf, "fused_ms": ms_fus,
            "unfused_env_frames_per_s": n_envs / (ms_unf * 1e-3), "fused_env_frames_per_s": n_envs / (ms_fus * 1e-3),
            "bit_identical": same}


def run_ours(args, ws, rank, local):
    import torch

    from paper_2604_12626_gb300 import api, shard, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n_envs = args.envs
    seed0 = shard.env_block(rank, n_envs).start  # weak scaling: every rank renders its own envs
    t0 = time.time()
    g, offs, cams = synth.batched_rooms(n_envs, N_MIN, N_MAX, W, H, seed0=seed0, scale=args.scale)
    t_gen = time.time() - t0
    N = int(offs[-1])
    T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)  # noqa: E731
    means, ls, quats, ologit = T(g["means"]), T(g["log_scales"]), T(g["quats"]), T(g["opacity_logits"])
    sh32 = T(g["sh"])
    sh16 = sh32.to(torch.float16)
    del g
    cams_d = api.cameras_tensor(cams, dev)
    batch = api.Batch(offs)
    G16 = api.Gaussians(means, ls, quats, ologit, sh16)
    G32 = api.Gaussians(means, ls, quats, ologit, sh32)

    # --- autotune the batched renderer (tile, batch depth), cached per GPU + workload
    fixed = [int(x) for x in args.tile.split(",")] + [1, 1] if args.tile else None
    cands = [fixed[:5]] if fixed else TILE_CANDIDATES
    rend = api.Renderer(batch, W, H, device=dev, tile=(8, 8), batch_depth=64, persistent=True, grad_overwrite=True,
                        tile_candidates=cands)
    cache_path = os.path.join(ROOT, "paper_2604_12626_gb300", "_build", "autotune.json")
    key = f"{torch.cuda.get_device_name(dev)}|{n_envs}x{W}x{H}|N={N}|f16|fwd+bwd"
    cache = {}
    try:
        with open(cache_path) as f:
            cache = json.load(f)
    except Exception:
        pass
    if fixed:
        rend.cfg.tile_w, rend.cfg.tile_h, rend.cfg.batch_depth, rend.cfg.pix_x, rend.cfg.pix_y = fixed[:5]
        tuned = {"choice": fixed[:5], "fixed": True}
    elif key in cache and not args.retune:
        ch = cache[key]["choice"]
        rend.cfg.tile_w, rend.cfg.tile_h, rend.cfg.batch_depth, rend.cfg.pix_x, rend.cfg.pix_y = ch
        tuned = dict(cache[key], cached=True)
    else:
        choice, best_ms = tune_fwd_bwd(api, rend, G16, cams_d, TILE_CANDIDATES, N, dev)
        tuned = {"choice": list(choice), "ms": best_ms, "cached": False}
        cache[key] = tuned
        try:
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except Exception:
            pass
    outs = rend.alloc_outputs()
    grads = dict(means=torch.empty((N, 3), device=dev), log_scales=torch.empty((N, 3), device=dev),
                 quats=torch.empty((N, 4), device=dev), opacity_logits=torch.empty((N,), device=dev),
                 sh=torch.empty((N, 16, 3), device=dev))
    rng = torch.Generator(device=dev)
    rng.manual_seed(1234 + rank)
    d_rgb = torch.randn((n_envs, 3, H, W), device=dev, generator=rng)
    d_depth = 0.1 * torch.randn((n_envs, H, W), device=dev, generator=rng)

    stream = torch.cuda.Stream(device=dev)

    def step_fwd():
        rend.forward(G16, cams_d, out=outs, stream=stream)

    def step_fb():
        rend.forward(G16, cams_d, out=outs, stream=stream)
        rend.backward(G16, cams_d, d_rgb, d_depth, grads=grads, stream=stream)

    with torch.cuda.stream(stream):
        step_fb()
    torch.cuda.synchronize()
    assert rend.status() == 0, "pair capacity exceeded"
    stats = rend.stats(stream)

    def capture(fn):
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr, stream=stream):
            fn()
        return gr

    g_fb = capture(step_fb)
    g_fwd = capture(step_fwd)

    def timed(replay, k, warm, sample_clocks=False):
        with torch.cuda.stream(stream):
            for _ in range(warm):
                replay()
        torch.cuda.synchronize()
        barrier(ws)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(smi_index(local)) if sample_clocks else None
        if sampler:
            sampler.__enter__()
            time.sleep(0.3)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(k):
                replay()
            e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        if sampler:
            sampler.__exit__(None, None, None)
        barrier(ws)
        ms = e0.elapsed_time(e1) / k
        return max_over_ranks(ms, ws), (sampler.summary() if sampler else None)

    ms_fb, clocks = timed(g_fb.replay, args.steps, args.warmup, sample_clocks=True)
    ms_fwd, _ = timed(g_fwd.replay, args.steps, args.warmup)
    assert rend.status(stream) == 0

    # --- the same step with the gradient clearing on a second stream beside the
    # forward (gs_zero_gradients, joined by an event; the backward pre-cleared)
    side = torch.cuda.Stream(device=dev)
    overlap = {}
    for n_ctas in (76,):
        def step_ov(n_ctas=n_ctas):
            e0 = torch.cuda.Event()
            e0.record(stream)
            side.wait_event(e0)
            api.zero_gradients(grads, n_ctas=n_ctas, stream=side)
            e1 = torch.cuda.Event()
            e1.record(side)
            rend.forward(G16, cams_d, out=outs, stream=stream)
            stream.wait_event(e1)
            rend.backward(G16, cams_d, d_rgb, d_depth, grads=grads, stream=stream, precleared=True)
        with torch.cuda.stream(stream):
            step_ov()
        torch.cuda.synchronize()
        g_ov = capture(step_ov)
        ms_ov, _ = timed(g_ov.replay, args.steps, args.warmup)
        overlap[str(n_ctas)] = {"ms_per_step": ms_ov, "value": shard.job_throughput(n_envs, ws, ms_ov)}
        del g_ov
    assert rend.status(stream) == 0

    # --- plain per-env path: one gs_render (+ gs_render_backward) per env, FP32
    # SH, 16x16 tiles, B=256, no graph; gradients of each env written in place
    plain_ms = plain_fb_ms = None
    if not args.no_plain:
        envs = []
        for e in range(n_envs):
            a, b = int(offs[e]), int(offs[e + 1])
            ge = api.Gaussians(means[a:b], ls[a:b], quats[a:b], ologit[a:b], sh32[a:b])
            envs.append(ge)
        sizes = np.diff(offs)
        big = int(np.argmax(sizes))
        r1 = api.Renderer(api.Batch(np.array([0, sizes[big]])), W, H, device=dev, grad_overwrite=True)
        outs1 = r1.alloc_outputs()
        cam_e = [cams_d[e:e + 1] for e in range(n_envs)]
        batches = [api.Batch(np.array([0, sizes[e]])) for e in range(n_envs)]
        nb = int(sizes[big])  # one set of gradient buffers, reused by every env (like the outputs)
        grads1 = dict(means=torch.empty((nb, 3), device=dev), log_scales=torch.empty((nb, 3), device=dev),
                      quats=torch.empty((nb, 4), device=dev), opacity_logits=torch.empty((nb,), device=dev),
                      sh=torch.empty((nb, 16, 3), device=dev))
        env_grads = [{k: v[:int(sizes[e])] for k, v in grads1.items()} for e in range(n_envs)]

        def plain_step():
            for e in range(n_envs):
                r1.batch = batches[e]
                r1.forward(envs[e], cam_e[e], out=outs1, stream=stream)

        def plain_fb_step():
            for e in range(n_envs):
                r1.batch = batches[e]
                r1.forward(envs[e], cam_e[e], out=outs1, stream=stream)
                r1.backward(envs[e], cam_e[e], d_rgb[e:e + 1], d_depth[e:e + 1], grads=env_grads[e],
                            stream=stream)

        plain_ms, _ = timed(plain_step, max(2, args.steps // 2), 1)
        plain_fb_ms, _ = timed(plain_fb_step, max(2, args.steps // 2), 1)
        del r1, outs1, envs, grads1, env_grads

    # --- the batched path with FP32 SH storage (same graph, same tile)
    def step_fwd32():
        rend.forward(G32, cams_d, out=outs, stream=stream)

    def step_fb32():
        rend.forward(G32, cams_d, out=outs, stream=stream)
        rend.backward(G32, cams_d, d_rgb, d_depth, grads=grads, stream=stream)

    g32_fb, g32_fwd = capture(step_fb32), capture(step_fwd32)
    ms32_fb, _ = timed(g32_fb.replay, args.steps, args.warmup)
    ms32_fwd, _ = timed(g32_fwd.replay, args.steps, args.warmup)
    del g32_fb, g32_fwd

    # --- live per-stage timing (same workload, launched without the graph)
    api.profile_enable(True)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            step_fb()
    torch.cuda.synchronize()
    prof = api.profile_read()
    api.profile_enable(False)
    stage_ms = {k: v[0] / max(v[1], 1) for k, v in prof.items()}

    # --- end to end through the public API with host buffers
    cams_host = torch.from_numpy(np.ascontiguousarray(cams, np.float32)).pin_memory()
    rgb_host = torch.empty((n_envs, 3, H, W), dtype=torch.float32).pin_memory()
    depth_host = torch.empty((n_envs, H, W), dtype=torch.float32).pin_memory()
    cams_dev2 = torch.empty_like(cams_d)

    def e2e_step():
        cams_dev2.copy_(cams_host.view(-1, 16), non_blocking=True)
        rend.forward(G16, cams_dev2, out=outs, stream=stream)
        rend.backward(G16, cams_dev2, d_rgb, d_depth, grads=grads, stream=stream)
        rgb_host.copy_(outs[0], non_blocking=True)
        depth_host.copy_(outs[1], non_blocking=True)

    with torch.cuda.stream(stream):
        e2e_ms, _ = timed(e2e_step, args.steps, 1)
    h2d = cams_host.numel() * 4
    d2h = (rgb_host.numel() + depth_host.numel()) * 4

    # --- exact work counts for the blend rooflines (outside the timed region)
    # (the counting forward lists every Gaussian by its square footprint, so
    # the counts follow the definition whatever tiles the fast path skips)
    with torch.cuda.stream(stream):
        n_eval_fwd = rend.count_evaluations(G16, cams_d, out=outs, stream=stream)
        n_eval_bwd = rend.stats(stream)["n_covered"]  # what the adjoint walks by the definition
    torch.cuda.synchronize()
    n_blended = int(outs[3].sum().item())  # sum of n_contrib: Gaussians blended into the pixels
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    e_rate = exp2_rate(api, torch, dev, stream, sm_count)
    roof, per_kernel = rooflines(stats, stage_ms, n_eval_fwd, n_eval_bwd, n_envs * W * H, N, sm_count,
                                 (clocks or {}).get("sm_max_mhz"), exp_rate=e_rate)

    # --- the avatar rows (LBS, its adjoint, keyframes + FK) and the composite,
    # timed on their own: 32 envs x 8 avatars x 50k Gaussians, and the
    # nearest-fragment merge of the bench frames with a second layer
    extra = avatar_and_composite_rows(api, synth, torch, dev, stream, outs, hbm_peak=peaks()[0])
    if not args.no_avatar_scene:
        extra["scene_with_avatars"] = fused_avatar_row(api, synth, torch, dev, stream)
    if not args.no_configs:
        extra["single_view"] = single_view_rows(api, synth, torch, dev, stream)
        extra["training_16x512px"] = training_row(api, synth, torch, dev, stream)

    # --- CPU oracle on a bounded sample (rank 0, N = 1)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        n, t = oracle_step(list(range(n_envs)), seed0, budget_s=args.cpu_budget, scale=args.scale)
        cpu = {"value": n / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n} env(s) of this batch (env 0..{n - 1}), FP64 forward (OpenMP, all cores) + "
                         f"backward (1 thread), {t:.1f} s"}
        if not args.no_configs:
            cpu["configs"] = oracle_configs(seed0)

    total_envs = n_envs * ws
    line = {
        "metric": METRIC, "value": shard.job_throughput(n_envs, ws, ms_fb), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_fb, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{n_envs} envs x synthetic room (U[300k,1.5M] Gaussians, uneven), {W}x{H} RGB-D, "
                               "forward+backward, SH stored fp16, persistent blend in one CUDA graph, "
                               "autotuned tile", "n_envs_per_gpu": n_envs, "gaussians_per_gpu": N,
                   "width": W, "height": H, "tile": [rend.cfg.tile_w, rend.cfg.tile_h],
                   "batch_depth": rend.cfg.batch_depth, "pixels_per_thread": [rend.cfg.pix_x, rend.cfg.pix_y],
                   "sh_storage": "f16", "autotune": tuned,
                   "l2_policy": "inputs larger than L2 (no flush)", "parallelism": f"env-sharded x{ws}"},
        "fwd": {"value": total_envs / (ms_fwd * 1e-3), "ms_per_step": ms_fwd},
        "plain_per_env": (None if plain_ms is None else
                          {"fwd": {"value": total_envs / (plain_ms * 1e-3), "ms_per_step": plain_ms},
                           "fwd_bwd": {"value": total_envs / (plain_fb_ms * 1e-3), "ms_per_step": plain_fb_ms},
                           "what": "64 single-env gs_render (+ gs_render_backward) calls, FP32 SH, 16x16 tiles, "
                                   "B=256, no graph",
                           "batched_fwd_speedup": plain_ms / ms_fwd, "batched_fwd_bwd_speedup": plain_fb_ms / ms_fb,
                           "batched_f32_fwd_speedup": plain_ms / ms32_fwd,
                           "batched_f32_fwd_bwd_speedup": plain_fb_ms / ms32_fb}),
        "clear_beside_forward": {"by_clearing_ctas": overlap,
                                 "what": "the headline step with gs_zero_gradients on a second stream beside the "
                                         "forward and the backward pre-cleared (slower: the clearing CTAs "
                                         "take SMs and HBM from the forward; 16 / 38 CTAs measured 19.7 / "
                                         "13.4 ms)"},
        "batched_f32_sh": {"fwd": {"value": total_envs / (ms32_fwd * 1e-3), "ms_per_step": ms32_fwd},
                           "fwd_bwd": {"value": total_envs / (ms32_fb * 1e-3), "ms_per_step": ms32_fb},
                           "what": "the headline step with SH stored FP32 (same graph, tile and launch shape)"},
        "roofline": roof,
        "roofline_per_kernel": per_kernel,
        "other_rows": extra,
        "cpu_baseline": cpu,
        "e2e": {"value": total_envs / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "what": "public API calls per step: cameras H2D from pinned memory, "
                                                   "gs_render + gs_render_backward, RGB + depth D2H"},
        # + clear_record_grads, blend_backward, preprocess_backward
        "exp2_rate": {"gops": e_rate / 1e9,
                      "per_sm_per_clk": e_rate / (sm_count * ((clocks or {}).get("sm_max_mhz") or 2070.0) * 1e6)},
        "gpu_launches": (rend.kernels_per_forward() + 3) * args.steps,
        "clocks": clocks,
        "stage_ms": stage_ms,
        "stats": {"records": stats["n_records"], "visible": stats["n_visible"],
                  "f_v": stats["n_visible"] / max(stats["n_records"], 1), "pairs": stats["n_pairs"],
                  "pairs_per_visible": stats["n_pairs"] / max(stats["n_visible"], 1), "max_bin": stats["max_bin"],
                  "evaluations_fwd": n_eval_fwd, "evaluations_bwd": n_eval_bwd, "blended": n_blended, "gen_s": t_gen},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="scale the per-env Gaussian counts (testing only)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-avatar-scene", action="store_true", help="skip the 32-env rooms-with-avatars forward")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the single-view and training-step rows (and their oracle timings)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--retune", action="store_true")
    ap.add_argument("--tile", default="", help="fixed tile_w,tile_h,batch_depth instead of the autotuner")
    ap.add_argument("--envs", type=int, default=N_ENVS, help="envs per GPU (64; fewer only for small profiling cases)")
    ap.add_argument("--ncu-summary", metavar="CSV",
                    help="print the per-kernel table of an ncu --csv launch list of this bench and exit")
    ap.add_argument("--ncu-table", nargs="+", metavar="RAW_CSV",
                    help="print the full-capture table of the kernel summary from raw-page CSVs and exit")
    ap.add_argument("--ncu-traffic", nargs="+", metavar="ARG",
                    help="LAUNCH_CSV STATS_JSON COMMAND RAW_CSV...: write profiles/dram_traffic.json from a "
                         "complete time-only launch list of the same launch shape (launches per call), the JSON "
                         "line of COMMAND and the raw-page CSVs of one-kernel captures of COMMAND, and exit")
    args = ap.parse_args()
    if args.ncu_summary:
        ncu_summary(args.ncu_summary)
        return
    if args.ncu_table:
        ncu_table(args.ncu_table)
        return
    if args.ncu_traffic:
        if len(args.ncu_traffic) < 4:
            ap.error("--ncu-traffic takes LAUNCH_CSV STATS_JSON COMMAND RAW_CSV...")
        launch_csv, stats_json, command = args.ncu_traffic[:3]
        ncu_traffic(launch_csv, args.ncu_traffic[3:], command, stats_json=stats_json)
        return
    if args.warmup < 3:
        args.warmup = 3
    from paper_2604_12626_gb300 import shard

    try:
        plan = shard.launch_plan(args.gpus)
    except ValueError as e:
        print(f"bench.py: {e}", file=sys.stderr)
        sys.exit(2)
    if plan == "spawn":  # started without a launcher: start the N ranks here
        sys.exit(subprocess.call(shard.spawn_command(args.gpus, os.path.abspath(__file__), sys.argv[1:])))
    ws, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
