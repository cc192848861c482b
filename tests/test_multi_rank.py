"""The multi-GPU path on CPU: two gloo ranks, each rendering its own block of
envs (weak scaling, no collective on the data path), a barrier around the timed
region and the maximum of the per-rank times -- the host logic bench.py runs
under torchrun, with the FP64 oracle standing in for the GPU renderer."""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

from paper_2604_12626_gb300 import shard, synth  # noqa: E402

ENVS_PER_RANK, W, H = 2, 24, 24


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _render_env(e):
    import oracle

    n = synth.batch_sizes(e + 1, 300, 600, 0)[e]
    g = synth.room_scene(n, seed=e)
    cam = synth.room_camera(e, W, H)
    return oracle.render(g, cam, W, H, nthreads=1)["rgb"]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    got_ws, got_rank, _ = shard.init("gloo")
    envs = list(shard.env_block(got_rank, ENVS_PER_RANK))
    shard.barrier(got_ws)
    sums = [float(_render_env(e).sum()) for e in envs]
    t_ms = 10.0 + 5.0 * got_rank  # stand-in per-rank step time
    shard.barrier(got_ws)
    t_max = shard.max_over_ranks(t_ms, got_ws)
    value = shard.job_throughput(ENVS_PER_RANK, got_ws, t_max)
    with open(os.path.join(out_dir, f"rank{got_rank}.json"), "w") as f:
        json.dump(dict(ws=got_ws, rank=got_rank, envs=envs, sums=sums, t_max=t_max, value=value), f)
    dist.destroy_process_group()


def test_two_gloo_ranks_render_disjoint_env_blocks(tmp_path, oracle):
    ws = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, str(tmp_path))) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(ws)]
    assert [r["rank"] for r in res] == [0, 1] and all(r["ws"] == ws for r in res)
    # the blocks partition envs 0..3 and every rank renders exactly its own envs
    assert res[0]["envs"] == [0, 1] and res[1]["envs"] == [2, 3]
    for r in res:
        for e, s in zip(r["envs"], r["sums"]):
            assert s == float(_render_env(e).sum())
    # max over ranks, and the job value counts every rank's envs
    assert all(r["t_max"] == 15.0 for r in res)
    assert all(r["value"] == pytest.approx(ENVS_PER_RANK * ws / 15e-3) for r in res)


def test_shard_helpers_single_process():
    assert list(shard.env_block(3, 4)) == [12, 13, 14, 15]
    parts = [shard.split_envs(10, 4, r) for r in range(4)]
    assert [len(p) for p in parts] == [3, 3, 2, 2]
    assert sorted(i for p in parts for i in p) == list(range(10))
    assert shard.max_over_ranks(7.5, 1) == 7.5
    assert shard.job_throughput(64, 1, 20.0) == pytest.approx(3200.0)
    # env e's scene depends only on its seed, not on which rank draws it
    a = synth.batch_sizes(6, 100, 1000, 0)
    b = synth.batch_sizes(2, 100, 1000, 4)
    assert a[4:] == b
    assert np.array_equal(synth.room_scene(500, seed=5)["means"], synth.room_scene(500, seed=5)["means"])


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_launch_plan():
    assert shard.launch_plan(1, {}) == "run"
    assert shard.launch_plan(2, {}) == "spawn"
    assert shard.launch_plan(4, {"WORLD_SIZE": "4"}) == "run"
    with pytest.raises(ValueError, match="WORLD_SIZE=2"):
        shard.launch_plan(8, {"WORLD_SIZE": "2"})
    with pytest.raises(ValueError):
        shard.launch_plan(0, {})
    cmd = shard.spawn_command(2, "bench.py", ["--gpus", "2"])
    assert cmd[1:3] == ["-m", "torch.distributed.run"] and "--nproc-per-node=2" in cmd
    assert cmd[-3:] == ["bench.py", "--gpus", "2"] and "127.0.0.1" in cmd


def _bench(args, extra_env=None):
    import subprocess
    import sys

    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", PYTHONPATH=ROOT)
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(k, None)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_bench_gpus_2_starts_two_ranks_itself(oracle):
    """bench.py --gpus 2 run without a launcher starts its two ranks (gloo here,
    with no GPU); the reference arm runs on rank 0 alone and reports n_gpus 2."""
    r = _bench(["--gpus", "2", "--impl", "reference", "--steps", "1", "--warmup", "3", "--scale", "0.002"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout  # rank 0 alone prints
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0


def test_bench_refuses_a_launcher_with_another_world_size():
    r = _bench(["--gpus", "4", "--impl", "reference", "--steps", "1"],
               {"WORLD_SIZE": "2", "RANK": "0", "LOCAL_RANK": "0"})
    assert r.returncode == 2
    assert "WORLD_SIZE=2" in r.stderr
