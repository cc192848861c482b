"""Environment sharding across GPUs (one process per GPU).

Rendering is independent per environment (each agent's observation comes from
its own scene, Sec. 3.2), so a multi-GPU job splits the envs across ranks and
needs no collective on the data path: rank r renders its own block of envs.
The only communication is host-side bookkeeping -- a barrier around the timed
region and the maximum of the per-rank times -- done with torch.distributed
on whatever backend the process group uses (NCCL between GPUs, gloo on CPU).
"""
from __future__ import annotations

import os
import socket
import sys


def world() -> tuple[int, int, int]:
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str) -> tuple[int, int, int]:
    """Joins the process group when world_size > 1 (rendezvous from MASTER_ADDR /
    MASTER_PORT); returns (world_size, rank, local_rank)."""
    ws, rank, local = world()
    if ws > 1:
        import torch.distributed as dist

        if not dist.is_initialized():
            dist.init_process_group(backend, rank=rank, world_size=ws)
    return ws, rank, local


def launch_plan(n_gpus: int, environ=None) -> str:
    """How a run asked for n_gpus ranks proceeds: "run" when this process is
    already one of n_gpus ranks (or n_gpus is 1 and no launcher is involved),
    "spawn" when it was started without a launcher for n_gpus > 1 (it then
    starts the n_gpus ranks itself).  A launcher whose WORLD_SIZE differs from
    n_gpus is an error (ValueError), so that a multi-GPU run can never
    silently measure another number of GPUs."""
    env = os.environ if environ is None else environ
    if n_gpus < 1:
        raise ValueError(f"--gpus must be >= 1, got {n_gpus}")
    ws = env.get("WORLD_SIZE")
    if ws is None:
        return "run" if n_gpus == 1 else "spawn"
    if int(ws) != n_gpus:
        raise ValueError(f"--gpus {n_gpus} but the launcher started WORLD_SIZE={ws} ranks")
    return "run"


def spawn_command(n_gpus: int, script: str, argv: list) -> list:
    """The torch.distributed.run command that starts n_gpus ranks of script
    (one per GPU, rendezvous on 127.0.0.1 at a free port)."""
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n_gpus}",
            "--master-addr", "127.0.0.1", "--master-port", str(port), script, *argv]


def env_block(rank: int, envs_per_rank: int) -> range:
    """Global env ids of a rank (weak scaling: every rank renders its own
    envs_per_rank envs; env e is generated from seed e)."""
    return range(rank * envs_per_rank, (rank + 1) * envs_per_rank)


def split_envs(n_envs: int, world_size: int, rank: int) -> range:
    """Contiguous, balanced split of n_envs envs (strong scaling)."""
    base, extra = divmod(n_envs, world_size)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def barrier(ws: int) -> None:
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    """The maximum of x over all ranks (the job's time is its slowest rank's)."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist

    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(envs_per_rank: int, ws: int, ms_max: float) -> float:
    """Env-frames per second of the whole job: all ranks' envs over the slowest
    rank's time per step."""
    return envs_per_rank * ws / (ms_max * 1e-3)
