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
