"""Replica plumbing for running the path on N GPUs of one node.

The tracking frames and batched mapping steps are independent problems, so
N GPUs run N replicas with no collective on the data path (weak scaling):
each rank takes its own seeded inputs, the timed region is bracketed by
barriers, and the job's time is the maximum over ranks.  Launched one
process per GPU (torch.distributed.run sets RANK / LOCAL_RANK /
WORLD_SIZE / MASTER_*); NCCL between GPUs, gloo for CPU tests.
"""
from __future__ import annotations

import os

import torch


def env():
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str = "nccl"):
    """Joins the process group when more than one rank runs; returns env()."""
    ws, rank, local = env()
    if ws > 1 and not torch.distributed.is_initialized():
        if backend == "nccl":
            torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            torch.distributed.init_process_group(backend)
    return ws, rank, local


def barrier():
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.barrier()


def max_over_ranks(x: float, device="cpu") -> float:
    """The maximum of a per-rank scalar (a timing) over all ranks."""
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def seed_base(rank: int) -> int:
    """Seed offset of a rank's inputs: ranks draw disjoint frames."""
    return 1000 * int(rank)


def weak_scaling_value(world_size: int, units_per_rank: float, max_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (units per second)."""
    return world_size * units_per_rank / (max_ms / 1e3)


def finish():
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.destroy_process_group()
