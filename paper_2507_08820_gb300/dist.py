"""Process-group plumbing for running independent replicas, one process per GPU.

The Reg-FLBM step has no exchange between independent boxes, so a multi-GPU run is N
replicas (weak scaling): rank r advances its own box with Philox replica word r, and the
only collectives are a barrier around the timed region and a max-reduction of the
per-rank times. torch.distributed is used for exactly that (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass
class RankInfo:
    rank: int
    world: int
    local_rank: int


def rank_info() -> RankInfo:
    """RANK / WORLD_SIZE / LOCAL_RANK from the environment (torchrun), else 0 / 1 / 0."""
    return RankInfo(int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
                    int(os.environ.get("LOCAL_RANK", "0")))


def init(info: RankInfo, backend: str):
    """Initialises the default process group when world > 1 (env:// rendezvous)."""
    if info.world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=info.rank, world_size=info.world)
    return dist


def barrier(info: RankInfo, device=None):
    if info.world <= 1:
        return
    import torch.distributed as dist
    if device is not None and dist.get_backend() == "nccl":
        dist.barrier(device_ids=[device])
    else:
        dist.barrier()


def max_over_ranks(info: RankInfo, value: float, device=None) -> float:
    """Maximum of a float over all ranks (the slowest rank's time)."""
    if info.world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(info: RankInfo, value: float, device=None) -> float:
    if info.world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def finalize(info: RankInfo):
    if info.world <= 1:
        return
    import torch.distributed as dist
    if dist.is_initialized():
        dist.destroy_process_group()
