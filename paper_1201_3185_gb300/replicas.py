"""Replica coordination for runs on several GPUs (one process per GPU).

The QUMOND path does not shard: a galaxy's boxes are solved in sequence and
each solve needs the whole grid.  Several GPUs therefore run independent
replicas (independent galaxies or parameter sets); the only collective
traffic is a barrier around timed regions and one reduction of the elapsed
times, never the data path.  Works with the NCCL backend on GPUs and with
gloo on the CPU (used by the tests).
"""
from __future__ import annotations

import os
from dataclasses import dataclass

import torch
import torch.distributed as dist


@dataclass
class Replicas:
    world_size: int
    rank: int
    local_rank: int
    device: torch.device

    @classmethod
    def from_env(cls, backend: str | None = None) -> "Replicas":
        """Reads RANK / LOCAL_RANK / WORLD_SIZE (torchrun) and joins the group
        when there is more than one rank.  backend: nccl on CUDA, else gloo."""
        ws = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        local = int(os.environ.get("LOCAL_RANK", "0"))
        use_cuda = torch.cuda.is_available() and backend != "gloo"
        dev = torch.device("cuda", local) if use_cuda else torch.device("cpu")
        if use_cuda:
            torch.cuda.set_device(dev)
        if ws > 1 and not dist.is_initialized():
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend or ("nccl" if use_cuda else "gloo"))
        return cls(ws, rank, local, dev)

    def barrier(self):
        """All ranks reach this point; on CUDA the device is also idle."""
        if self.world_size > 1:
            dist.barrier()
        if self.device.type == "cuda":
            torch.cuda.synchronize(self.device)

    def max(self, value: float) -> float:
        """Maximum of a per-rank value over all ranks (e.g. elapsed times)."""
        if self.world_size == 1:
            return float(value)
        t = torch.tensor([float(value)], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def total(self, value: float) -> float:
        """Sum of a per-rank value over all ranks (e.g. units processed)."""
        if self.world_size == 1:
            return float(value)
        t = torch.tensor([float(value)], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    def replica_seed(self, base_seed: int) -> int:
        """Seed of this rank's replica: different galaxies on different ranks."""
        return base_seed + 7919 * self.rank

    def close(self):
        if self.world_size > 1 and dist.is_initialized():
            dist.destroy_process_group()
