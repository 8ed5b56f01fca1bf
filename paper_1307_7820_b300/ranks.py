"""Host logic for several GPUs of one node, one process per GPU.

A single fold does not shard (every tile diagonal needs whole row and column
strips of the table), so `bench.py --gpus N` runs one replica per rank for the
headline fold.  A batch's sequences are independent problems: they are split
across ranks by `partition_lpt` (longest processing time first, work ~ n^3 as
in Eq. 1's cubic recurrence), and each rank folds its share with no collective
on the data path.  `Ranks` wraps the barrier and the max-over-ranks used to
time a step across ranks.
"""
from __future__ import annotations

import heapq
import os


def fold_work(n: int) -> int:
    """Relative cost of folding a sequence of length n (cells times splits, ~n^3 / 6)."""
    return n * (n - 1) * (n + 1) // 6 if n > 1 else 1


def partition_lpt(lengths, world: int) -> list[list[int]]:
    """Indices of `lengths` split into `world` lists of about equal work: the longest sequence
    goes to the rank with the least work so far (ties: the lower rank).  Deterministic, so every
    rank computes the same partition without communicating."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(lengths)), key=lambda k: (-fold_work(int(lengths[k])), k))
    heap = [(0, r) for r in range(world)]
    parts: list[list[int]] = [[] for _ in range(world)]
    for k in order:
        w, r = heapq.heappop(heap)
        parts[r].append(k)
        heapq.heappush(heap, (w + fold_work(int(lengths[k])), r))
    for p in parts:
        p.sort()
    return parts


class Ranks:
    """Rank, world size, barrier and max over ranks (torch.distributed when WORLD_SIZE > 1)."""

    def __init__(self, backend: str = "nccl", device=None):
        import torch

        self.torch = torch
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.device = device
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist

            if not dist.is_initialized():
                dist.init_process_group(backend)
            self.dist = dist

    def barrier(self) -> None:
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x: float) -> float:
        if self.dist is None:
            return x
        t = self.torch.tensor([x], dtype=self.torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self) -> None:
        if self.dist is not None and self.dist.is_initialized():
            self.dist.destroy_process_group()
