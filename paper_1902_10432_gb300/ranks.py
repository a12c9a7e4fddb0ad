"""Host-side logic of runs on several GPUs of one node (one process per GPU, torchrun environment).

The method itself has no exchange step between independent problems: several GPUs run replicas of
one lattice, or disjoint shares of a batch of independent instances, and meet only to time the run
(barrier on both sides, maximum of the per-rank times) and to add up the work done. Nothing here
touches the data path.
"""
from __future__ import annotations

import os


def shard(n: int, rank: int, world: int) -> list:
    """Indices of the n independent instances that rank `rank` of `world` runs (round robin, so the
    shares differ in size by at most one and every index is run exactly once)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d out of range for world %d" % (rank, world))
    return list(range(rank, n, world))


class Ranks:
    """The torchrun environment and the two reductions the timing needs. With one process there is
    no process group and every call is local."""

    def __init__(self, backend: str = "nccl"):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.backend = backend
        self._dist = None
        if self.world > 1:
            import torch.distributed as dist

            if not dist.is_initialized():
                dist.init_process_group(backend)
            self._dist = dist

    @property
    def root(self) -> bool:
        return self.rank == 0

    def barrier(self):
        if self._dist is not None:
            self._dist.barrier()

    def _reduce(self, value: float, op) -> float:
        if self._dist is None:
            return float(value)
        import torch

        dev = "cuda" if self.backend == "nccl" else "cpu"
        t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
        self._dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, value: float) -> float:
        return self._reduce(value, None if self._dist is None else self._dist.ReduceOp.MAX)

    def sum(self, value: float) -> float:
        return self._reduce(value, None if self._dist is None else self._dist.ReduceOp.SUM)

    def close(self):
        if self._dist is not None and self._dist.is_initialized():
            self._dist.destroy_process_group()
            self._dist = None
