"""Host-side helpers for running independent scene replicas on several GPUs.

A single MLS-MPM scene does not shard without a halo exchange, so N GPUs run
N independent replicas (weak scaling) and no collective touches the data
path.  The only cross-rank operations are a barrier around the timed region
and the max-reduction of the per-rank times.
"""
from __future__ import annotations

import os


def env():
    """(world, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


class Ranks:
    """Barrier and max-over-ranks for the benchmark; a no-op for one rank."""

    def __init__(self, backend=None, device=None):
        self.world, self.rank, self.local = env()
        self.device = device
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            if backend is None:
                backend = "nccl" if torch.cuda.is_available() else "gloo"
            kw = {}
            if backend == "nccl" and device is not None:
                kw["device_id"] = torch.device("cuda", device)
            dist.init_process_group(backend, **kw)
            self.backend = backend
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, value: float) -> float:
        if not self.pg:
            return float(value)
        import torch
        dev = "cuda" if self.backend == "nccl" else "cpu"
        t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()
            self.pg = None


def replica_seed(rank: int) -> int:
    """Seed of the scene a rank simulates: every replica is a distinct scene."""
    return int(rank)
