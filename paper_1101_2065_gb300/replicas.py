"""Replica bookkeeping for multi-GPU runs.

Molecules are independent GW problems, so N GPUs run N replicas with no
data-path collective.  The only cross-rank operations are a barrier before
and after the timed region and the maximum of the per-rank elapsed times;
the aggregate throughput is the units all ranks processed divided by that
maximum (weak scaling: fixed work per GPU).
"""
import os


def world():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class Replicas:
    def __init__(self, backend="nccl"):
        self.rank, self.size, self.local = world()
        self.dist = None
        self.device = "cpu"
        if self.size > 1:
            import torch.distributed as dist
            if not dist.is_initialized():
                dist.init_process_group(backend)
            self.dist = dist
            if backend == "nccl":
                self.device = "cuda"

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x):
        """Maximum of a float over ranks."""
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def throughput(self, units_per_rank, elapsed_ms):
        """Whole-job units per second: all ranks' units over the slowest rank's time."""
        return self.size * units_per_rank / (self.max(elapsed_ms) / 1e3)

    def close(self):
        if self.dist is not None and self.dist.is_initialized():
            self.dist.destroy_process_group()
