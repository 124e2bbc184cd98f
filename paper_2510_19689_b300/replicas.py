"""Row-sharded replicas: one process per GPU, no collective on the data path.

TabNet inference with running-statistics batch norm treats every row on its
own, so a batch splits into contiguous row ranges, one per rank, and each
rank runs its own model replica (its own `tabnet_create`) on its own GPU and
writes its own output slice.  The only collectives are in the measurement:
a barrier on each side of the timed region and the maximum of the ranks'
elapsed times.  Ranks are started one per GPU by torch.distributed.run,
which sets RANK, LOCAL_RANK, WORLD_SIZE and the rendezvous address.
"""
import os
from typing import Optional, Tuple


def shard(total_rows: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous row range [start, start + count) of `rank` out of `world`.

    Every row lands in exactly one range; the first total_rows % world
    ranks take one row more than the rest."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} out of range for world size {world}")
    if total_rows < 0:
        raise ValueError("negative row count")
    base, extra = divmod(total_rows, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


class Group:
    """This process's place in the replica group (world size 1 when alone)."""

    def __init__(self, backend: Optional[str] = None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        self.backend = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            if backend is None:
                backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.dist = dist
            self.backend = backend

    def _device(self):
        import torch
        return torch.device("cuda", self.local) if self.backend == "nccl" else torch.device("cpu")

    def barrier(self) -> None:
        if self.dist is not None:
            self.dist.barrier()

    def max(self, value: float) -> float:
        """The largest `value` over all ranks (every rank gets it)."""
        if self.dist is None:
            return float(value)
        import torch
        t = torch.tensor([float(value)], dtype=torch.float64, device=self._device())
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def sum(self, value: float) -> float:
        """The sum of `value` over all ranks (every rank gets it)."""
        if self.dist is None:
            return float(value)
        import torch
        t = torch.tensor([float(value)], dtype=torch.float64, device=self._device())
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return float(t.item())

    def close(self) -> None:
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def throughput(rows_all_ranks: float, ms_max: float) -> float:
    """Whole-job rows/s: every rank's rows over the slowest rank's time."""
    if ms_max <= 0:
        raise ValueError("elapsed time must be positive")
    return rows_all_ranks / (ms_max / 1e3)
