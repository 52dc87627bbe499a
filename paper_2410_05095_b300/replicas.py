"""Host logic of multi-GPU runs: the path has no exchange step, so N GPUs run
N independent replicas.  Each rank renders its own frames (or its own row
band of one image); the job's time is the slowest rank's."""
from __future__ import annotations


def row_bands(height: int, world: int):
    """Split image rows into `world` contiguous bands [r0, r1) (covering every
    row once; the first bands take the remainder)."""
    base, extra = divmod(height, world)
    out, r = [], 0
    for k in range(world):
        n = base + (1 if k < extra else 0)
        out.append((r, r + n))
        r += n
    return out


def max_over_ranks(value: float, device=None) -> float:
    """All-reduce MAX of a per-rank time (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_ms_per_frame(local_ms_total: float, frames_per_rank: int, device=None) -> float:
    """Whole-job milliseconds per frame: slowest rank's time over all frames
    that all ranks rendered."""
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    return max_over_ranks(local_ms_total, device) / (frames_per_rank * world)
