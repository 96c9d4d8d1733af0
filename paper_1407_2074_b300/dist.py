"""Multi-rank bookkeeping of the benchmark.  The hot path shards by rays / frames with a replicated
volume and no data exchange, so the only cross-rank operations are the barrier around the timed
region and the reduction of its results: time = max over ranks, work = sum over ranks."""
from __future__ import annotations


def env():
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 without it)."""
    import os

    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def aggregate(elapsed_ms: float, work: float, device=None):
    """Returns (max elapsed over ranks, summed work over ranks); identity without a process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed_ms), float(work)
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def frames_for_rank(rank: int, steps: int, n_frames: int):
    """Orbit frames of one rank: rank r renders frames r*steps, r*steps + 1, ... of the orbit, wrapping
    around it.  The ranks' frames are disjoint while ranks x steps <= n_frames; beyond that the
    orbit repeats and ranks render some of the same views.  Each rank holds its own replica of the
    volume on its own GPU, so a repeated view is still a full render there (nothing is shared or
    cached across ranks); only the mix of view angles in the timed region changes."""
    return [(rank * steps + i) % n_frames for i in range(steps)]
