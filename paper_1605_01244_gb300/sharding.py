"""Multi-GPU sharding of the evaluation: independent point batches per rank.

Points are independent once the oversampled grid exists, so the evaluation
shards by points with no data-path collective: every rank holds the same
coefficients and evaluates its own points (weak scaling: a fixed number of
points per rank).  The only collective is the timing reduction, the
maximum step time over ranks.  (The adjoint would need a sum all-reduce of
the N^3 coefficients; it is not part of the timed step.)
"""
from __future__ import annotations

import torch


def point_seed(rank: int, base: int = 100) -> int:
    """Seed of rank r's point batch (distinct batches per rank)."""
    return base + 7919 * rank


def shard_range(M_total: int, rank: int, world: int):
    """Contiguous [start, stop) slice of M_total points owned by ``rank``
    (a strong-scaling split of one point set; sizes differ by at most one)."""
    q, r = divmod(M_total, world)
    start = rank * q + min(rank, r)
    return start, start + q + (1 if rank < r else 0)


def _initialised():
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized()


def _reduce_device(device):
    """NCCL reduces device tensors; gloo (CPU ranks, or several ranks sharing
    one GPU in tests) reduces host tensors."""
    import torch.distributed as dist
    return device if dist.get_backend() == "nccl" else "cpu"


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar (e.g. a step time) over the process group;
    the value itself when torch.distributed is not initialised."""
    import torch.distributed as dist
    if not _initialised():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=_reduce_device(device))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device=None) -> None:
    """All ranks' queued work done: a process-group barrier (when one is
    initialised) and a device synchronize."""
    import torch.distributed as dist
    if _initialised():
        dist.barrier()
    torch.cuda.synchronize(device)


def timed_steps(step, steps: int, stream, device=None) -> float:
    """Milliseconds per call of ``step()`` over ``steps`` calls: CUDA events
    on ``stream`` (the stream the library launches on), bracketed by a
    barrier and a synchronize on both sides; the maximum over ranks."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(device)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    barrier(device)
    return max_over_ranks(e0.elapsed_time(e1) / max(steps, 1), device)
