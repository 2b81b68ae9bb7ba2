"""Sharding of the particle sum across ranks (one process per GPU, torch.distributed).

The spectrum is a sum over particles (Sec. IV's ensemble average), so ranks take disjoint
particle ranges, compute their partial sums independently, and one all-reduce adds them.
No other data moves between ranks.
"""
from __future__ import annotations


def particle_range(n_particles: int, world: int, rank: int) -> tuple:
    """Contiguous, balanced [p0, p1) of rank `rank` out of `world` (sizes differ by at most 1)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    return (n_particles * rank) // world, (n_particles * (rank + 1)) // world


def step_batch(step: int, rank: int, world: int, batch: int, n_particles: int) -> tuple:
    """[p0, p1) processed by `rank` at `step` in a weak-scaling loop: every rank gets its own
    batch of `batch` particles, batches of one step are disjoint, cycling through the ensemble."""
    n_batches = n_particles // batch
    if n_batches < 1:
        raise ValueError("batch larger than the ensemble")
    b = (step * world + rank) % n_batches
    return b * batch, (b + 1) * batch


def allreduce_sum(tensor, group=None):
    """In-place sum of `tensor` over all ranks (no-op without an initialised process group)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(tensor, op=dist.ReduceOp.SUM, group=group)
    return tensor
