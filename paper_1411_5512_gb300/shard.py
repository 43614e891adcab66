"""Placement of independent units (jobs, samples) across ranks.

Samples and jobs of the ageing study are independent (Sec. III: separate
batches ran on separate GPUs), so a multi-GPU run is a partition of the units
with no exchange on the data path.  Every random number is keyed by the
job-local sample index, so a unit's results do not depend on where it runs;
integer observable sums from different ranks add exactly in any order.
"""


def shard(units, rank, world):
    """The units of `rank`: a contiguous, balanced block (sizes differ by <= 1)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    n = len(units)
    lo = (n * rank) // world
    hi = (n * (rank + 1)) // world
    return list(units[lo:hi])


def sample_range(n_samples, rank, world):
    """[lo, hi) sample indices of one job handled by `rank`."""
    r = shard(list(range(n_samples)), rank, world)
    return (r[0], r[-1] + 1) if r else (0, 0)


def allreduce_int64(values, group=None):
    """Exact sum over ranks of an int64 array (host tensors, any backend)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    t = torch.from_numpy(np.ascontiguousarray(values, dtype=np.int64).copy())
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.numpy()


def max_over_ranks(x, device=None):
    """Max of a float over ranks (the bench's step time)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
