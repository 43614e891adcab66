"""One lattice split into y-slabs over ranks: the single-lattice decomposition that
Sec. III sketches for lattices larger than one GPU.

Rank r of `world` owns the rows [lo, hi) of the lattice (sides 64 and 128, whose
word lattice keeps every lane along z, so that a row of words is a row of sites).
Half-step h updates spin area h and reads area 1 - h as neighbours; before it,
every rank publishes its first and last row of area 1 - h and takes the row just
below its slab from the previous rank and the row just above from the next one
(periodic).  Only that halo crosses ranks: the couplings and the initial state are
drawn identically on every rank from the job's seed, and every random number is
keyed by the site's own coordinates, so the result is bit-identical to the
undivided lattice.  The exchange runs on the host (torch.distributed, any
backend) between the half-steps; no kernel ever waits on another rank.
"""
import numpy as np

from . import shard


def slab(L, rank, world):
    """[lo, hi): the rows of an L-row lattice that `rank` updates."""
    return shard.sample_range(L, rank, world)


def halo_sources(L, rank, world):
    """((rank, row) of the row below the slab, (rank, row) of the row above it):
    the previous rank's last row and the next rank's first row, periodic."""
    lo, hi = slab(L, rank, world)
    prev, nxt = (rank - 1) % world, (rank + 1) % world
    return (prev, slab(L, prev, world)[1] - 1), (nxt, slab(L, nxt, world)[0])


def exchange_halo(job, area, rank, world, group=None):
    """Bring rows lo - 1 and hi of spin area `area` up to date from the neighbours."""
    import torch
    import torch.distributed as dist

    L = job.L
    lo, hi = slab(L, rank, world)
    mine = np.concatenate([job.get_rows(area, lo, 1), job.get_rows(area, hi - 1, 1)], axis=2)
    if world == 1:
        gathered = [mine]
    else:
        t = torch.from_numpy(mine.view(np.int32).copy())
        bufs = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(bufs, t, group=group)
        gathered = [b.numpy().view(np.uint32) for b in bufs]
    (pr, prow), (nr, nrow) = halo_sources(L, rank, world)
    job.set_rows(area, (lo - 1) % L, gathered[pr][:, :, 1:2, :])  # their last row
    job.set_rows(area, hi % L, gathered[nr][:, :, 0:1, :])        # their first row
    assert prow == (lo - 1) % L and nrow == hi % L


def run_slab(L, p_neg, seed, n_samples, T, rule, sweeps, rank, world, group=None,
             stream=None):
    """Sweep the slab of `rank`; returns the job (its own rows are the result)."""
    from . import job as jobmod

    lo, hi = slab(L, rank, world)
    j = jobmod.EAJob(L, p_neg, seed, n_samples, stream=stream)
    j.quench(T, rule)
    j.set_row_range(lo, hi)
    for _ in range(sweeps):
        for h in (0, 1):
            exchange_halo(j, 1 - h, rank, world, group)
            j.half_sweep()
    return j
