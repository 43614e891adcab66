"""The multi-GPU path on CPU: two gloo ranks split the samples of a job, compute
their observables independently and reduce the int64 sums; the result equals
the single-process run exactly (the oracle stands in for each rank's device)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle as ora
from paper_1411_5512_gb300 import shard

JOB = dict(L=6, p_neg=0.5, seed=17, n_samples=5, T=0.8, rule=0, t_w=[0, 2], t=[0, 1, 4],
           n_sweeps=6)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _sums(out, samples_total, samples):
    """Observable sums of a run_job result placed into full-size arrays."""
    keys = []
    vals = []
    for k in sorted(out["A"]):
        a = np.zeros((samples_total, 2), dtype=np.int64)
        a[samples] = out["A"][k]
        vals.append(a.ravel())
    for k in sorted(out["G"]):
        g = np.zeros((samples_total,) + out["G"][k].shape[1:], dtype=np.int64)
        g[samples] = out["G"][k]
        vals.append(g.ravel())
    for k in sorted(out["Q"]):
        q = np.zeros(samples_total, dtype=np.int64)
        q[samples] = out["Q"][k]
        vals.append(q)
    return np.concatenate(vals)


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = shard.sample_range(JOB["n_samples"], rank, world)
    mine = list(range(lo, hi))
    out = ora.run_job(JOB["L"], JOB["p_neg"], JOB["seed"], JOB["n_samples"], JOB["T"],
                      JOB["rule"], JOB["t_w"], JOB["t"], JOB["n_sweeps"], samples=mine)
    total = shard.allreduce_int64(_sums(out, JOB["n_samples"], mine))
    tmax = shard.max_over_ranks(float(rank + 1))
    if rank == 0:
        q.put((total, tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_partition():
    units = list(range(11))
    parts = [shard.shard(units, r, 3) for r in range(3)]
    assert sum(parts, []) == units
    assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
    assert shard.sample_range(4, 3, 4) == (3, 4)
    assert shard.sample_range(2, 0, 3) == (0, 0)  # more ranks than samples: an empty share
    assert shard.sample_range(2, 2, 3) == (1, 2)
    with pytest.raises(ValueError):
        shard.shard(units, 3, 3)


def test_two_gloo_ranks_sum_to_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    total, tmax = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    full = ora.run_job(JOB["L"], JOB["p_neg"], JOB["seed"], JOB["n_samples"], JOB["T"],
                       JOB["rule"], JOB["t_w"], JOB["t"], JOB["n_sweeps"])
    ref = _sums(full, JOB["n_samples"], list(range(JOB["n_samples"])))
    assert np.array_equal(total, ref)
    assert tmax == 2.0


@pytest.mark.parametrize("L", [64, 128])
@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_slabs_and_halo_sources(L, world):
    """The y-slabs of one lattice cover every row once; the row below a slab is the
    previous rank's last row and the row above it the next rank's first (periodic)."""
    from paper_1411_5512_gb300 import domain
    rows = []
    for r in range(world):
        lo, hi = domain.slab(L, r, world)
        assert hi > lo
        rows += list(range(lo, hi))
        (pr, prow), (nr, nrow) = domain.halo_sources(L, r, world)
        assert prow == (lo - 1) % L and nrow == hi % L
        plo, phi = domain.slab(L, pr, world)
        nlo, nhi = domain.slab(L, nr, world)
        assert plo <= prow < phi and nlo <= nrow < nhi
    assert rows == list(range(L))
