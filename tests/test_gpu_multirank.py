"""The multi-GPU partition on the library: two gloo processes each create their
range of a job's samples (shard.sample_range, ea_create_samples_range), sweep them
and reduce the int64 sums on the host.  The totals equal the single-process run of
the whole job bit for bit, and each rank's samples equal the whole job's.  Both
processes share the one GPU here; their kernels never wait on each other, and the
only exchange is the host-side reduction (Sec. III: independent sample batches per
GPU)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

JOB = dict(L=32, p_neg=0.5, seed=23, n_samples=5, T=0.8, rule=0, t_w=[0, 2, 4], t=[0, 1, 2, 4],
           n_sweeps=8, G=1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(job_mod, lo, hi):
    """Integer sums of samples [lo, hi) placed into whole-job arrays, and their spins."""
    S = JOB["n_samples"]
    j = job_mod.EAJob(JOB["L"], JOB["p_neg"], JOB["seed"], hi - lo, rng_group=JOB["G"],
                      first_sample=lo)
    j.set_schedule(JOB["t_w"], JOB["t"])
    j.quench(JOB["T"], JOB["rule"])
    j.sweep(JOB["n_sweeps"])
    vals = []
    for tw in JOB["t_w"]:
        for lag in JOB["t"]:
            m = j.measure(tw, lag)
            for k in ("A", "Q", "E", "G"):
                full = np.zeros((S,) + m[k].shape[1:], dtype=np.int64)
                full[lo:hi] = m[k]
                vals.append(full.ravel())
    spins = [j.all_spins(i) for i in range(hi - lo)]
    j.close()
    return np.concatenate(vals), spins


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist

    from paper_1411_5512_gb300 import job, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    lo, hi = shard.sample_range(JOB["n_samples"], rank, world)
    sums, spins = _run(job, lo, hi)
    total = shard.allreduce_int64(sums)
    q.put((rank, lo, hi, spins, total if rank == 0 else None))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_on_the_library_sum_to_single_process():
    from paper_1411_5512_gb300 import build, job
    build.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=600) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ref, ref_spins = _run(job, 0, JOB["n_samples"])
    total = [g[4] for g in got if g[0] == 0][0]
    assert np.array_equal(total, ref)
    covered = []
    for rank, lo, hi, spins, _ in got:
        for i, s in enumerate(range(lo, hi)):
            assert np.array_equal(spins[i], ref_spins[s]), (rank, s)
            covered.append(s)
    assert sorted(covered) == list(range(JOB["n_samples"]))


def _slab_rank(rank, world, port, q, L, rule):
    import torch
    import torch.distributed as dist

    from paper_1411_5512_gb300 import domain
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    j = domain.run_slab(L, 0.5, 77, 2, 0.8, rule, 3, rank, world)
    lo, hi = domain.slab(L, rank, world)
    q.put((rank, lo, hi, [j.get_rows(a, lo, hi - lo) for a in (0, 1)], j.time))
    j.close()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("L,world,rule", [(128, 2, 0), (64, 3, 1)])
def test_ranks_split_one_lattice(L, world, rule):
    """One lattice in y-slabs over ranks (processes sharing the one GPU) with the halo
    rows exchanged by gloo between the half-steps: every slab equals those rows of the
    undivided lattice, bit for bit."""
    from paper_1411_5512_gb300 import build, job
    build.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_rank, args=(r, world, port, q, L, rule))
             for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=600) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    whole = job.EAJob(L, 0.5, 77, 2)
    whole.quench(0.8, rule)
    whole.sweep(3)
    ref = [whole.get_rows(a, 0, L) for a in (0, 1)]
    covered = []
    for rank, lo, hi, areas, t in got:
        assert t == 3
        for a in (0, 1):
            assert np.array_equal(areas[a], ref[a][:, :, lo:hi, :]), (rank, a)
        covered += list(range(lo, hi))
    assert sorted(covered) == list(range(L))
    whole.close()
