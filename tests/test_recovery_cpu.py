"""Recovery from a rank that stops, on the host: two CPU ranks share a TCP store and a
checkpoint directory; the oracle stands in for the device.  When rank 1 stops after
its first chunk, rank 0 notices that its heartbeat stands still, continues the job
from its checkpoint, runs rank 1's other jobs, and every result equals the
uninterrupted run exactly."""
import datetime
import multiprocessing
import os
import socket

import numpy as np
import pytest

import oracle as ora
from paper_1411_5512_gb300 import recovery

JOBS = [dict(L=6, p_neg=0.5, seed=31 + i, n_samples=2, T=0.8, rule=i % 2, sweeps=9)
        for i in range(5)]


class OracleRunner:
    """A job on the CPU oracle: the state is the spins of every sample and the
    time; the result is A(0, t), Q(t) and E(t) at the end."""

    def __init__(self, spec):
        self.spec = spec

    def start(self):
        s = self.spec
        self.J = [ora.init_couplings(s["L"], s["p_neg"], s["seed"], k) for k in range(s["n_samples"])]
        self.S = [ora.init_spins(s["L"], s["seed"], k) for k in range(s["n_samples"])]
        self.S0 = [x.copy() for x in self.S]
        self.t = 0

    def resume(self, path):
        open(path + ".resumed", "w").close()  # evidence for the test
        with open(path, "rb") as f:
            z = np.load(f)
            self.J, self.S, self.S0 = list(z["J"]), list(z["S"]), list(z["S0"])
            self.t = int(z["t"])

    def time(self):
        return self.t

    def advance(self, n):
        s = self.spec
        for k in range(s["n_samples"]):
            ora.sweeps(s["L"], s["seed"], k, self.S[k], self.J[k], s["T"], s["rule"], self.t, n)
        self.t += n

    def save(self, path):
        with open(path, "wb") as f:
            np.savez(f, J=np.stack(self.J), S=np.stack(self.S), S0=np.stack(self.S0), t=self.t)

    def result(self):
        return {"A": [ora.autocorr_sum(a, b).tolist() for a, b in zip(self.S0, self.S)],
                "Q": [int(ora.overlap_sum(x)) for x in self.S],
                "E": [ora.energy(x, j).tolist() for x, j in zip(self.S, self.J)]}

    def close(self):
        pass


def _reference():
    out = {}
    for i, spec in enumerate(JOBS):
        r = OracleRunner(spec)
        r.start()
        r.advance(spec["sweeps"])
        out[i] = r.result()
    return out


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ckpt_dir, fail_rank, q):
    import torch.distributed as dist
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0,
                          timeout=datetime.timedelta(seconds=60))
    # fail_rank: the rank that stops after its first chunk; with three ranks, rank 2
    # also stops, before any chunk
    fail = 1 if rank == fail_rank else (0 if (world == 3 and rank == 2 and fail_rank) else None)
    try:
        res = recovery.run_jobs(JOBS, rank, world, store, ckpt_dir, runner_factory=OracleRunner,
                                chunk=4, timeout=2.0, fail_after=fail)
    except RuntimeError:
        os._exit(3)  # this rank stops: no result, no further heartbeat
    if rank == 0:
        q.put({int(k): v for k, v in res.items()})
    store.add("exited/%d" % rank, 1)


def _run(world, fail_rank, tmp_path):
    ctx = multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, str(tmp_path), fail_rank, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    codes = [p.exitcode for p in procs]
    return res, codes


@pytest.mark.parametrize("fail_rank", [None, 1])
def test_jobs_of_a_stopped_rank_continue_from_their_checkpoints(tmp_path, fail_rank):
    ref = _reference()
    res, codes = _run(2, fail_rank, tmp_path)
    assert sorted(res) == list(range(len(JOBS)))
    for i in ref:
        assert res[i] == ref[i], i
    if fail_rank is None:
        assert codes == [0, 0]
    else:
        assert codes[0] == 0 and codes[1] == 3
        # rank 1's first job was continued from the checkpoint written after its first
        # chunk; its second job had none and ran from the start on rank 0
        assert os.path.exists(os.path.join(str(tmp_path), "job1.ckpt.resumed"))
        assert not os.path.exists(os.path.join(str(tmp_path), "job3.ckpt.resumed"))


def test_two_ranks_stop_one_before_its_first_chunk(tmp_path):
    """Three ranks: rank 1 stops after one chunk, rank 2 before any.  Rank 0 continues
    rank 1's job from its checkpoint and runs rank 2's jobs from the start."""
    ref = _reference()
    res, codes = _run(3, 1, tmp_path)
    assert sorted(res) == list(range(len(JOBS)))
    for i in ref:
        assert res[i] == ref[i], i
    assert codes[0] == 0 and codes[1] == 3 and codes[2] == 3
    assert os.path.exists(os.path.join(str(tmp_path), "job1.ckpt.resumed"))
    # rank 2 wrote no checkpoint, so rank 0 ran its jobs from the start
    assert not os.path.exists(os.path.join(str(tmp_path), "job2.ckpt.resumed"))
