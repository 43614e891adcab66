"""Failures made on the host, never on the GPU: an allocator that refuses memory,
cancelled jobs, calls out of order.  The library must return clean status codes,
leak nothing, and leave other jobs' results unchanged."""
import ctypes
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def J():
    from paper_1411_5512_gb300 import build, job
    build.build()
    return job


class FailingAllocator:
    """Routes allocations to torch, refusing every one after the first `budget`."""

    def __init__(self, budget):
        import torch
        from paper_1411_5512_gb300 import _lib
        self.torch = torch
        self.budget = budget
        self.live = {}

        def _alloc(nbytes, stream, user):
            if self.budget <= 0:
                return None
            self.budget -= 1
            p = int(torch.cuda.caching_allocator_alloc(int(nbytes)))
            self.live[p] = nbytes
            return p

        def _free(ptr, nbytes, stream, user):
            self.live.pop(int(ptr), None)
            torch.cuda.caching_allocator_delete(int(ptr))

        self.a = _lib.ALLOC_FN(_alloc)
        self.f = _lib.FREE_FN(_free)
        _lib.check(_lib.load().ea_set_allocator(self.a, self.f, None))

    def close(self):
        from paper_1411_5512_gb300 import _lib
        _lib.check(_lib.load().ea_set_allocator(_lib.ALLOC_FN(), _lib.FREE_FN(), None))


def test_create_reports_oom_and_frees_partial_allocations(J):
    from paper_1411_5512_gb300 import _lib
    for budget in range(0, 3):  # a job holds three allocations: spins, couplings, its table row
        fa = FailingAllocator(budget)
        try:
            with pytest.raises(_lib.EAError) as e:
                J.EAJob(16, 0.5, 1, 2)
            assert e.value.status == _lib.EA_ERR_OOM
            assert fa.live == {}  # everything handed out was given back
        finally:
            fa.close()
    # a schedule that cannot get its snapshot memory fails cleanly too
    fa = FailingAllocator(3)
    try:
        j = J.EAJob(16, 0.5, 1, 2)
        with pytest.raises(_lib.EAError) as e:
            j.set_schedule([0, 1, 2], [0, 1])
        assert e.value.status == _lib.EA_ERR_OOM
        j.close()
        assert fa.live == {}
    finally:
        fa.close()


def test_server_keeps_unadmittable_jobs_queued_and_cancels(J):
    srv = J.EAServer(1 << 30, max_running=1, chunk_sweeps=4)
    a = srv.submit(16, 0.5, 3, 1, 0.7, 12, t_w=[0], t=[0, 8])
    b = srv.submit(16, 0.5, 4, 1, 0.7, 12, t_w=[0], t=[0, 8])
    c = srv.submit(16, 0.5, 5, 1, 0.7, 12)
    srv.step()
    assert srv.state(a)[0] == 1 and srv.state(b)[0] == 0  # one slot
    srv.cancel(b)                     # queued job leaves the queue
    srv.step()
    srv.cancel(a)                     # running job leaves the batch
    while srv.state(c)[0] != 2:
        srv.step()
    assert srv.stats()["running"] == 0 and srv.stats()["queued"] == 0
    # c is unaffected by the cancellations: same result as alone
    ref = J.EAJob(16, 0.5, 5, 1)
    ref.quench(0.7)
    ref.sweep(12)
    assert np.array_equal(srv.job(c).all_spins(0), ref.all_spins(0))
    ref.close()
    srv.cancel(c)                     # a done job is released
    assert srv.stats()["bytes_in_use"] == 0
    from paper_1411_5512_gb300 import _lib
    with pytest.raises(_lib.EAError):
        srv.cancel(c)
    srv.close()


def test_library_job_continues_from_its_checkpoint(J, tmp_path):
    """The recovery runner on the library: a job stopped after its first chunk and
    continued from its checkpoint gives every scheduled sum of an uninterrupted run."""
    import torch.distributed as dist
    from paper_1411_5512_gb300 import recovery
    spec = dict(L=32, p_neg=0.5, seed=5, n_samples=2, T=0.7, rule=0, sweeps=20,
                t_w=[0, 8], t=[0, 4, 12])
    with pytest.raises(RuntimeError):
        recovery._run_job(0, spec, recovery.LibraryRunner, str(tmp_path), 8, lambda: None,
                          resume=False, fail_after=1)
    resumed = recovery._run_job(0, spec, recovery.LibraryRunner, str(tmp_path), 8,
                                lambda: None, resume=True)
    fresh = recovery._run_job(1, spec, recovery.LibraryRunner, str(tmp_path), 20,
                              lambda: None, resume=False)
    assert resumed == fresh and len(fresh) == 6
    # one rank, the whole list through the coordinator
    os.makedirs(str(tmp_path / "all"))
    res = recovery.run_jobs([spec, dict(spec, seed=6, rule=1)], 0, 1, dist.HashStore(),
                            str(tmp_path / "all"), chunk=7)
    assert sorted(res) == [0, 1] and res[0] == fresh


def test_bounded_wait_runs_out_cleanly(J):
    """A bounded device wait that runs out: the staged side-128 kernel waits on a
    barrier that nothing completes (a test mode), gives up after a few polls, waits
    for its own copies in flight and returns; the status word reports it, and the
    context stays usable: with the normal policy back, a fresh job matches the
    oracle bit for bit."""
    import oracle as ora
    L, p_neg, seed, T = 128, 0.5, 13, 0.7
    j = J.EAJob(L, p_neg, seed, 2)
    j.quench(T)
    b = J.EABatch()
    b.set_variant(1)
    b.add(j)
    assert J.device_status() == 0
    try:
        J.debug_set_wait(16, wait_for_nothing=True)
        b.sweep(1)
        assert J.device_status() & 1
    finally:
        J.debug_set_wait(1 << 22, wait_for_nothing=False)
    assert J.device_status() == 0
    b.close()
    j.close()
    j = J.EAJob(L, p_neg, seed, 2)
    j.quench(T)
    b = J.EABatch()
    b.set_variant(1)
    b.add(j)
    b.sweep(2)
    assert J.device_status() == 0
    ref = ora.run_job(L, p_neg, seed, 2, T, 0, [], [], 2, samples=[1], keep_spins=True)
    assert np.array_equal(j.all_spins(1), ref["spins"][0])
    b.close()
    j.close()
