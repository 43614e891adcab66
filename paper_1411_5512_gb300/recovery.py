"""Independent jobs over ranks, with recovery from a rank that stops.

Jobs are independent and every random number is keyed by (seed, sample,
sweep), so a job continued from a checkpoint on another rank gives the same
results bit for bit (checkpoints hold the whole state: spins, couplings,
snapshots and the time).  A run proceeds as follows:

- job i belongs to rank i mod world;
- a rank runs its jobs in chunks of sweeps; after each chunk it writes the
  job's checkpoint (to a temporary name, then renamed, so a checkpoint is
  always whole) and bumps its heartbeat counter in the key-value store;
- a finished job's result goes to the store;
- rank 0, when done with its own jobs, collects the others' results.  A rank
  whose heartbeat has not moved for `timeout` seconds is declared stopped, and
  rank 0 continues each of its unfinished jobs from its last checkpoint (or
  from the start, without one).

Failures are detected on the host only: a stopped rank is a process that
exits or stops answering, never a device fault.  Only the store is used after
a failure, no collective, so a missing rank cannot block the others.

The runner decides what a job is and where it runs: `LibraryRunner` drives the
CUDA library (ea_checkpoint / ea_restore); the tests pass a CPU runner.
"""
import json
import os
import time


class LibraryRunner:
    """A job of the CUDA library: spec = dict(L, p_neg, seed, n_samples, T, rule,
    sweeps, t_w, t).  The result is the integer sums of every scheduled (t_w, t)."""

    def __init__(self, spec):
        self.spec = spec
        self.job = None

    def start(self):
        from . import job
        s = self.spec
        self.job = job.EAJob(s["L"], s["p_neg"], s["seed"], s["n_samples"])
        self.job.set_schedule(s.get("t_w", []), s.get("t", []))
        self.job.quench(s["T"], s.get("rule", 0))

    def resume(self, path):
        from . import job
        self.job = job.EAJob.restore(path)

    def time(self):
        return self.job.time

    def advance(self, n):
        self.job.sweep(n)

    def save(self, path):
        self.job.checkpoint(path)

    def result(self):
        s = self.spec
        out = {}
        for tw in s.get("t_w", []):
            for lag in s.get("t", []):
                if tw + lag <= self.job.time:
                    m = self.job.measure(tw, lag)
                    out["%d,%d" % (tw, lag)] = {k: m[k].tolist() for k in ("A", "Q", "E", "G")}
        return out

    def close(self):
        if self.job is not None:
            self.job.close()
            self.job = None


def _ckpt(ckpt_dir, i):
    return os.path.join(ckpt_dir, "job%d.ckpt" % i)


def _run_job(i, spec, runner_factory, ckpt_dir, chunk, beat, resume, fail_after=None):
    """Run job i to its end in chunks, checkpointing after each; beat() after each
    chunk.  fail_after: stop (raise) once that many chunks are done, 0 before the
    first (for tests)."""
    r = runner_factory(spec)
    path = _ckpt(ckpt_dir, i)
    try:
        if resume and os.path.exists(path):
            r.resume(path)
        else:
            r.start()
        chunks = 0
        while r.time() < spec["sweeps"]:
            if fail_after is not None and chunks >= fail_after:
                raise RuntimeError("rank stopped on purpose after %d chunks" % chunks)
            r.advance(min(chunk, spec["sweeps"] - r.time()))
            r.save(path + ".tmp")
            os.replace(path + ".tmp", path)
            chunks += 1
            beat()
        return r.result()
    finally:
        r.close()


def run_jobs(jobs, rank, world, store, ckpt_dir, runner_factory=LibraryRunner, chunk=1000,
             timeout=30.0, poll=0.05, fail_after=None):
    """Run `jobs` (a list of specs) over `world` ranks sharing `store` (a
    torch.distributed Store) and `ckpt_dir` (a directory all ranks see).  Rank 0
    returns {job index: result} for every job, including those of ranks that
    stopped; the other ranks return their own.  fail_after: this rank stops
    after that many chunks of its first job (for tests)."""
    mine = [i for i in range(len(jobs)) if i % world == rank]
    done = {}

    def beat():
        store.add("hb/%d" % rank, 1)

    beat()
    for n, i in enumerate(mine):
        res = _run_job(i, jobs[i], runner_factory, ckpt_dir, chunk, beat, resume=False,
                       fail_after=fail_after if n == 0 else None)
        store.set("res/%d" % i, json.dumps(res))
        done[i] = res
    store.add("finished/%d" % rank, 1)
    if rank != 0:
        return done

    # rank 0 collects; a rank whose heartbeat stands still for `timeout` seconds has stopped
    last = {r: (store.add("hb/%d" % r, 0), time.monotonic()) for r in range(1, world)}
    stopped = set()
    pending = [i for i in range(len(jobs)) if i % world != 0]
    while pending:
        for i in list(pending):
            if store.check(["res/%d" % i]):
                done[i] = json.loads(store.get("res/%d" % i))
                pending.remove(i)
        for r in range(1, world):
            if r in stopped or store.add("finished/%d" % r, 0) > 0:
                continue
            hb = store.add("hb/%d" % r, 0)
            if hb != last[r][0]:
                last[r] = (hb, time.monotonic())
            elif time.monotonic() - last[r][1] > timeout:
                stopped.add(r)
        # continue the unfinished jobs of the stopped ranks from their checkpoints
        for i in list(pending):
            if i % world in stopped:
                res = _run_job(i, jobs[i], runner_factory, ckpt_dir, chunk, beat, resume=True)
                store.set("res/%d" % i, json.dumps(res))
                done[i] = res
                pending.remove(i)
        if pending:
            time.sleep(poll)
    return done
