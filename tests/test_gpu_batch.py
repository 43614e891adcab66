"""Batched sweeps: a job's results are bit-identical alone, in any batch, under
any launch shape, across joins and leaves, and equal to the oracle."""
import numpy as np
import pytest

import oracle as ora

pytestmark = pytest.mark.gpu

# L, p_neg, seed, S, T, rule, t_w, t
MIX = [
    (16, 0.5, 11, 2, 0.7, 0, [0, 2, 8], [0, 1, 4]),
    (24, 0.3, 12, 1, 0.9, 0, [0, 4], [0, 2, 8]),
    (8, 0.1, 13, 3, 0.6, 0, [0, 1, 3], [0, 5]),
    (12, 0.5, 14, 1, 1.2, 1, [0, 8], [0, 1]),   # heat bath in the same batch
    (32, 0.4, 15, 1, 0.5, 0, [0], [0, 16]),
    (6, 0.5, 16, 2, 0.8, 0, [], []),
    (64, 0.3, 17, 1, 0.7, 0, [0, 4], [0, 8]),  # tile kernel run, forked from the column kernel's
    (128, 0.5, 18, 1, 0.7, 0, [0, 2], [0, 4]),  # a second tile kernel run on the other side stream
]


@pytest.fixture(scope="module")
def J():
    from paper_1411_5512_gb300 import build, job
    build.build()
    return job


def make(J, spec, stream=None):
    L, p, seed, S, T, rule, tw, tt = spec
    j = J.EAJob(L, p, seed, S, stream=stream)
    j.set_schedule(tw, tt)
    j.quench(T, rule)
    return j


def snapshot(j, spec, n):
    L, p, seed, S, T, rule, tw, tt = spec
    out = {"spins": [j.all_spins(s) for s in range(S)], "m": {}}
    for a in tw:
        for b in tt:
            if a + b <= n:
                m = j.measure(a, b)
                out["m"][(a, b)] = {k: m[k] for k in ("A", "Q", "E", "G")}
    return out


def same(x, y):
    if len(x["spins"]) != len(y["spins"]):
        return False
    for a, b in zip(x["spins"], y["spins"]):
        if not np.array_equal(a, b):
            return False
    if set(x["m"]) != set(y["m"]):
        return False
    for k in x["m"]:
        for f in ("A", "Q", "E", "G"):
            if not np.array_equal(x["m"][k][f], y["m"][k][f]):
                return False
    return True


def alone(J, n):
    res = []
    for spec in MIX:
        j = make(J, spec)
        j.sweep(n)
        res.append(snapshot(j, spec, n))
        j.close()
    return res


@pytest.mark.parametrize("cpt,graph,res", [(0, 0, 64), (1, 0, 0), (2, 4, 64), (4, 16, 0),
                                           (1, 7, 64), (2, 0, 32)])
def test_batch_equals_alone(J, cpt, graph, res):
    """A job alone (sample-resident where its side allows) equals the same job in a
    mixed batch under every launch shape, graph length and resident limit."""
    import torch
    n = 21
    ref = alone(J, n)
    stream = torch.cuda.Stream()
    b = J.EABatch(stream=stream)
    b.configure(cpt, graph)
    b.set_resident(res)
    jobs = [make(J, spec, stream=stream) for spec in MIX]
    for j in jobs:
        b.add(j)
    assert len(b) == len(MIX)
    b.sweep(5)
    b.sweep(16)
    for j, spec, r in zip(jobs, MIX, ref):
        assert same(snapshot(j, spec, n), r), spec
    b.close()
    for j in jobs:
        j.close()


def test_batch_matches_oracle(J):
    import torch
    stream = torch.cuda.Stream()
    b = J.EABatch(stream=stream)
    b.configure(2, 8)
    jobs = [make(J, spec, stream=stream) for spec in MIX[:4]]
    for j in jobs:
        b.add(j)
    n = 12
    b.sweep(n)
    for j, spec in zip(jobs, MIX[:4]):
        L, p, seed, S, T, rule, tw, tt = spec
        out = ora.run_job(L, p, seed, S, T, rule, tw, tt, n, keep_spins=True)
        for s in range(S):
            assert np.array_equal(j.all_spins(s), out["spins"][s])
        for a in tw:
            for c in tt:
                if a + c <= n:
                    m = j.measure(a, c)
                    assert np.array_equal(m["A"], out["A"][(a, c)])
                    assert np.array_equal(m["G"], out["G"][a])
    b.close()


def test_join_and_leave_mid_run(J):
    import torch
    n = 30
    ref = alone(J, n)
    stream = torch.cuda.Stream()
    b = J.EABatch(stream=stream)
    b.configure(1, 4)
    jobs = [make(J, spec) for spec in MIX]  # own (default) streams
    # first two jobs run alone for a while, then join; the others join at once
    jobs[0].sweep(7)
    jobs[1].sweep(3)
    for j in jobs[2:]:
        b.add(j)
    b.sweep(3)
    b.add(jobs[1])
    b.sweep(4)
    b.add(jobs[0])
    # now jobs[0] is at 7, jobs[1] at 7, others at 7: run to n together
    b.sweep(n - 7 - 10)
    b.remove(jobs[2])
    jobs[2].sweep(10)  # finishes alone
    b.sweep(10)
    for j, spec, r in zip(jobs, MIX, ref):
        assert j.time == n
        assert same(snapshot(j, spec, n), r), spec
    b.close()
    for j in jobs:
        j.close()


def test_autotune_changes_nothing(J):
    import torch
    n = 16
    ref = alone(J, n)
    stream = torch.cuda.Stream()
    b = J.EABatch(stream=stream)
    jobs = [make(J, spec, stream=stream) for spec in MIX]
    for j in jobs:
        b.add(j)
    b.sweep(4)
    cfg = b.autotune(trial_sweeps=6)
    assert cfg[0] in (1, 2, 4) and 0 <= cfg[1] <= 6
    assert 1 <= b.streams() <= 4 and b.resident() in (32, 64, 0)
    b.sweep(n - 4)
    for j, spec, r in zip(jobs, MIX, ref):
        assert same(snapshot(j, spec, n), r), spec
    b.close()
    for j in jobs:
        j.close()


@pytest.mark.parametrize("L", [24, 64, 128])
def test_profile_counts_words_and_restores_state(J, L):
    """The counting launch visits every word once per half-step, counts at least
    one Philox call per two words that need one, and leaves the state as it was."""
    spec = (L, 0.5, 77, 2, 0.8, 0, [], [])
    S, n = spec[3], 3
    j, ref = make(J, spec), make(J, spec)
    b = J.EABatch()
    b.add(j)
    prof = b.profile(sweeps=n)
    words = L ** 3 // 32  # all three sides have 32 lanes per word
    assert prof["words"] == n * 2 * S * words
    assert prof["flips"] == n * 2 * S * L ** 3
    assert prof["rare_calls"] <= prof["philox_calls"] <= prof["words"]
    assert prof["philox_calls"] >= prof["words"] // 4
    b.sweep(5)
    ref.sweep(5)
    for s in range(S):
        assert np.array_equal(j.all_spins(s), ref.all_spins(s))
    b.close()
    j.close()
    ref.close()


def test_launch_count(J):
    """The library's launch counter: two half-step launches per sweep, or one
    sample-resident launch for up to 1024 sweeps; a batch adds one time-advance kernel
    per enqueue, and a graph of K sweeps, replayed, counts the kernels it holds and its
    time advance."""
    import torch
    j = make(J, (16, 0.5, 3, 1, 0.7, 0, [], []))
    n0 = J.launch_count()
    j.sweep(5)  # side 16 swept on its own: sample-resident
    assert J.launch_count() - n0 == 1
    n0 = J.launch_count()
    j.sweep(1500)
    assert J.launch_count() - n0 == 2
    b = J.EABatch()  # default stream: direct launches, no graph
    b.configure(1, 4)
    b.set_resident(0)
    b.add(j)
    n0 = J.launch_count()
    b.sweep(8)
    assert J.launch_count() - n0 == 2 * 8 + 1
    b.set_resident(64)
    n0 = J.launch_count()
    b.sweep(8)
    assert J.launch_count() - n0 == 1 + 1
    b.close()
    stream = torch.cuda.Stream()
    b = J.EABatch(stream=stream)
    b.configure(1, 4)
    b.set_resident(0)
    b.add(j)
    b.sweep(4)  # captures the graph (capturing counts nothing) and replays it once
    n0 = J.launch_count()
    b.sweep(8)
    assert J.launch_count() - n0 == 2 * (2 * 4 + 1)
    b.close()
    j.close()


def test_graph_follows_member_swaps_and_requench(J):
    """A captured graph holds the members' pointers and class flags in its launches:
    swapping a member for another of the same shape, or quenching one again at another
    temperature, must take a new graph.  Every job equals the same job run alone."""
    import torch
    stream = torch.cuda.Stream()
    b = J.EABatch(stream=stream)
    b.configure(1, 4)
    L, S = 32, 2
    a = J.EAJob(L, 0.5, 901, S, stream=stream)
    c = J.EAJob(L, 0.5, 902, S, stream=stream)  # the same shape as a
    a.quench(0.7)
    c.quench(0.7)
    b.add(a)
    b.sweep(8)                  # a graph with a's pointers
    b.remove(a)
    b.add(c)
    b.sweep(8)                  # the same table size and shape: a new graph all the same
    c.quench(0.0)               # again at T = 0: other class flags (no random numbers)
    b.sweep(8)
    b.close()
    ra = J.EAJob(L, 0.5, 901, S)
    ra.quench(0.7)
    ra.sweep(8)
    rc = J.EAJob(L, 0.5, 902, S)
    rc.quench(0.0)
    rc.sweep(8)
    for s in range(S):
        assert np.array_equal(a.all_spins(s), ra.all_spins(s)), s
        assert np.array_equal(c.all_spins(s), rc.all_spins(s)), s
    assert a.time == 8 and c.time == 8
    for j in (a, c, ra, rc):
        j.close()


# Batches whose members all run on one kernel, so that the batch splits them
# into groups of whole jobs over its streams: side 128 (tile kernel), side 96
# (general tiles), side 64 heat bath, side 24 (column kernel, not resident here)
ONE_KERNEL = {
    "tile128": [(128, p, 30 + i, 1, 0.7, 0, [0, 2], [0, 4])
                for i, p in enumerate((0.5, 0.4, 0.3, 0.2, 0.1))],
    "gtile96": [(96, 0.5, 40 + i, 1, 0.8, 0, [0, 4], [0, 2]) for i in range(3)],
    "heat64": [(64, 0.5, 50 + i, 1, 0.8, 1, [0, 4], [0, 8]) for i in range(4)],
    "column24": [(24, 0.3, 60 + i, 2, 0.7, 0, [0], [0, 2, 8]) for i in range(6)],
}


@pytest.mark.parametrize("streams", [1, 2, 3, 5])
@pytest.mark.parametrize("case", sorted(ONE_KERNEL))
def test_streams_split_changes_nothing(J, case, streams):
    """A batch of jobs on one kernel, split into 1, 2, 3 or 5 groups on streams of
    their own, gives every job exactly what it gives alone; the side-64 heat-bath and
    side-24 groups are also checked against the oracle."""
    import torch
    specs = ONE_KERNEL[case]
    n = 21
    ref = []
    for spec in specs:
        j = make(J, spec)
        j.sweep(n)
        ref.append(snapshot(j, spec, n))
        j.close()
    stream = torch.cuda.Stream()
    b = J.EABatch(stream=stream)
    b.configure(2, 4)
    b.set_resident(0)
    b.set_streams(streams)
    assert b.streams() == streams
    jobs = [make(J, spec, stream=stream) for spec in specs]
    for j in jobs:
        b.add(j)
    b.sweep(5)
    b.sweep(16)
    for j, spec, r in zip(jobs, specs, ref):
        assert same(snapshot(j, spec, n), r), (case, streams, spec)
    if case in ("heat64", "column24") and streams == 3:
        for j, spec in zip(jobs[:2], specs[:2]):
            L, p, seed, S, T, rule, tw, tt = spec
            out = ora.run_job(L, p, seed, S, T, rule, tw, tt, n, keep_spins=True)
            for s in range(S):
                assert np.array_equal(j.all_spins(s), out["spins"][s])
    b.close()
    for j in jobs:
        j.close()


def test_streams_rejects_bad_counts(J):
    b = J.EABatch()
    for bad in (0, 6, -1):
        with pytest.raises(Exception):
            b.set_streams(bad)
    assert b.streams() == 3
    b.close()
