"""Serving: jobs submitted while others run are admitted by footprint and slots,
share launches, and give bit-identical results alone and in the mix."""
import numpy as np
import pytest

import oracle as ora

pytestmark = pytest.mark.gpu

# L, p_neg, seed, S, T, rule, sweeps, t_w, t
STREAM = [
    (16, 0.5, 101, 2, 0.7, 0, 40, [0, 4, 16], [0, 2, 8]),
    (8, 0.2, 102, 1, 0.5, 0, 13, [0, 1], [0, 4]),
    (24, 0.4, 103, 1, 0.9, 0, 25, [0, 8], [0, 1, 16]),
    (12, 0.5, 104, 3, 1.1, 1, 9, [0], [0, 8]),
    (16, 0.1, 105, 1, 0.6, 0, 70, [0, 32], [0, 32]),
    (32, 0.3, 106, 1, 0.8, 0, 6, [0, 2], [0, 4]),
    (6, 0.5, 107, 2, 0.7, 0, 31, [], []),
    (8, 0.5, 108, 1, 0.7, 0, 0, [0], [0]),          # zero sweeps
    (16, 0.5, 109, 1, 0.7, 0, 17, [0, 16], [0, 1]),
    (24, 0.25, 110, 2, 0.55, 0, 12, [0, 4], [0, 8]),
    (48, 0.5, 111, 1, 0.7, 0, 9, [0, 8], [0, 1]),   # the general tile kernel
    (64, 0.3, 112, 1, 0.8, 1, 7, [0], [0, 4]),      # the heat-bath tile kernel
]


@pytest.fixture(scope="module")
def J():
    from paper_1411_5512_gb300 import build, job
    build.build()
    return job


def results(j, spec):
    L, p, seed, S, T, rule, n, tw, tt = spec
    out = {"spins": [j.all_spins(s) for s in range(S)], "m": {}}
    for a in tw:
        for b in tt:
            if a + b <= n:
                m = j.measure(a, b)
                out["m"][(a, b)] = [m[k].copy() for k in ("A", "Q", "E", "G")]
    return out


def alone(J, spec):
    L, p, seed, S, T, rule, n, tw, tt = spec
    j = J.EAJob(L, p, seed, S)
    j.set_schedule(tw, tt)
    j.quench(T, rule)
    j.sweep(n)
    r = results(j, spec)
    j.close()
    return r


def same(a, b):
    if any(not np.array_equal(x, y) for x, y in zip(a["spins"], b["spins"])):
        return False
    if set(a["m"]) != set(b["m"]):
        return False
    return all(np.array_equal(x, y) for k in a["m"] for x, y in zip(a["m"][k], b["m"][k]))


@pytest.mark.parametrize("max_running,chunk,budget_jobs", [(3, 8, 3), (16, 5, 16), (4, 64, 2)])
def test_serving_mix_equals_alone(J, max_running, chunk, budget_jobs):
    import torch
    ref = [alone(J, spec) for spec in STREAM]
    stream = torch.cuda.Stream()
    # budget: about `budget_jobs` of the largest footprints
    fp = max(J.footprint(s[0], s[3], len(s[7]), len(s[8])) for s in STREAM)
    srv = J.EAServer(budget_jobs * fp, max_running=max_running, chunk_sweeps=chunk, stream=stream)
    ids = {}
    pending = list(enumerate(STREAM))
    done = {}
    rounds = 0
    while len(done) < len(STREAM):
        # two new arrivals per round, while earlier jobs are on the GPU
        for _ in range(2):
            if pending:
                i, spec = pending.pop(0)
                L, p, seed, S, T, rule, n, tw, tt = spec
                ids[i] = srv.submit(L, p, seed, S, T, n, tw, tt, rule=rule)
        srv.step()
        st = srv.stats()
        assert st["running"] <= max_running
        assert st["bytes_in_use"] <= budget_jobs * fp
        for i, jid in ids.items():
            if i in done:
                continue
            state, t = srv.state(jid)
            if state == 2:
                spec = STREAM[i]
                assert t == spec[6]
                done[i] = results(srv.job(jid), spec)
                srv.release(jid)
        rounds += 1
        assert rounds < 1000
    for i, spec in enumerate(STREAM):
        assert same(done[i], ref[i]), spec
    # the oracle agrees with one job of the mix
    L, p, seed, S, T, rule, n, tw, tt = STREAM[0]
    out = ora.run_job(L, p, seed, S, T, rule, tw, tt, n, keep_spins=True)
    for s in range(S):
        assert np.array_equal(done[0]["spins"][s], out["spins"][s])
    srv.close()


def test_server_rejects_oversized_and_bad_jobs(J):
    from paper_1411_5512_gb300 import _lib
    srv = J.EAServer(1 << 20, max_running=2, chunk_sweeps=4)
    with pytest.raises(_lib.EAError):
        srv.submit(128, 0.5, 1, 4, 0.7, 10)  # 5 MB of state > 1 MB budget
    with pytest.raises(_lib.EAError):
        srv.submit(15, 0.5, 1, 1, 0.7, 10)   # odd L
    jid = srv.submit(8, 0.5, 1, 1, 0.7, 3)
    with pytest.raises(_lib.EAError):
        srv.release(jid)                     # not done yet
    while srv.state(jid)[0] != 2:
        srv.step()
    srv.release(jid)
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()
