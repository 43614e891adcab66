"""Full-length runs against the oracle, from t = 0 on both sides.

* The side-32 configuration of 64 samples x 2 replicas at T = 0.6 and T = 0.8,
  10^5 sweeps with waiting times and lags 0, 1, 2, 4, ..., 65536: every integer
  observable at every scheduled time (the sums behind C(t, t_w) of Eq. 7, q of
  Eq. 2, C4 of Eq. 3 and the energy of Eq. 1) and the final spins, bit for bit.
* The side-128 benchmark batch (five jobs of 16 samples, autotuned launch shape and
  graph replay), aged to t = 10^4 and beyond, where the lattice has coarsened and
  the rare path is taken at its late-time rate: the spins of the first and the last
  sample at t = 4096, 10000 and 10003; and the heat-bath rule on the first job.

The expected values are SHA-256 digests written by tests/golden/make_long_runs.py,
which runs the oracle alone (about 11 core-hours); no value comes from the GPU.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle as ora
from paper_1411_5512_gb300 import workloads

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "long_runs.json")
REL = 1e-12


@pytest.fixture(scope="module")
def J():
    from paper_1411_5512_gb300 import build, job
    build.build()
    return job


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def digest(arr, dtype):
    return hashlib.sha256(np.ascontiguousarray(arr, dtype=dtype).tobytes()).hexdigest()


@pytest.mark.parametrize("k", [0, 1])
def test_side32_full_length(J, golden, k):
    rec = golden["c2"][k]
    w = workloads.SMALL[k]
    assert (rec["L"], rec["T"], rec["seed"], rec["n_samples"], rec["sweeps"]) == \
        (w["L"], w["T"], w["seed"], w["n_samples"], w["sweeps"])
    L, S = w["L"], w["n_samples"]
    j = J.EAJob(L, w["p_neg"], w["seed"], S)
    j.set_schedule(w["t_w"], w["t"])
    j.quench(w["T"])
    b = J.EABatch()
    b.add(j)
    b.autotune(trial_sweeps=8)
    b.sweep(w["sweeps"])
    b.close()
    assert j.time == w["sweeps"]
    pairs = [tuple(p) for p in rec["pairs"]]
    meas = {p: j.measure(*p) for p in pairs}
    A = np.stack([meas[p]["A"] for p in pairs])
    at_time = {}
    for p in pairs:
        at_time.setdefault(p[0] + p[1], meas[p])
    Q = np.stack([at_time[m]["Q"] for m in rec["times"]])
    E = np.stack([at_time[m]["E"] for m in rec["times"]])
    G = np.stack([meas[(a, 0)]["G"] for a in rec["tws"]])
    got = {"A": digest(A, "<i8"), "Q": digest(Q, "<i8"), "E": digest(E, "<i8"),
           "G": digest(G, "<i8")}
    for key in ("A", "Q", "E", "G"):
        if got[key] != rec["sha256"][key]:
            arr = {"A": A.sum(axis=(1, 2)), "Q": Q.sum(axis=1), "E": E.sum(axis=(1, 2)),
                   "G": G.sum(axis=(1, 2, 3))}[key]
            bad = [i for i, (x, y) in enumerate(zip(arr, rec["totals"][key])) if int(x) != y]
            pytest.fail("%s differs from the oracle; first differing entry %r" % (key, bad[:3]))
    spins = np.stack([j.all_spins(s) for s in range(S)])
    assert digest(spins, np.int8) == rec["sha256"]["spins"]
    # the FP64 values the library derives, against the oracle's formulas on the
    # integer sums just shown equal to the oracle's
    out = {"A": {p: meas[p]["A"] for p in pairs}, "Q": {m: at_time[m]["Q"] for m in rec["times"]},
           "G": {a: meas[(a, 0)]["G"] for a in rec["tws"]}}
    for p in [(0, 0), (1, 64), (256, 4096), (32768, 65536)]:
        d = ora.derived(out, L, *p)
        g = meas[p]
        assert abs(g["C"] - d["C"]) <= REL * abs(d["C"])
        assert np.allclose(g["C4"], d["C4"], rtol=REL, atol=0)
        assert np.allclose(g["C4_sem"], d["C4_sem"], rtol=REL, atol=0, equal_nan=True)
        assert g["r_cut"] == d["r_cut"]
        assert (np.isnan(g["xi1"]) and np.isnan(d["xi1"])) or \
            abs(g["xi1"] - d["xi1"]) <= REL * abs(d["xi1"])
    j.close()


def test_side128_aged_batch(J, golden):
    """The benchmark's batch, autotuned and replayed as graphs, aged past 10^4 sweeps."""
    import torch
    late = [r for r in golden["late"] if r["rule"] == 0]
    stream = torch.cuda.Stream()
    jobs = []
    for w in workloads.PAPER_SCALE:
        j = J.EAJob(w["L"], w["p_neg"], w["seed"], w["n_samples"], stream=stream)
        j.quench(w["T"])
        jobs.append(j)
    b = J.EABatch(stream=stream)
    for j in jobs:
        b.add(j)
    b.autotune(trial_sweeps=8)
    now = 0
    for m in sorted(int(k) for k in late[0]["spins_sha256"]):
        b.sweep(m - now)
        now = m
        for r in late:
            assert jobs[r["job"]].time == m
            got = digest(jobs[r["job"]].all_spins(r["sample"]), np.int8)
            assert got == r["spins_sha256"][str(m)], (r["job"], r["sample"], m)
    assert J.device_status(stream) == 0
    b.close()
    for j in jobs:
        j.close()


def test_side128_heat_bath_aged(J, golden):
    rec = [r for r in golden["late"] if r["rule"] == 1][0]
    w = workloads.PAPER_SCALE[rec["job"]]
    j = J.EAJob(w["L"], w["p_neg"], w["seed"], w["n_samples"])
    j.quench(w["T"], 1)
    b = J.EABatch()
    b.add(j)
    b.autotune(trial_sweeps=8)
    now = 0
    for m in sorted(int(k) for k in rec["spins_sha256"]):
        b.sweep(m - now)
        now = m
        assert digest(j.all_spins(rec["sample"]), np.int8) == rec["spins_sha256"][str(m)], m
    b.close()
    j.close()
