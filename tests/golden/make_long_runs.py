"""Write tests/golden/long_runs.json: digests of full-length runs of the CPU oracle.

Only the oracle runs here (the plain C chain and its numpy observables); nothing of
the CUDA library is imported.  Two sets of runs, each from t = 0:

* the side-32 workload of 64 samples x 2 replicas, p_neg = 0.5, T = 0.6 (seed 1)
  and T = 0.8 (seed 2), 10^5 sweeps, waiting times and lags 0, 1, 2, 4, ..., 65536
  (the configuration "L=32, 64 disorder samples, T in {0.6, 0.8}, 10^5 sweeps");
* late times of the side-128 benchmark jobs (T = 0.7): sample 0 of the
  p_neg = 0.5 job and sample 15 of the p_neg = 0.1 job under the Metropolis rule,
  and sample 0 of the p_neg = 0.5 job under the heat-bath rule, with the spins
  recorded at t = 4096, 10000 and 10003.

Each integer observable is stored as the SHA-256 of its int64 array (little
endian, C order) and each spin state as the SHA-256 of its int8 array
[sample][replica][z][y][x], with plain totals beside them to read a mismatch by.

    python tests/golden/make_long_runs.py [--workers 7]

About 11 core-hours of oracle time; the runs go to a process pool (spawn).
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "long_runs.json")

LATE_TIMES = (4096, 10000, 10003)
# (job index in the side-128 workload list, sample, rule)
LATE_CASES = ((0, 0, 0), (4, 15, 0), (0, 0, 1))


def digest(arr, dtype):
    return hashlib.sha256(np.ascontiguousarray(arr, dtype=dtype).tobytes()).hexdigest()


def _c2_sample(args):
    k, s = args
    sys.path.insert(0, ROOT)
    import oracle as ora
    from paper_1411_5512_gb300 import workloads

    w = workloads.SMALL[k]
    out = ora.run_job(w["L"], w["p_neg"], w["seed"], w["n_samples"], w["T"], 0, w["t_w"],
                      w["t"], w["sweeps"], samples=[s], keep_spins=True)
    return ("c2", k, s, out)


def _late_sample(args):
    job, s, rule = args
    sys.path.insert(0, ROOT)
    import oracle as ora
    from paper_1411_5512_gb300 import workloads

    w = workloads.PAPER_SCALE[job]
    L = w["L"]
    J = ora.init_couplings(L, w["p_neg"], w["seed"], s)
    S = ora.init_spins(L, w["seed"], s)
    states = {}
    now = 0
    for m in LATE_TIMES:
        ora.sweeps(L, w["seed"], s, S, J, w["T"], rule, now, m - now)
        now = m
        states[m] = digest(S, np.int8)
    return ("late", job, s, rule, states)


def c2_record(k, per_sample):
    """Digests of one side-32 job from its samples' run_job results, in sample order."""
    from paper_1411_5512_gb300 import workloads

    w = workloads.SMALL[k]
    outs = [per_sample[s] for s in range(w["n_samples"])]
    pairs = sorted(outs[0]["A"].keys())
    times = sorted(outs[0]["Q"].keys())
    tws = sorted(outs[0]["G"].keys())
    A = np.stack([np.concatenate([o["A"][p] for o in outs]) for p in pairs])   # [pair][S][2]
    Q = np.stack([np.concatenate([o["Q"][m] for o in outs]) for m in times])   # [time][S]
    E = np.stack([np.concatenate([o["E"][m] for o in outs]) for m in times])   # [time][S][2]
    G = np.stack([np.concatenate([o["G"][a] for o in outs]) for a in tws])     # [t_w][S][3][R]
    spins = np.concatenate([o["spins"] for o in outs])                         # [S][2][L][L][L]
    return {"name": w["name"], "L": w["L"], "p_neg": w["p_neg"], "T": w["T"],
            "seed": w["seed"], "n_samples": w["n_samples"], "sweeps": w["sweeps"],
            "t_w": w["t_w"], "t": w["t"],
            "pairs": [list(p) for p in pairs], "times": times, "tws": tws,
            "sha256": {"A": digest(A, "<i8"), "Q": digest(Q, "<i8"), "E": digest(E, "<i8"),
                       "G": digest(G, "<i8"), "spins": digest(spins, np.int8)},
            "totals": {"A": [int(x) for x in A.sum(axis=(1, 2))],
                       "Q": [int(x) for x in Q.sum(axis=1)],
                       "E": [int(x) for x in E.sum(axis=(1, 2))],
                       "G": [int(x) for x in G.sum(axis=(1, 2, 3))]}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    args = ap.parse_args()
    sys.path.insert(0, ROOT)
    import oracle as ora
    from paper_1411_5512_gb300 import workloads

    ora.lib()  # build once before the workers start
    tasks = [(_late_sample, c) for c in LATE_CASES]
    tasks += [(_c2_sample, (k, s)) for k in range(len(workloads.SMALL))
              for s in range(workloads.SMALL[k]["n_samples"])]
    t0 = time.time()
    c2 = {k: {} for k in range(len(workloads.SMALL))}
    late = []
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.workers) as pool:
        results = [pool.apply_async(fn, (a,)) for fn, a in tasks]
        for n, r in enumerate(results):
            res = r.get()
            if res[0] == "c2":
                c2[res[1]][res[2]] = res[3]
            else:
                _, job, s, rule, states = res
                w = workloads.PAPER_SCALE[job]
                late.append({"job": job, "name": w["name"], "L": w["L"], "p_neg": w["p_neg"],
                             "T": w["T"], "seed": w["seed"], "n_samples": w["n_samples"],
                             "sample": s, "rule": rule,
                             "spins_sha256": {str(m): d for m, d in states.items()}})
            print("%d/%d done after %.0f s" % (n + 1, len(tasks), time.time() - t0), flush=True)
    rec = {"what": "digests of full-length oracle runs (see make_long_runs.py)",
           "digest": "sha256 of int64 little-endian (observables) or int8 (spins) arrays, "
                     "C order",
           "c2": [c2_record(k, c2[k]) for k in sorted(c2)],
           "late": late}
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
