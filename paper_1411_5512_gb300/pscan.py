"""A reduced scan over the bond concentration (Sec. IV).

  python -m paper_1411_5512_gb300.pscan [--L 128] [--samples 16] [--T 0.8]
                                        [--log2-sweeps 20] [--pneg 0.5,0.4,...]
                                        [--out scan.npz]

All values of p_neg run together in one batch: quench from a random start, then
sweeps up to 2^log2_sweeps with the observables measured at t_w = 2^k and lags
t = 2^j.  For each p_neg the host analysis (analysis.py) extracts, from the
measured curves:
- alpha, beta and xi(t_w) by the C4 multifit over t_w >= 10;
- xi_1(t_w) with the fitted tail;
- z from both xi series;
- x from C(t, t_w) on t in [100, t_w / 1000].
- the error bars of alpha and beta as Sec. IV makes them: the multifit on the
  axis points against the multifit on every displacement vector with
  3 <= r <= L/2 (ea_c4_radial), their difference plus both statistical errors.
The paper's p is 1 - p_neg.  The table is printed, and the raw curves are
written to --out.
"""
import argparse
import json
import sys

import numpy as np


def run(L, samples, T, log2_sweeps, pnegs, seed0=300):
    import torch

    from . import job

    total = 1 << log2_sweeps
    t_w = [0] + [1 << k for k in range(0, log2_sweeps)]
    lags = [0] + [1 << k for k in range(0, log2_sweeps)]
    stream = torch.cuda.Stream()
    jobs = []
    for i, p in enumerate(pnegs):
        j = job.EAJob(L, p, seed0 + i, samples, stream=stream)
        j.set_schedule(t_w, lags)
        j.quench(T)
        jobs.append(j)
    b = job.EABatch(stream=stream)
    for j in jobs:
        b.add(j)
    b.autotune(trial_sweeps=8)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        start.record()
        b.sweep(total)
        end.record()
    stream.synchronize()
    seconds = start.elapsed_time(end) / 1e3
    out = {"L": L, "samples": samples, "T": T, "sweeps": total, "pneg": list(pnegs),
           "seconds": seconds, "flips": 2.0 * total * samples * L ** 3 * len(pnegs)}
    curves = []
    for p, j in zip(pnegs, jobs):
        c4 = {}
        c4_all = {}
        C = {}
        for tw in t_w:
            m = j.measure(tw, 0)
            c4[tw] = (m["C4"], m["C4_sem"], m["r_cut"])
            if tw >= 10:
                rad = j.c4_radial(tw)
                keep = rad["r"] <= L // 2
                c4_all[tw] = (rad["r"][keep], rad["C4"][keep], rad["C4_sem"][keep])
            for lag in lags:
                if tw + lag <= total and lag > 0 and tw > 0:
                    C[(tw, lag)] = j.measure(tw, lag)["C"]
        curves.append({"pneg": p, "c4": c4, "c4_all": c4_all, "C": C})
    b.close()
    for j in jobs:
        j.close()
    return out, curves


def analyse(L, curves, tw_min=10):
    """Per p_neg: alpha, beta, z from the fitted xi and from xi_1 with tail, and x."""
    from . import analysis as an

    r = np.arange(0, L // 2 + 1, dtype=np.float64)
    rows = []
    for cur in curves:
        tws = sorted(tw for tw in cur["c4"] if tw >= tw_min)
        try:
            fit = an.multifit_c4([(r, cur["c4"][tw][0], cur["c4"][tw][1]) for tw in tws],
                                 r_min=3)
        except (ValueError, RuntimeError, np.linalg.LinAlgError):
            rows.append({"pneg": cur["pneg"], "p": 1.0 - cur["pneg"], "alpha": np.nan,
                         "beta": np.nan, "z_fit": np.nan, "z_int": np.nan, "x": np.nan,
                         "xi_fit_last": np.nan, "xi_int_last": np.nan, "chi2_dof": np.nan,
                         "alpha_err": np.nan, "beta_err": np.nan})
            continue
        # the error bars of Sec. IV from the axis points and every displacement vector
        a_err = b_err = np.nan
        if all(tw in cur.get("c4_all", {}) for tw in tws):
            try:
                e = an.multifit_error([(r, cur["c4"][tw][0], cur["c4"][tw][1]) for tw in tws],
                                      [cur["c4_all"][tw] for tw in tws], r_min=3)
                a_err, b_err = e["alpha_err"], e["beta_err"]
            except (ValueError, RuntimeError, np.linalg.LinAlgError):
                pass
        xi_fit = fit["xi"]
        xi_int = []
        for k, tw in enumerate(tws):
            c4, sem, r_c = cur["c4"][tw]
            xi_int.append(an.xi1_with_tail(r, c4, r_c, L,
                                           (fit["A"][k], fit["alpha"], xi_fit[k], fit["beta"])))
        xi_int = np.array(xi_int)
        zf = zi = np.nan
        try:
            zf = an.fit_z(np.array(tws, dtype=np.float64), xi_fit)["z"]
            zi = an.fit_z(np.array(tws, dtype=np.float64), xi_int)["z"]
        except (ValueError, RuntimeError):
            pass
        Cc = []
        for tw in sorted({tw for tw, _ in cur["C"]}):
            lags = sorted(lag for t2, lag in cur["C"] if t2 == tw)
            Cc.append((tw, np.array(lags, dtype=np.float64),
                       np.array([cur["C"][(tw, lag)] for lag in lags])))
        x = an.fit_x_mean(Cc)
        rows.append({"pneg": cur["pneg"], "p": 1.0 - cur["pneg"], "alpha": fit["alpha"],
                     "beta": fit["beta"], "z_fit": zf, "z_int": zi, "x": x,
                     "xi_fit_last": float(xi_fit[-1]), "xi_int_last": float(xi_int[-1]),
                     "chi2_dof": fit["chi2_dof"], "alpha_err": a_err, "beta_err": b_err})
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=128)
    ap.add_argument("--samples", type=int, default=16)
    ap.add_argument("--T", type=float, default=0.8)
    ap.add_argument("--log2-sweeps", type=int, default=20)
    ap.add_argument("--pneg", default="0.5,0.4,0.3,0.25,0.2,0.15,0.1,0.05,0.0")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    pnegs = [float(v) for v in a.pneg.split(",")]
    meta, curves = run(a.L, a.samples, a.T, a.log2_sweeps, pnegs)
    rows = analyse(a.L, curves)
    print(json.dumps({**meta, "flips_per_ns": meta["flips"] / (meta["seconds"] * 1e9)}))
    print("| p | p_neg | alpha | beta | z (fit) | z (xi_1) | x | xi(t_w max), fit / xi_1 |")
    print("|---|---|---|---|---|---|---|---|")
    for row in rows:
        print("| %.2f | %.2f | %.3f(%.3f) | %.3f(%.3f) | %.2f | %.2f | %.4f | %.1f / %.1f |" % (
            row["p"], row["pneg"], row["alpha"], row["alpha_err"], row["beta"], row["beta_err"],
            row["z_fit"], row["z_int"], row["x"], row["xi_fit_last"], row["xi_int_last"]))
    if a.out:
        flat = {}
        for cur in curves:
            key = "p%.2f" % cur["pneg"]
            for tw, (c4, sem, r_c) in cur["c4"].items():
                flat["%s_c4_%d" % (key, tw)] = np.asarray(c4)
                flat["%s_sem_%d" % (key, tw)] = np.asarray(sem)
                flat["%s_rc_%d" % (key, tw)] = np.asarray([r_c])
            for (tw, lag), v in cur["C"].items():
                flat["%s_C_%d_%d" % (key, tw, lag)] = np.asarray([v])
        np.savez(a.out, meta=json.dumps(meta), **flat)
    return 0


if __name__ == "__main__":
    sys.exit(main())
