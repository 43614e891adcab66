"""Seeded synthetic workloads of the ageing study (no simulation arithmetic here).

The paper's workload is itself synthetic: i.i.d. bimodal couplings and uniform
random starts on L^3 periodic lattices (Sec. II), T = 0.8, p in [0.5, 1] (the
fraction of positive bonds), L up to 128, two replicas per sample, measurement
at logarithmically spaced waiting times (Sec. IV).  The configurations below
restate those shapes; p_neg is the fraction of NEGATIVE bonds (1 - p).
"""
import math

import numpy as np


def pow2_times(n_max, include_zero=True):
    """0, 1, 2, 4, ... up to n_max (logarithmically spaced times)."""
    out = [0] if include_zero else []
    k = 1
    while k <= n_max:
        out.append(k)
        k *= 2
    return out


# one 3D +-J sample of side 16, 1000 sweeps, C(t, t_w) at t_w = 2^k
TINY = dict(name="L16_S1_T0.7", L=16, p_neg=0.5, T=0.7, n_samples=1, seed=1, sweeps=1000,
            t_w=pow2_times(512), t=pow2_times(512))

# side 32, 64 samples, T in {0.6, 0.8}, 10^5 sweeps
SMALL = [dict(name="L32_S64_T%.1f" % T, L=32, p_neg=0.5, T=T, n_samples=64, seed=s,
              sweeps=100_000, t_w=pow2_times(65536), t=pow2_times(65536))
         for s, T in ((1, 0.6), (2, 0.8))]

# paper scale: side 128, p_neg in {0.5 .. 0.1}, 16 samples each, T = 0.7, 10^6 sweeps
PAPER_SCALE = [dict(name="L128_S16_p%.1f" % p, L=128, p_neg=p, T=0.7, n_samples=16,
                    seed=100 + k, sweeps=1_000_000, t_w=pow2_times(2 ** 19),
                    t=pow2_times(2 ** 19))
               for k, p in enumerate((0.5, 0.4, 0.3, 0.2, 0.1))]

# mixed-L batch: L in {24, 48, 64, 96, 128} with 256/64/32/8/4 samples, p_neg drawn
# uniform in [0.1, 0.5] per sample (each sample its own job), T = 0.7, 10^4 sweeps
MIXED_L = dict(name="mixedL_24-128", sizes=((24, 256), (48, 64), (64, 32), (96, 8), (128, 4)),
               T=0.7, p_range=(0.1, 0.5), sweeps=10_000, seed=11)


def mixed_l_jobs(spec=MIXED_L):
    rng = np.random.default_rng(spec["seed"])
    jobs = []
    for L, n in spec["sizes"]:
        for i in range(n):
            jobs.append(dict(L=L, p_neg=float(rng.uniform(*spec["p_range"])), T=spec["T"],
                             n_samples=1, seed=int(rng.integers(1, 2 ** 63)),
                             sweeps=spec["sweeps"]))
    return jobs


# serving: Poisson arrivals (rate 50/s) of ageing jobs, L in {16, 32, 64, 128},
# p_neg in [0.1, 0.5], T in [0.5, 1.0], sweeps log-uniform in [10^3, 10^6]
SERVING = dict(name="serve_poisson50", rate=50.0, sizes=(16, 32, 64, 128), p_range=(0.1, 0.5),
               T_range=(0.5, 1.0), sweeps_range=(1e3, 1e6), seed=7)


def serving_stream(n_jobs, spec=SERVING, max_sweeps=None):
    rng = np.random.default_rng(spec["seed"])
    t = 0.0
    jobs = []
    lo, hi = math.log(spec["sweeps_range"][0]), math.log(spec["sweeps_range"][1])
    for j in range(n_jobs):
        t += float(rng.exponential(1.0 / spec["rate"]))
        sweeps = int(round(math.exp(rng.uniform(lo, hi))))
        if max_sweeps is not None:
            sweeps = min(sweeps, max_sweeps)
        jobs.append(dict(arrival=t, L=int(rng.choice(spec["sizes"])),
                         p_neg=float(rng.uniform(*spec["p_range"])),
                         T=float(rng.uniform(*spec["T_range"])), n_samples=1,
                         seed=int(rng.integers(1, 2 ** 63)), sweeps=sweeps))
    return jobs
