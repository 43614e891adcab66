"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these tests compares the oracle with itself: they check published
known-answer vectors, closed forms, exact Boltzmann enumeration, limits
(T = 0, T = infinity), exact invariants (gauge covariance, energy bookkeeping)
and brute-force loops on tiny lattices.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle as ora

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------------
# Philox4x32-10: published known-answer vectors
# ----------------------------------------------------------------------------------
def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([int(v, 16) for v in line.split()])
    return rows


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for r in rows:
        out = ora.philox4x32_10(r[0:4], r[4:6])
        assert [int(v) for v in out] == r[6:10]


# ----------------------------------------------------------------------------------
# geometry of the random-number mapping
# ----------------------------------------------------------------------------------
def _geometry_table():
    tab = {}
    with open(os.path.join(GOLDEN, "geometry_lanes.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                L, kx, ky, kz = (int(v) for v in line.split())
                tab[L] = (kx, ky, kz)
    return tab


def test_geometry_table():
    for L, k in _geometry_table().items():
        g = ora.geometry(L)
        assert g[:3] == k
        assert g[3:] == (L // k[0], L // k[1], L // k[2])


@pytest.mark.parametrize("L", [2, 4, 6, 8, 12, 16, 24])
def test_geometry_bijection_and_colour(L):
    kx, ky, kz, Lx, Ly, Lz = ora.geometry(L)
    lanes = kx * ky * kz
    seen = {}
    for z, y, x in itertools.product(range(L), repeat=3):
        w, b = ora.site_to_word(L, x, y, z)
        assert 0 <= w < Lx * Ly * Lz and 0 <= b < lanes
        assert (w, b) not in seen
        seen[(w, b)] = (x, y, z)
    assert len(seen) == L ** 3
    # every site of a word-site has the same checkerboard colour
    colours = {}
    for (w, b), (x, y, z) in seen.items():
        colours.setdefault(w, set()).add((x + y + z) & 1)
    assert all(len(c) == 1 for c in colours.values())


def test_geometry_rejects_bad_sizes():
    for L in [0, 1, 3, 7, 1025, -2]:
        with pytest.raises(ValueError):
            ora.geometry(L)


# ----------------------------------------------------------------------------------
# acceptance thresholds (Eq. 9 and the heat-bath rule)
# ----------------------------------------------------------------------------------
TWO64 = 2.0 ** 64


def test_metropolis_thresholds_closed_form_limits():
    thr, alw = ora.thresholds(0.7, 0)
    # dE = -12..0 always accepted, dE > 0 not
    assert list(alw) == [1, 1, 1, 1, 0, 0, 0]
    # exact values at T = 4/ln 2: exp(-4/T) = 1/2, so dE = 4, 8, 12 give 2^63, 2^62, 2^61
    T = 4.0 / math.log(2.0)
    thr, alw = ora.thresholds(T, 0)
    for k, e in [(4, 63), (5, 62), (6, 61)]:
        assert abs(int(thr[k]) - 2 ** e) <= 2 ** (e - 48)
    # T = 0: no uphill move; T = infinity: every move
    thr, alw = ora.thresholds(0.0, 0)
    assert list(alw) == [1, 1, 1, 1, 0, 0, 0] and list(thr[4:]) == [0, 0, 0]
    thr, alw = ora.thresholds(float("inf"), 0)
    assert list(alw) == [1] * 7


def test_thresholds_sign_and_scale():
    # the probability falls with dE and with 1/T; at T = 1, dE = 4: e^-4
    thr, _ = ora.thresholds(1.0, 0)
    assert abs(int(thr[4]) / TWO64 - math.exp(-4.0)) < 1e-15
    assert abs(int(thr[6]) / TWO64 - math.exp(-12.0)) < 1e-15
    assert int(thr[4]) > int(thr[5]) > int(thr[6]) > 0
    # T = 0.5, dE = 12 has probability e^-24 ~ 3.8e-11, below 2^-32, still positive
    thr, _ = ora.thresholds(0.5, 0)
    # floor() loses less than one unit of 2^-64
    assert int(thr[6]) > 0 and abs(int(thr[6]) - math.ldexp(math.exp(-24.0), 64)) <= 1.0


def test_heatbath_thresholds():
    thr, alw = ora.thresholds(1.3, 1)
    assert not any(alw)
    assert int(thr[3]) == 2 ** 63  # dE = 0: probability 1/2 exactly
    for k in range(7):
        # p(dE) + p(-dE) = 1
        assert abs(int(thr[k]) + int(thr[6 - k]) - 2 ** 64) <= 2 ** 12
    assert abs(int(thr[4]) / TWO64 - 1.0 / (1.0 + math.exp(4.0 / 1.3))) < 1e-15
    thr, alw = ora.thresholds(0.0, 1)
    assert list(alw) == [1, 1, 1, 0, 0, 0, 0] and int(thr[3]) == 2 ** 63
    assert list(thr[4:]) == [0, 0, 0]
    thr, alw = ora.thresholds(float("inf"), 1)
    assert all(int(v) == 2 ** 63 for v in thr)


def test_thresholds_reject_bad_args():
    for T, rule in [(-1.0, 0), (float("nan"), 0), (1.0, 2)]:
        with pytest.raises(ValueError):
            ora.thresholds(T, rule)


# ----------------------------------------------------------------------------------
# random numbers and initial state
# ----------------------------------------------------------------------------------
def test_couplings_bimodal_fraction():
    L = 16
    assert np.all(ora.init_couplings(L, 0.0, 5, 0) == 1)
    assert np.all(ora.init_couplings(L, 1.0, 5, 0) == -1)
    J = ora.init_couplings(L, 0.3, 5, 1)
    n = J.size
    frac = float(np.mean(J == -1))
    assert abs(frac - 0.3) < 5 * math.sqrt(0.3 * 0.7 / n)
    assert set(np.unique(J)) == {-1, 1}
    # different samples get different disorder
    assert np.any(ora.init_couplings(L, 0.5, 5, 0) != ora.init_couplings(L, 0.5, 5, 1))


def test_spins_uniform_start():
    S = ora.init_spins(16, 9, 0)
    n = S.size
    assert abs(float(np.mean(S == -1)) - 0.5) < 5 * math.sqrt(0.25 / n)
    assert np.any(S[0] != S[1])  # the replicas start from different states


# ----------------------------------------------------------------------------------
# exact enumeration of the Boltzmann distribution at L = 2
# ----------------------------------------------------------------------------------
def _energy_table_L2(J):
    """Energy of all 256 states of the 2^3 lattice; state bit i = site i is -1."""
    E = np.zeros(256)
    for st in range(256):
        s = np.array([-1 if (st >> i) & 1 else 1 for i in range(8)], dtype=np.int8)
        S = np.stack([s.reshape(2, 2, 2), s.reshape(2, 2, 2)])
        E[st] = ora.energy(S, J)[0]
    return E


def _state_index(S_a):
    flat = S_a.reshape(-1)
    return int(sum(1 << i for i in range(8) if flat[i] == -1))


def _chain_histogram(J, T, rule, seed, n_sweeps, burn=200):
    L = 2
    S = ora.init_spins(L, seed, 0)
    hist = np.zeros(256)
    ora.sweeps(L, seed, 0, S, J, T, rule, 0, burn)
    for t in range(burn, burn + n_sweeps):
        ora.sweeps(L, seed, 0, S, J, T, rule, t, 1)
        hist[_state_index(S[0])] += 1
        hist[_state_index(S[1])] += 1
    return hist


def _chi2(hist, E, T):
    """chi2 of the histogram against exp(-E/T)/Z, each state folded with its global
    flip (H(S) = H(-S) for every J).  Folding removes the slow tunnelling between
    the two halves of state space of an ordered lattice, which would otherwise
    dominate the statistic, and keeps every energy level."""
    w = np.exp(-(E - E.min()) / T)
    p = w / w.sum()
    flip = 255 - np.arange(256)
    hf = (hist + hist[flip])[:128]
    pf = (p + p[flip])[:128]
    exp_ = hist.sum() * pf
    return float(np.sum((hf - exp_) ** 2 / exp_))


@pytest.mark.parametrize("p_neg,T,rule,seed", [(0.0, 3.0, 0, 1), (0.5, 2.0, 0, 2),
                                               (0.5, 2.0, 1, 3), (0.25, 2.5, 0, 4)])
def test_L2_chain_samples_boltzmann(p_neg, T, rule, seed):
    J = ora.init_couplings(2, p_neg, 100 + seed, 0)
    E = _energy_table_L2(J)
    hist = _chain_histogram(J, T, rule, seed, 60000)
    chi2 = _chi2(hist, E, T)
    dof = 127
    # samples are correlated in time (chi2/dof falls towards 1 as the run grows,
    # where a biased chain would make it grow); a 2x allowance is still far below
    # the value for a wrong temperature or a wrong sign of dE
    assert chi2 / dof < 2.0, chi2 / dof
    assert _chi2(hist, E, 0.7 * T) / dof > 6.0
    assert _chi2(hist, -E, T) / dof > 6.0


# ----------------------------------------------------------------------------------
# limits and invariants of the dynamics
# ----------------------------------------------------------------------------------
def test_infinite_temperature_flips_every_spin_every_sweep():
    L = 6
    J = ora.init_couplings(L, 0.5, 3, 0)
    S0 = ora.init_spins(L, 3, 0)
    S = S0.copy()
    E0 = ora.energy(S0, J)
    for t in range(5):
        ora.sweeps(L, 3, 0, S, J, float("inf"), 0, t, 1)
        assert np.array_equal(S, S0 if t % 2 else -S0)
        # C(t_w, t) = (-1)^t exactly and E(t) = E(0)
        assert np.all(ora.autocorr_sum(S0, S) == (-1) ** (t + 1) * L ** 3)
        assert np.array_equal(ora.energy(S, J), E0)


def test_zero_temperature_ferromagnet():
    L = 8
    J = ora.init_couplings(L, 0.0, 4, 0)
    # the all-up state is absorbing
    S = np.ones((2, L, L, L), dtype=np.int8)
    ora.sweeps(L, 4, 0, S, J, 0.0, 0, 0, 5)
    assert np.all(S == 1)
    # from a random start the energy never rises
    S = ora.init_spins(L, 4, 0)
    prev = ora.energy(S, J)
    for t in range(30):
        ora.sweeps(L, 4, 0, S, J, 0.0, 0, t, 1)
        e = ora.energy(S, J)
        assert np.all(e <= prev)
        prev = e
    assert np.all(prev < 0)


@pytest.mark.parametrize("L,p_neg,T,rule", [(4, 0.5, 0.7, 0), (6, 0.3, 1.1, 0),
                                            (8, 0.5, 0.8, 1), (2, 0.5, 1.0, 0)])
def test_energy_bookkeeping(L, p_neg, T, rule):
    """Sum of accepted dE equals the change of the energy computed from scratch."""
    J = ora.init_couplings(L, p_neg, 21, 2)
    S = ora.init_spins(L, 21, 2)
    E0 = ora.energy(S, J)
    acc = np.zeros(2, dtype=np.int64)
    for t in range(0, 40, 5):
        acc += ora.sweeps(L, 21, 2, S, J, T, rule, t, 5)
        assert np.array_equal(ora.energy(S, J) - E0, acc)


@pytest.mark.parametrize("L,rule", [(4, 0), (6, 0), (8, 1), (12, 0)])
def test_gauge_covariance(L, rule):
    """J'_ij = e_i e_j J_ij and S'(0) = e S(0) give S'(t) = e S(t) with the same randoms."""
    rng = np.random.default_rng(L)
    eps = rng.choice(np.array([-1, 1], dtype=np.int8), size=(L, L, L))
    J = ora.init_couplings(L, 0.5, 77, 1)
    S = ora.init_spins(L, 77, 1)
    Jg = np.empty_like(J)
    for d, ax in ((0, 2), (1, 1), (2, 0)):
        Jg[d] = J[d] * eps * np.roll(eps, -1, axis=ax)
    Sg = (S * eps[None]).astype(np.int8)
    ora.sweeps(L, 77, 1, S, J, 0.8, rule, 0, 12)
    ora.sweeps(L, 77, 1, Sg, Jg, 0.8, rule, 0, 12)
    assert np.array_equal(Sg, S * eps[None])
    assert ora.overlap_sum(Sg) == ora.overlap_sum(S)
    assert np.array_equal(ora.c4_sums(Sg), ora.c4_sums(S))
    assert np.array_equal(ora.energy(Sg, Jg), ora.energy(S, J))


def test_mattis_disorder_is_a_ferromagnet():
    """J_ij = e_i e_j has an unfrustrated ground state S = e with E = -3N."""
    L = 6
    eps = np.random.default_rng(3).choice(np.array([-1, 1], dtype=np.int8), size=(L, L, L))
    J = np.empty((3, L, L, L), dtype=np.int8)
    for d, ax in ((0, 2), (1, 1), (2, 0)):
        J[d] = eps * np.roll(eps, -1, axis=ax)
    S = np.stack([eps, eps]).astype(np.int8)
    assert np.all(ora.energy(S, J) == -3 * L ** 3)
    ora.sweeps(L, 1, 0, S, J, 0.0, 0, 0, 4)
    assert np.array_equal(S[0], eps) and np.array_equal(S[1], eps)


def test_acceptance_rate_matches_threshold():
    """At T = infinity for heat bath every move has probability 1/2."""
    L = 16
    J = ora.init_couplings(L, 0.5, 8, 0)
    S = ora.init_spins(L, 8, 0)
    S0 = S.copy()
    ora.sweeps(L, 8, 0, S, J, float("inf"), 1, 0, 1)
    n = S.size
    frac = float(np.mean(S != S0))
    assert abs(frac - 0.5) < 5 * math.sqrt(0.25 / n)


# ----------------------------------------------------------------------------------
# observables: brute-force loops on tiny lattices
# ----------------------------------------------------------------------------------
def _brute(S, J):
    L = S.shape[1]
    N = L ** 3
    Q = 0
    G = np.zeros((3, L), dtype=np.int64)
    E = [0, 0]
    for z in range(L):
        for y in range(L):
            for x in range(L):
                q = int(S[0, z, y, x]) * int(S[1, z, y, x])
                Q += q
                for r in range(L):
                    G[0, r] += q * int(S[0, z, y, (x + r) % L]) * int(S[1, z, y, (x + r) % L])
                    G[1, r] += q * int(S[0, z, (y + r) % L, x]) * int(S[1, z, (y + r) % L, x])
                    G[2, r] += q * int(S[0, (z + r) % L, y, x]) * int(S[1, (z + r) % L, y, x])
                for a in range(2):
                    s = int(S[a, z, y, x])
                    E[a] -= int(J[0, z, y, x]) * s * int(S[a, z, y, (x + 1) % L])
                    E[a] -= int(J[1, z, y, x]) * s * int(S[a, z, (y + 1) % L, x])
                    E[a] -= int(J[2, z, y, x]) * s * int(S[a, (z + 1) % L, y, x])
    return Q, G, E, N


@pytest.mark.parametrize("L", [2, 4, 6])
def test_observables_brute_force(L):
    J = ora.init_couplings(L, 0.4, 31, 0)
    S = ora.init_spins(L, 31, 0)
    ora.sweeps(L, 31, 0, S, J, 0.9, 0, 0, 3)
    Q, G, E, N = _brute(S, J)
    assert ora.overlap_sum(S) == Q
    assert np.array_equal(ora.c4_sums(S), G[:, : L // 2 + 1])
    assert list(ora.energy(S, J)) == E
    # C4(0) = 1 and the periodic symmetry C4(r) = C4(L - r)
    assert np.all(G[:, 0] == N)
    for r in range(1, L):
        assert np.array_equal(G[:, r], G[:, L - r])
    # C(t_w, t_w) = 1
    assert np.all(ora.autocorr_sum(S, S) == N)


def test_run_job_schedule():
    out = ora.run_job(4, 0.5, 5, 2, 0.7, 0, t_w=[0, 2], t=[0, 1, 3], n_sweeps=5)
    N = 64
    assert set(out["A"]) == {(0, 0), (0, 1), (0, 3), (2, 0), (2, 1), (2, 3)}
    assert np.all(out["A"][(0, 0)] == N) and np.all(out["A"][(2, 0)] == N)
    assert set(out["G"]) == {0, 2}
    assert sorted(out["Q"]) == [0, 1, 2, 3, 5]
    for tw in (0, 2):
        assert np.all(out["G"][tw][:, :, 0] == N)
    # energy bookkeeping across the whole run
    E5 = out["E"][5]
    E0 = out["E"][0]
    assert np.array_equal(E5 - E0, out["dE"])


# ----------------------------------------------------------------------------------
# FP64 derived quantities (Eqs. 5-6)
# ----------------------------------------------------------------------------------
def test_xi1_closed_forms():
    for n in (4, 8, 64):
        c4 = np.full(n + 1, 0.37)
        assert ora.xi1(c4, n) == pytest.approx((2 * n + 1) / 3.0, rel=1e-14)
    # a cut at r_c = 4 keeps r = 1..4: sum r^2 / sum r = 30 / 10
    assert ora.xi1(np.full(9, 1.0), 4) == pytest.approx(3.0, rel=1e-15)
    assert math.isnan(ora.xi1(np.zeros(9), 8))
    assert math.isnan(ora.xi1(np.full(9, 1.0), 0))


def test_cutoff_rule():
    c4 = np.array([1.0, 0.5, 0.3, 0.1, 0.02, 0.01])
    sem = np.array([0.0, 0.01, 0.01, 0.01, 0.01, 0.01])
    assert ora.cutoff(c4, sem) == 3  # first r with C4 < 3 sem is r = 4
    assert ora.cutoff(c4, np.zeros(6)) == 5
    assert ora.cutoff(c4, np.full(6, np.nan)) == 5
    assert ora.cutoff(np.array([1.0, -0.1, 0.5]), np.array([0, 0.01, 0.01])) == 0


def test_c4_curve_average_and_sem():
    N = 8
    G = np.zeros((2, 3, 2), dtype=np.int64)
    G[:, :, 0] = N
    G[0, :, 1] = [8, 4, 0]   # sample 0: mean over axes 4/8 = 0.5
    G[1, :, 1] = [0, 0, 0]   # sample 1: 0
    c4, sem = ora.c4_curve(G, N)
    assert c4[0] == 1.0 and c4[1] == 0.25
    assert sem[1] == pytest.approx(0.25, rel=1e-15)  # std([0.5, 0]) / sqrt(2)


# ----------------------------------------------------------------------------------
# Metropolis by geometric gaps (Eq. 9 decided per class of a word-site)
# ----------------------------------------------------------------------------------
def test_geo_table_closed_form():
    # p = 1/2: C[g] = 2^64 (1 - 2^-g)
    C = ora.geo_table(0.5)
    assert int(C[0]) == 0
    for g in range(1, 33):
        assert abs(int(C[g]) - (2 ** 64 - 2 ** (64 - g))) <= 2 ** 12
    # tiny p: 1 - (1-p)^g = g p - g(g-1)/2 p^2 + O(p^3); floor loses < 1 unit
    p = math.exp(-24.0)
    C = ora.geo_table(p)
    for g in (1, 2, 7, 32):
        expect = math.ldexp(g * p - g * (g - 1) / 2.0 * p * p, 64)
        assert abs(int(C[g]) - expect) <= 4.0, g
    C = ora.geo_table(0.3)
    assert all(int(C[g]) < int(C[g + 1]) for g in range(32))
    for bad in (0.0, 1.0, -0.1, float("nan")):
        with pytest.raises(ValueError):
            ora.geo_table(bad)


def _half_step_stats(L, T, n_rep, seed=5, rule=0):
    """Flip outcomes of the sites updated in half-step 0, grouped per word-site and
    dE, over n_rep independent half-steps from the same state."""
    kx, ky, kz, Lx, Ly, Lz = ora.geometry(L)
    J = ora.init_couplings(L, 0.5, seed, 0)
    S0 = ora.init_spins(L, seed, 0)
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    widx = (x % Lx) + Lx * ((y % Ly) + Ly * (z % Lz))
    lane = (x // Lx) + kx * ((y // Ly) + ky * (z // Lz))
    colour = (x + y + z) & 1
    dEs = []
    for a in range(2):
        s = S0[a].astype(np.int64)
        hloc = np.zeros_like(s)
        for d, ax in ((0, 2), (1, 1), (2, 0)):
            hloc += J[d] * np.roll(s, -1, axis=ax) + np.roll(J[d] * s, 1, axis=ax)
        dEs.append(2 * s * hloc)
    groups = {}  # (rep, a, widx, dE) -> list of (lane, flipped)
    for rep in range(n_rep):
        S = S0.copy()
        ora.half_step(L, seed, 0, S, J, T, rule, 1000 + rep, 0)
        for a in range(2):
            upd = colour == (0 ^ a)
            fl = (S[a] != S0[a]) & upd
            for dE in ((4, 8, 12) if rule == 0 else (-12, -8, -4, 0, 4, 8, 12)):
                m = upd & (dEs[a] == dE)
                for w, b, f in zip(widx[m], lane[m], fl[m]):
                    groups.setdefault((rep, a, int(w), dE), []).append((int(b), bool(f)))
            if rule == 0:  # sites with dE <= 0 always flip
                assert np.all(fl[upd & (dEs[a] <= 0)])
    return groups


def _class_checks(groups, dE, p):
    """Each site of class dE flips with probability p, at every rank within its
    word-site, and the first and last site of a class decide independently."""
    tot = acc = 0
    rank_n = np.zeros(32)
    rank_acc = np.zeros(32)
    pair_n = pair_both = 0
    for (rep, a, w, e), lst in groups.items():
        if e != dE:
            continue
        lst.sort()
        f = [x[1] for x in lst]
        tot += len(f)
        acc += sum(f)
        for j, v in enumerate(f):
            rank_n[j] += 1
            rank_acc[j] += v
        if len(f) >= 2:
            pair_n += 1
            pair_both += f[0] and f[-1]
    sig = math.sqrt(tot * p * (1 - p))
    assert abs(acc - tot * p) < 5 * sig, (dE, acc, tot * p)
    for j in range(4):  # the first ranks each accept with probability p
        if rank_n[j] > 200:
            sj = math.sqrt(rank_n[j] * p * (1 - p))
            assert abs(rank_acc[j] - rank_n[j] * p) < 5 * sj, (dE, j)
    if pair_n > 200:  # first and last site of a class decide independently
        q = p * p
        assert abs(pair_both - pair_n * q) < 5 * math.sqrt(pair_n * q * (1 - q)) + 1, dE


def test_metropolis_class_statistics():
    T = 3.0
    groups = _half_step_stats(32, T, 6)
    for dE in (4, 8, 12):
        _class_checks(groups, dE, math.exp(-dE / T))


@pytest.mark.parametrize("T", [1.5, 4.0])
def test_heatbath_class_statistics(T):
    """Every class, the gap-selected (dE > 0), the coin (dE = 0) and the
    complement-selected (dE < 0), flips with 1 / (1 + e^(dE/T))."""
    groups = _half_step_stats(32, T, 6, rule=1)
    for dE in (-12, -8, -4, 0, 4, 8, 12):
        _class_checks(groups, dE, 1.0 / (1.0 + math.exp(dE / T)))


def test_metropolis_zero_and_infinite_temperature_classes():
    # T = 0: no uphill flip; T = inf: every site flips
    L = 8
    J = ora.init_couplings(L, 0.5, 2, 0)
    S0 = ora.init_spins(L, 2, 0)
    S = S0.copy()
    E0 = ora.energy(S, J)
    ora.half_step(L, 2, 0, S, J, 0.0, 0, 0, 0)
    assert np.all(ora.energy(S, J) <= E0)
    S = S0.copy()
    ora.half_step(L, 2, 0, S, J, float("inf"), 0, 0, 0)
    colour = np.indices((L, L, L)).sum(axis=0) & 1
    assert np.array_equal(S[0][colour == 0], -S0[0][colour == 0])
    assert np.array_equal(S[0][colour == 1], S0[0][colour == 1])


def test_heatbath_zero_temperature_classes():
    """T = 0: every dE < 0 site flips, no dE > 0 site does, dE = 0 sites flip by a
    fair coin; the coin of a word-site is shared by no two sites (one bit each)."""
    L = 16
    J = ora.init_couplings(L, 0.5, 6, 0)
    S0 = ora.init_spins(L, 6, 0)
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    colour = (x + y + z) & 1
    s = S0[0].astype(np.int64)
    hloc = np.zeros_like(s)
    for d, ax in ((0, 2), (1, 1), (2, 0)):
        hloc += J[d] * np.roll(s, -1, axis=ax) + np.roll(J[d] * s, 1, axis=ax)
    dE = 2 * s * hloc
    upd = colour == 0
    zero = 0
    n_zero = 0
    for t in range(8):
        S = S0.copy()
        ora.half_step(L, 6, 0, S, J, 0.0, 1, t, 0)
        fl = S[0] != S0[0]
        assert np.all(fl[upd & (dE < 0)]) and not np.any(fl[upd & (dE > 0)])
        assert not np.any(fl[~upd])
        zero += int(np.sum(fl[upd & (dE == 0)]))
        n_zero += int(np.sum(upd & (dE == 0)))
    assert n_zero > 1000
    assert abs(zero - n_zero / 2) < 5 * math.sqrt(n_zero / 4)


# ----------------------------------------------------------------------------------
# four-point sums over every displacement vector
# ----------------------------------------------------------------------------------
def _loop_full(S):
    """Pure-Python loops over sites and vectors with explicit periodic indices."""
    L = S.shape[1]
    q = [[[int(S[0, z, y, x]) * int(S[1, z, y, x]) for x in range(L)] for y in range(L)]
         for z in range(L)]
    G = np.zeros((L, L, L), dtype=np.int64)
    for dz in range(L):
        for dy in range(L):
            for dx in range(L):
                tot = 0
                for z in range(L):
                    for y in range(L):
                        for x in range(L):
                            tot += q[z][y][x] * q[(z + dz) % L][(y + dy) % L][(x + dx) % L]
                G[dz, dy, dx] = tot
    return G


@pytest.mark.parametrize("L", [2, 4])
def test_c4_full_brute_force(L):
    S = ora.init_spins(L, 40 + L, 0)
    assert np.array_equal(ora.c4_full_sums(S), _loop_full(S))


@pytest.mark.parametrize("L", [6, 8, 12])
def test_c4_full_identities(L):
    S = ora.init_spins(L, 50 + L, 1)
    J = ora.init_couplings(L, 0.5, 50 + L, 1)
    ora.sweeps(L, 50 + L, 1, S, J, 0.8, 0, 0, 3)
    G = ora.c4_full_sums(S)
    N = L ** 3
    q = S[0].astype(np.int64) * S[1]
    assert G[0, 0, 0] == N
    assert int(G.sum()) == int(q.sum()) ** 2  # sum over vectors = (sum_i q_i)^2
    # G(v) = G(-v)
    assert np.array_equal(G, np.roll(G[::-1, ::-1, ::-1], 1, axis=(0, 1, 2)))
    # the axis points are the axis sums
    ax = ora.c4_sums(S)
    r = np.arange(L // 2 + 1)
    assert np.array_equal(G[0, 0, r], ax[0]) and np.array_equal(G[0, r, 0], ax[1])
    assert np.array_equal(G[r, 0, 0], ax[2])
    # the correlation theorem with numpy's FFT, rounded
    F = np.fft.fftn(q)
    Gf = np.rint(np.fft.ifftn(F * np.conj(F)).real).astype(np.int64)
    assert np.array_equal(G, Gf)
    v = [(1, 2, 3), (L - 1, 0, 2), (L // 2, L // 2, L // 2)]
    assert np.array_equal(ora.c4_at(S, v), [G[dz, dy, dx] for dx, dy, dz in v])


@pytest.mark.parametrize("L", [4, 6, 16])
def test_radial_bins(L):
    r2 = ora.radial_index(L)
    n_bins = 3 * (L // 2) ** 2 + 1
    G = np.ones((L, L, L), dtype=np.int64)
    sums, counts = ora.c4_radial_sums(G)
    assert len(counts) == n_bins and counts.sum() == L ** 3 and np.array_equal(sums, counts)
    assert counts[0] == 1 and counts[1] == 6 and counts[n_bins - 1] == 1
    # r^2 = 2: the 12 face diagonals; r^2 = 3: the 8 body diagonals (L >= 4)
    assert counts[2] == 12 and counts[3] == 8
    assert r2[0, 0, 1] == 1 and r2[0, 0, L - 1] == 1 and r2[L // 2, L // 2, L // 2] == n_bins - 1


# ----------------------------------------------------------------------------------
# couplings with an exact count of negative bonds
# ----------------------------------------------------------------------------------
def _exact_by_sorting(L, p_neg, seed, s):
    """The K first bonds in the order of (key, bond index), with Python's sort."""
    N = L ** 3
    key = [seed & 0xFFFFFFFF, seed >> 32]
    keys = []
    for d in range(3):
        for i in range(N):
            o = ora.philox4x32_10([i, 1 + d, 0, s], key)
            keys.append(((int(o[0]) << 32) | int(o[1]), d * N + i))
    K = int(math.floor(p_neg * 3 * N + 0.5))
    J = np.ones(3 * N, dtype=np.int8)
    for _, b in sorted(keys)[:K]:
        J[b] = -1
    return J.reshape(3, L, L, L)


@pytest.mark.parametrize("L,p_neg", [(2, 0.5), (4, 0.3), (4, 0.0), (4, 1.0), (6, 0.137)])
def test_exact_couplings_count_and_order(L, p_neg):
    J = ora.init_couplings_exact(L, p_neg, 11, 2)
    N = L ** 3
    assert int(np.sum(J == -1)) == int(math.floor(p_neg * 3 * N + 0.5))
    assert np.array_equal(J, _exact_by_sorting(L, p_neg, 11, 2))


def test_exact_couplings_nested_and_sample_dependent():
    L = 8
    a = ora.init_couplings_exact(L, 0.2, 5, 0)
    b = ora.init_couplings_exact(L, 0.3, 5, 0)
    assert np.all(b[a == -1] == -1)  # the selection grows with K
    assert np.any(a != ora.init_couplings_exact(L, 0.2, 5, 1))


def test_exact_couplings_hypergeometric():
    """At L = 2 (n = 24 bonds), K = 12: every bond is negative with probability 1/2,
    and the count X in a fixed half of the bonds is hypergeometric, with variance
    12 (1/2)(1/2)(12/23) = 1.565, not the binomial 3 of independent bonds."""
    n, K, reps = 24, 12, 4000
    one = np.zeros(n)
    xs = []
    for s in range(reps):
        J = (ora.init_couplings_exact(2, 0.5, 1234, s).ravel() == -1)
        one += J
        xs.append(int(J[:12].sum()))
    p1 = K / n
    assert np.all(np.abs(one / reps - p1) < 5 * math.sqrt(p1 * (1 - p1) / reps))
    var = float(np.var(xs, ddof=1))
    expect = 12 * 0.5 * 0.5 * (n - 12) / (n - 1)
    assert abs(var - expect) < 5 * expect * math.sqrt(2.0 / reps), var
    assert abs(float(np.mean(xs)) - 6.0) < 5 * math.sqrt(expect / reps)


# ----------------------------------------------------------------------------------
# the draw contract: the joint law of the flips it produces
#
# Eq. 9 asks each site of a class to flip independently with its probability.
# The oracle spends the random bits word-site by word-site (draw64 in
# ea_oracle.c): leads shared by the four words of a quad, extension and
# continuation calls, a coin word.  Whatever the layout, the result must be
# independent fair bits in every draw and independent Bernoulli flips in every
# class, between the classes of a word-site and between the words of a quad.
# These pins hold one configuration fixed and vary only the sweep t.
# ----------------------------------------------------------------------------------
from scipy import stats  # noqa: E402

DRAW_L = 32  # word lattice 32 x 16 x 2, 32 lanes (kx, ky, kz = 1, 2, 16)
# the four word-sites of the quad (x' 0..1) x (z' 0..1) at y' = 3, with the replica
# that half-step 0 updates there (colour (x' + y' + z') mod 2 = h XOR a)
QUAD = [((0, 3, 0), 1), ((1, 3, 0), 0), ((0, 3, 1), 0), ((1, 3, 1), 1)]
DRAW_SEED, DRAW_S = 0x5EED1234ABCDEF, 3
N_SWEEPS = 10_000
METRO_CLASSES = (0, 1, 2)
HEAT_CLASSES = (0, 1, 2, 4, 5, 6)


def _draw_table(rule, n_t=1024):
    """V[(u, d)] -> uint64 array over (quad word, sweep t)."""
    classes = METRO_CLASSES if rule == 0 else HEAT_CLASSES
    out = {}
    for u in classes:
        for d in (0, 1, 2):
            v = np.zeros((len(QUAD), n_t), dtype=np.uint64)
            for k, (ws, a) in enumerate(QUAD):
                for t in range(n_t):
                    v[k, t] = ora.draw64(rule, DRAW_L, DRAW_SEED, DRAW_S, a, 7000 + t, ws, u, d)
            out[(u, d)] = v
    return out


_DRAWS = {}


def _draws(rule):
    if rule not in _DRAWS:
        _DRAWS[rule] = _draw_table(rule)
    return _DRAWS[rule]


def _bits(v):
    """[..., 64] 0/1 array of the bits of uint64 values (bit 63 first)."""
    b = np.unpackbits(v.astype(">u8").view(np.uint8).reshape(v.shape + (8,)), axis=-1)
    return b.astype(np.int64)


@pytest.mark.parametrize("rule", [0, 1])
def test_draw_bits_are_fair(rule):
    """Each of the 64 bits of every draw is a fair coin (a bit stuck, or two
    sources OR-ed into one bit, shows at once)."""
    for key, v in _draws(rule).items():
        b = _bits(v.ravel())
        n = b.shape[0]
        z = np.abs(b.sum(axis=0) - n / 2) / math.sqrt(n / 4)
        assert z.max() < 5.0, (rule, key, int(np.argmax(z)), float(z.max()))


@pytest.mark.parametrize("rule", [0, 1])
def test_draws_share_no_bits(rule):
    """Two different draws of a word-site (other class or other draw index) agree on
    each bit half of the time: no lead, extension or continuation is shared."""
    tab = _draws(rule)
    keys = sorted(tab)
    bits = {k: _bits(tab[k]) for k in keys}  # [word][t][64]
    for k1, k2 in itertools.combinations(keys, 2):
        agree = (bits[k1] == bits[k2]).reshape(-1, 64)
        n = agree.shape[0]
        z = np.abs(agree.sum(axis=0) - n / 2) / math.sqrt(n / 4)
        assert z.max() < 5.5, (rule, k1, k2, int(np.argmax(z)), float(z.max()))


def test_quad_words_share_no_bits():
    """The four words of a quad take their leads from one Philox call; each must
    get bits of its own."""
    tab = _draws(0)
    for u in METRO_CLASSES:
        b = _bits(tab[(u, 0)])  # [word][t][64]
        for w1, w2 in itertools.combinations(range(len(QUAD)), 2):
            agree = b[w1] == b[w2]
            n = agree.shape[0]
            z = np.abs(agree.sum(axis=0) - n / 2) / math.sqrt(n / 4)
            assert z.max() < 5.0, (u, w1, w2, int(np.argmax(z)), float(z.max()))


def _flip_p(rule, u, T):
    dE = 12 - 4 * u
    if rule == 0:
        return min(1.0, math.exp(-dE / T))
    return 1.0 / (1.0 + math.exp(dE / T))


def _lanes(lst):
    return sum(1 << b for b in lst)


def _patterns(masks, lane_lists):
    """Pack the flips of the listed lanes of each mask into one integer pattern per
    sweep: bit i of the pattern is lane lane_lists[...][i] (in the order given)."""
    pat = np.zeros(masks[0].shape[0], dtype=np.int64)
    i = 0
    for m, lst in zip(masks, lane_lists):
        for b in lst:
            pat |= ((m.astype(np.int64) >> b) & 1) << i
            i += 1
    return pat, i


def _chi2_product_law(pat, probs):
    """chi^2 p-value of observed patterns against independent bits, bit i set with
    probability probs[i]; cells expected below 5 are pooled."""
    n_bits = len(probs)
    n = pat.shape[0]
    obs = np.bincount(pat, minlength=1 << n_bits).astype(np.float64)
    exp = np.ones(1 << n_bits)
    for i, p in enumerate(probs):
        on = ((np.arange(1 << n_bits) >> i) & 1).astype(bool)
        exp *= np.where(on, p, 1.0 - p)
    exp *= n
    small = exp < 5.0
    o = np.append(obs[~small], obs[small].sum())
    e = np.append(exp[~small], exp[small].sum())
    if e[-1] == 0.0:
        o, e = o[:-1], e[:-1]
    assert o.sum() == n
    chi2 = float(np.sum((o - e) ** 2 / e))
    return float(stats.chi2.sf(chi2, len(e) - 1))


JOINT_LANES = [((0, 3, 0), 1, [4, 19]), ((1, 3, 1), 1, [0, 13, 31]),
               ((1, 3, 0), 0, [2, 9, 10, 22, 27])]


@pytest.mark.parametrize("rule,u", [(0, u) for u in METRO_CLASSES] +
                         [(1, u) for u in range(7)])
@pytest.mark.parametrize("T", [5.0, 12.0])
def test_class_flips_joint_law(rule, u, T):
    """Over 10^4 sweeps, the 2^n flip patterns of n = 2, 3, 5 lanes of one class
    follow the product law Bernoulli(p)^n, p = min(1, e^(-dE/T)) (Eq. 9) or
    1/(1 + e^(dE/T)) (heat bath): gap-selected (dE > 0), coin (dE = 0) and
    complement-selected (dE < 0) classes alike."""
    p = _flip_p(rule, u, T)
    for ws, a, lst in JOINT_LANES:
        m = ora.class_flips(rule, DRAW_L, T, DRAW_SEED, DRAW_S, a, 20_000, N_SWEEPS, ws, u,
                            _lanes(lst))
        assert np.all((m & ~np.uint32(_lanes(lst))) == 0)
        pat, nb = _patterns([m], [lst])
        pv = _chi2_product_law(pat, [p] * nb)
        assert pv > 1e-6, (rule, u, T, ws, lst, pv)


CROSS_PAIRS = {0: [(2, 1), (2, 0), (1, 0)],
               1: [(2, 4), (1, 5), (0, 6), (2, 1), (2, 0), (1, 0), (4, 5), (4, 6), (3, 2),
                   (3, 6)]}


@pytest.mark.parametrize("rule", [0, 1])
@pytest.mark.parametrize("T", [5.0, 12.0])
def test_classes_of_a_word_site_flip_independently(rule, T):
    """Lanes of two classes of one word-site, decided at the same sweep (their
    leads come from one Philox output), flip independently: the joint pattern
    of 3 + 3 lanes follows the product law."""
    la, lb = [1, 14, 25], [6, 18, 30]
    for ws, a, _ in JOINT_LANES[:2]:
        for ua, ub in CROSS_PAIRS[rule]:
            ma = ora.class_flips(rule, DRAW_L, T, DRAW_SEED, DRAW_S, a, 40_000, N_SWEEPS, ws,
                                 ua, _lanes(la))
            mb = ora.class_flips(rule, DRAW_L, T, DRAW_SEED, DRAW_S, a, 40_000, N_SWEEPS, ws,
                                 ub, _lanes(lb))
            pat, nb = _patterns([ma, mb], [la, lb])
            probs = [_flip_p(rule, ua, T)] * 3 + [_flip_p(rule, ub, T)] * 3
            pv = _chi2_product_law(pat, probs)
            assert pv > 1e-6, (rule, T, ws, ua, ub, pv)


@pytest.mark.parametrize("T", [5.0, 12.0])
def test_words_of_a_quad_flip_independently(T):
    """The four words of a quad share one main Philox call; the same-rank lanes of
    one class in the four words flip independently (4 x 2 lanes, product law)."""
    lst = [3, 17]
    for u in METRO_CLASSES:
        masks = [ora.class_flips(0, DRAW_L, T, DRAW_SEED, DRAW_S, a, 60_000, N_SWEEPS, ws, u,
                                 _lanes(lst)) for ws, a in QUAD]
        pat, nb = _patterns(masks, [lst] * 4)
        pv = _chi2_product_law(pat, [_flip_p(0, u, T)] * nb)
        assert pv > 1e-6, (u, T, pv)


def test_coin_word_lanes_are_fair_and_independent():
    """Class dE = 0 of the heat bath flips lane b by bit b of the coin word: every
    lane at rate 1/2, and the lanes independent (nibble patterns uniform)."""
    all_lanes = (1 << 32) - 1
    for ws, a in QUAD[:2]:
        m = ora.class_flips(1, DRAW_L, 3.0, DRAW_SEED, DRAW_S, a, 80_000, N_SWEEPS, ws, 3,
                            all_lanes)
        b = ((m[:, None].astype(np.int64) >> np.arange(32)) & 1)
        n = b.shape[0]
        z = np.abs(b.sum(axis=0) - n / 2) / math.sqrt(n / 4)
        assert z.max() < 5.0, (ws, int(np.argmax(z)), float(z.max()))
        for shift in range(0, 32, 4):
            nib = (m.astype(np.int64) >> shift) & 0xF
            assert _chi2_product_law(nib, [0.5] * 4) > 1e-6, (ws, shift)
        assert np.array_equal(
            m, [ora.coin_word(DRAW_L, DRAW_SEED, DRAW_S, a, 80_000 + t, ws)
                for t in range(N_SWEEPS)])
