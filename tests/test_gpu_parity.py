"""GPU parity: the CUDA library against the CPU oracle on the same seeded inputs.

Spins, couplings and every integer observable must match bit for bit; the FP64
derived quantities (C, q, C4 and its error, xi_1) within 1e-12 relative.  All
calls go through the C ABI (ctypes binding).
"""
import math
import os
import tempfile

import numpy as np
import pytest

import oracle as ora
from paper_1411_5512_gb300 import workloads

pytestmark = pytest.mark.gpu

REL = 1e-12


@pytest.fixture(scope="module")
def J():
    from paper_1411_5512_gb300 import build, job
    build.build()
    return job


def close(a, b, rel=REL):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    both_nan = np.isnan(a) & np.isnan(b)
    ok = both_nan | (np.abs(a - b) <= rel * np.maximum(np.abs(b), 1e-300)) | (a == b)
    return bool(np.all(ok))


def gpu_run(jm, L, p_neg, seed, S, T, rule, t_w, t, n, G=1):
    j = jm.EAJob(L, p_neg, seed, S, rng_group=G)
    j.set_schedule(t_w, t)
    j.quench(T, rule)
    j.sweep(n)
    return j


def compare_job(j, out, L, S_idx, t_w, t, n):
    """Integer sums of every scheduled pair and derived values against the oracle."""
    N = L ** 3
    for tw in t_w:
        for lag in t:
            if tw + lag > n:
                continue
            g = j.measure(tw, lag)
            assert np.array_equal(g["A"][S_idx], out["A"][(tw, lag)]), (tw, lag)
            assert np.array_equal(g["Q"][S_idx], out["Q"][tw + lag]), (tw, lag)
            assert np.array_equal(g["E"][S_idx], out["E"][tw + lag]), (tw, lag)
            assert np.array_equal(g["G"][S_idx], out["G"][tw]), tw
            if len(S_idx) == j.n_samples:
                d = ora.derived(out, L, tw, lag)
                assert close(g["C"], d["C"]) and close(g["q_mean"], np.mean(d["q"]))
                assert close(g["C4"], d["C4"]) and close(g["C4_sem"], d["C4_sem"])
                assert g["r_cut"] == d["r_cut"]
                assert close(g["xi1"], d["xi1"])
    return True


# ----------------------------------------------------------------------------------
# initial state
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("L,p_neg", [(2, 0.5), (4, 0.5), (6, 0.3), (8, 0.5), (12, 0.0),
                                     (16, 1.0), (24, 0.25), (32, 0.5), (48, 0.1)])
def test_initial_state_bit_exact(J, L, p_neg):
    S = 3
    j = J.EAJob(L, p_neg, 1000 + L, S)
    j.quench(0.7)
    for s in range(S):
        assert np.array_equal(j.couplings(s), ora.init_couplings(L, p_neg, 1000 + L, s))
        assert np.array_equal(j.all_spins(s), ora.init_spins(L, 1000 + L, s))
    j.close()


# ----------------------------------------------------------------------------------
# sweeps: final spins of every sample and replica
# ----------------------------------------------------------------------------------
SWEEP_CASES = [
    # L, p_neg, T, rule, G, S, sweeps
    (2, 0.5, 0.7, 0, 1, 2, 40),
    (4, 0.5, 0.7, 0, 1, 2, 30),
    (6, 0.5, 0.7, 0, 1, 2, 25),   # one site per word (L/2 odd)
    (8, 0.4, 0.9, 0, 1, 2, 25),
    (12, 0.5, 0.7, 0, 1, 2, 20),
    (16, 0.5, 0.7, 0, 1, 3, 30),
    (16, 0.5, 1.3, 1, 1, 2, 20),  # heat bath
    (4, 0.5, 0.8, 1, 1, 2, 30),   # heat bath, 8 lanes per word
    (6, 0.5, 1.0, 1, 1, 3, 25),   # heat bath, one site per word
    (8, 0.3, 0.7, 1, 1, 2, 25),
    (16, 0.5, float("inf"), 1, 1, 2, 4),  # heat bath at T = inf: every class by p = 1/2
    (16, 0.5, 0.7, 1, 2, 4, 20),  # heat bath, pairs of samples share random numbers
    (32, 0.5, 0.7, 1, 1, 2, 10),
    (32, 0.5, 3.0, 1, 1, 2, 6),   # many words take the rare path, and later draws
    (64, 0.5, 0.7, 1, 1, 1, 3),
    (16, 0.5, 0.7, 0, 2, 4, 20),  # pairs of samples share random numbers
    (16, 0.0, 0.0, 0, 1, 2, 10),  # T = 0 ferromagnet
    (16, 0.5, float("inf"), 0, 1, 2, 3),
    (16, 0.5, 0.0, 1, 1, 2, 8),   # heat bath at T = 0: dE = 0 flips with 1/2
    (16, 1.0, 0.5, 0, 1, 2, 10),
    (16, 0.5, 1e17, 0, 1, 2, 3),  # exp(-4/T) rounds to 1: dE = 4 accepted outright
    (24, 0.3, 0.9, 0, 1, 2, 15),
    (32, 0.5, 0.6, 0, 1, 2, 12),
    (48, 0.2, 0.7, 0, 1, 1, 4),
    (64, 0.5, 0.7, 0, 1, 1, 3),
    (96, 0.5, 0.7, 0, 1, 1, 2),
]


@pytest.mark.parametrize("L,p_neg,T,rule,G,S,n", SWEEP_CASES)
def test_sweeps_bit_exact(J, L, p_neg, T, rule, G, S, n):
    """Swept on its own: Metropolis samples of side up to 64 run sample-resident."""
    seed = 7 + L
    j = gpu_run(J, L, p_neg, seed, S, T, rule, [], [], n, G=G)
    ref = ora.run_job(L, p_neg, seed, S, T, rule, [], [], n, keep_spins=True, rng_group=G)
    for s in range(S):
        assert np.array_equal(j.all_spins(s), ref["spins"][s]), s
    j.close()


@pytest.mark.parametrize("L,p_neg,T,rule,G,S,n",
                         [c for c in SWEEP_CASES if c[3] == 0 and c[0] <= 64])
def test_sweeps_bit_exact_per_half_step(J, L, p_neg, T, rule, G, S, n):
    """The same Metropolis cases through a batch that keeps them off the sample-resident
    kernel: one launch per half-step (column, general-tile and side-64 kernels)."""
    seed = 7 + L
    j = J.EAJob(L, p_neg, seed, S, rng_group=G)
    j.quench(T, rule)
    b = J.EABatch()
    b.set_resident(0)
    b.add(j)
    b.sweep(n)
    b.close()
    ref = ora.run_job(L, p_neg, seed, S, T, rule, [], [], n, keep_spins=True, rng_group=G)
    for s in range(S):
        assert np.array_equal(j.all_spins(s), ref["spins"][s]), s
    j.close()


# the sample-resident kernel: several jobs of different sides in one launch, sweeps
# beyond one launch, the temperature limits, shared random numbers, many rare paths
RESIDENT_JOBS = [
    # tuples of (L, p_neg, T, G, S) swept together, sweeps
    ([(64, 0.5, 0.7, 1, 2), (16, 0.3, 1.1, 1, 3), (6, 0.5, 0.7, 1, 2)], 6),
    ([(32, 0.5, 0.6, 1, 4), (48, 0.2, 0.8, 2, 4)], 5),
    ([(8, 0.5, 0.7, 1, 2), (4, 0.5, 2.0, 1, 2), (2, 0.5, 1.0, 1, 2)], 1100),
    ([(24, 0.5, 5.0, 1, 2), (16, 0.5, float("inf"), 1, 2), (16, 0.0, 0.0, 1, 2)], 4),
    ([(64, 0.5, 1e17, 1, 1), (12, 0.5, 0.7, 2, 4)], 3),
]


@pytest.mark.parametrize("jobs,n", RESIDENT_JOBS)
def test_resident_kernel_bit_exact(J, jobs, n):
    handles = []
    b = J.EABatch()
    b.set_resident(64)
    for k, (L, p_neg, T, G, S) in enumerate(jobs):
        j = J.EAJob(L, p_neg, 900 + k + L, S, rng_group=G)
        j.quench(T)
        b.add(j)
        handles.append(j)
    b.sweep(n)
    b.close()
    for k, ((L, p_neg, T, G, S), j) in enumerate(zip(jobs, handles)):
        assert j.time == n
        pick = [0, S - 1] if S > 1 else [0]
        ref = ora.run_job(L, p_neg, 900 + k + L, S, T, 0, [], [], n, samples=pick,
                          keep_spins=True, rng_group=G)
        for i, s in enumerate(pick):
            assert np.array_equal(j.all_spins(s), ref["spins"][i]), (L, s)
        j.close()


# the side-64/128 kernel (2 x 2 word tiles, rows along y) under each segment length,
# including temperatures where many words take the rare path and its later draws
TILE_CASES = [
    # L, p_neg, T, cols_per_thread (segments of 4, 8, 16 rows; launches of fewer than
    # four blocks per SM take shorter segments, down to 2 rows, and launches of fewer
    # than one block per SM single rows), S, sweeps
    (128, 0.5, 0.7, 4, 80, 2),  # 16 rows
    (128, 0.4, 1.2, 2, 40, 2),  # 8 rows
    (64, 0.5, 0.9, 1, 160, 2),  # 4 rows
    (64, 0.5, 0.7, 1, 2, 4),    # the small cases: 1 row
    (64, 0.3, 2.0, 2, 2, 3),
    (64, 0.5, 5.0, 4, 2, 3),
    (64, 0.5, 0.0, 2, 1, 3),   # T = 0: no random numbers
    (64, 0.5, 1e17, 1, 1, 2),  # dE = 4 accepted outright, dE = 8, 12 by draws
    (128, 0.5, 1.5, 1, 3, 2),
    (128, 0.2, 0.7, 4, 3, 2),
]


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("L,p_neg,T,cpt,S,n", TILE_CASES)
def test_tile_kernel_bit_exact(J, L, p_neg, T, cpt, S, n, variant):
    """Sides 64 and 128 on the register-window tile kernel (variant 0) and, at side
    128 where the tables allow, the staged kernel (variant 1)."""
    if variant == 1 and L != 128:
        pytest.skip("the staged kernel is for side 128")
    seed = 500 + L + cpt
    j = J.EAJob(L, p_neg, seed, S)
    j.quench(T)
    b = J.EABatch()
    b.configure(cpt, 0)
    b.set_resident(0)  # side 64 on its tile kernel
    b.set_variant(variant)
    b.add(j)
    b.sweep(n)
    pick = [0, S - 1] if S > 1 else [0]
    ref = ora.run_job(L, p_neg, seed, S, T, 0, [], [], n, samples=pick, keep_spins=True)
    for i, s in enumerate(pick):
        assert np.array_equal(j.all_spins(s), ref["spins"][i]), s
    b.close()
    j.close()


@pytest.mark.parametrize("t0", [(1 << 32) - 1, (1 << 44) + 77])
@pytest.mark.parametrize("resident", [0, 64])
def test_tile_kernel_late_time(J, t0, resident):
    """The high bits of the sweep counter in the draws of the side-64 tile kernel and
    of the sample-resident kernel."""
    L, seed, p_neg, T = 64, 41, 0.5, 0.9
    Jc = ora.init_couplings(L, p_neg, seed, 0)
    S0 = ora.init_spins(L, seed, 0)
    ref = S0.copy()
    ora.sweeps(L, seed, 0, ref, Jc, T, 0, t0, 3)
    j = J.EAJob(L, p_neg, seed, 1)
    j.quench(T)
    j.set_time(t0)
    b = J.EABatch()
    b.set_resident(resident)
    b.add(j)
    b.sweep(3)
    b.close()
    assert np.array_equal(j.all_spins(0), ref)
    j.close()


GTILE_CASES = [
    # L, p_neg, T, cols_per_thread, S, sweeps: the general tile kernel (L divisible by
    # 16, lanes along y and z, realigned across the y and z wraps)
    (48, 0.5, 0.7, 1, 3, 3),
    (96, 0.4, 1.2, 2, 2, 2),
    (32, 0.5, 0.9, 4, 5, 3),
    (80, 0.5, 0.7, 2, 2, 2),     # 20 rows of words: segments of 4
    (160, 0.3, 2.0, 1, 1, 2),
    (48, 0.5, 0.0, 2, 2, 3),     # T = 0: no random numbers
    (48, 0.5, 1e17, 1, 2, 2),    # dE = 4 accepted outright
    (32, 0.5, float("inf"), 1, 2, 2),
]


@pytest.mark.parametrize("L,p_neg,T,cpt,S,n", GTILE_CASES)
def test_general_tile_kernel_bit_exact(J, L, p_neg, T, cpt, S, n):
    seed = 600 + L + cpt
    j = J.EAJob(L, p_neg, seed, S)
    j.quench(T)
    b = J.EABatch()
    b.configure(cpt, 0)
    b.set_resident(0)  # sides 32 and 48 on the general tiles
    b.add(j)
    b.sweep(n)
    pick = [0, S - 1] if S > 1 else [0]
    ref = ora.run_job(L, p_neg, seed, S, T, 0, [], [], n, samples=pick, keep_spins=True)
    for i, s in enumerate(pick):
        assert np.array_equal(j.all_spins(s), ref["spins"][i]), s
    b.close()
    j.close()


HEAT_CASES = [
    # L, p_neg, T, cols_per_thread, S, sweeps: the heat bath through a batch
    (128, 0.5, 0.7, 1, 3, 2),
    (128, 0.1, 0.7, 4, 2, 2),
    (64, 0.3, 1.0, 2, 5, 3),
    (64, 0.5, 6.0, 1, 2, 2),
    (48, 0.5, 0.7, 2, 2, 3),     # the general tiles (run-time lattice)
    (96, 0.4, 1.5, 1, 2, 2),
    (32, 0.5, 0.7, 4, 5, 3),
    (80, 0.5, 3.0, 2, 2, 2),     # many rare paths
    (16, 0.5, 0.7, 1, 3, 3),     # the column kernel
    (24, 0.3, 0.9, 2, 2, 3),
]


@pytest.mark.parametrize("L,p_neg,T,cpt,S,n", HEAT_CASES)
def test_heat_bath_batch_bit_exact(J, L, p_neg, T, cpt, S, n):
    seed = 700 + L + cpt
    j = J.EAJob(L, p_neg, seed, S)
    j.quench(T, 1)
    b = J.EABatch()
    b.configure(cpt, 0)
    b.add(j)
    b.sweep(n)
    pick = [0, S - 1] if S > 1 else [0]
    ref = ora.run_job(L, p_neg, seed, S, T, 1, [], [], n, samples=pick, keep_spins=True)
    for i, s in enumerate(pick):
        assert np.array_equal(j.all_spins(s), ref["spins"][i]), s
    b.close()
    j.close()


@pytest.mark.parametrize("L,rule,S,resident", [(64, 0, 4, 0), (64, 0, 4, 64), (64, 1, 4, 0),
                                                (48, 0, 3, 0), (96, 1, 2, 0), (128, 0, 2, 0)])
def test_shared_random_numbers_on_the_tiles(J, L, rule, S, resident):
    """Pairs of samples sharing their random numbers (G = 2) through the tile kernels of
    both rules and the sample-resident kernel: every sample against the oracle with the
    same share groups."""
    seed, p_neg, T, n = 40 + L, 0.5, 0.8, 3
    j = J.EAJob(L, p_neg, seed, S, rng_group=2)
    j.quench(T, rule)
    b = J.EABatch()
    b.set_resident(resident)
    b.add(j)
    b.sweep(n)
    b.close()
    pick = list(range(S)) if L <= 64 else [0, S - 1]
    ref = ora.run_job(L, p_neg, seed, S, T, rule, [], [], n, samples=pick, keep_spins=True,
                      rng_group=2)
    for i, s in enumerate(pick):
        assert np.array_equal(j.all_spins(s), ref["spins"][i]), s
    j.close()


@pytest.mark.parametrize("L,t0", [(16, (1 << 32) - 1), (64, (1 << 44) + 77)])
def test_heat_bath_late_time(J, L, t0):
    """The high bits of the sweep counter in the heat-bath draws, from an oracle-made state."""
    seed, p_neg, T = 43, 0.5, 0.8
    Jc = ora.init_couplings(L, p_neg, seed, 0)
    S0 = ora.init_spins(L, seed, 0)
    ora.sweeps(L, seed, 0, S0, Jc, T, 1, 0, 3)
    ref = S0.copy()
    ora.sweeps(L, seed, 0, ref, Jc, T, 1, t0, 3)
    j = J.EAJob(L, p_neg, seed, 1)
    j.quench(T, 1)
    j.set_couplings(0, Jc)
    j.set_spins(0, 0, S0[0])
    j.set_spins(0, 1, S0[1])
    j.set_time(t0)
    j.sweep(3)
    assert np.array_equal(j.all_spins(0), ref)
    j.close()


@pytest.mark.parametrize("L,S,n,T", [(2, 3, 4, 0.8), (4, 2, 6, 0.7), (6, 2, 5, 0.9), (8, 3, 4, 0.7),
                                     (12, 2, 3, 1.2), (16, 2, 4, 0.7), (32, 1, 3, 0.7)])
def test_c4_radial_matches_oracle(J, L, S, n, T):
    """Every bin of the four-point sums over all displacement vectors, exact, against
    the oracle's brute force on its own spins (multi-lane words for L < 64)."""
    seed, p_neg = 80 + L, 0.5
    j = J.EAJob(L, p_neg, seed, S)
    j.set_schedule([0, n], [0])
    j.quench(T)
    j.sweep(n)
    out = j.c4_radial(n)
    ref = ora.run_job(L, p_neg, seed, S, T, 0, [], [], n, keep_spins=True)
    ref_sums = []
    for s in range(S):
        sums, counts = ora.c4_radial_sums(ora.c4_full_sums(ref["spins"][s]))
        assert np.array_equal(out["counts"], counts)
        assert np.array_equal(out["sums"][s], sums), s
        ref_sums.append(sums)
    # the library's FP64 curve against the oracle's sums normalised here (Eq. 3 over
    # every vector of length r): C4 = sum / (count N S), the error over samples
    occ = np.nonzero(counts)[0]
    ref_sums = np.stack(ref_sums)[:, occ]
    norm = counts[occ] * float(L) ** 3
    assert close(out["C4"], ref_sums.sum(axis=0) / (norm * S))
    if S > 1:
        assert close(out["C4_sem"], (ref_sums / norm).std(axis=0, ddof=1) / math.sqrt(S))
    else:
        assert np.all(np.isnan(out["C4_sem"]))
    # the quenched state, from the snapshot at t_w = 0
    out0 = j.c4_radial(0)
    for s in range(S):
        S0 = np.stack([ora.init_spins(L, seed, s)[a] for a in range(2)])
        assert np.array_equal(out0["sums"][s], ora.c4_radial_sums(ora.c4_full_sums(S0))[0])
    j.close()


@pytest.mark.parametrize("L", [64, 128])
def test_c4_radial_full_size(J, L):
    """Sides 64 and 128: every vector at once through sum_v G(v) = Q^2, the r = 0 bin, and
    the shells of up to 12 vectors against the oracle on its own spins."""
    seed, p_neg, T, n, S = 90 + L, 0.5, 0.7, 2, 2
    j = J.EAJob(L, p_neg, seed, S)
    j.set_schedule([n], [0])
    j.quench(T)
    j.sweep(n)
    out = j.c4_radial(n)
    Q = j.measure(n, 0)["Q"]
    ref = ora.run_job(L, p_neg, seed, S, T, 0, [], [], n, keep_spins=True)
    N = L ** 3
    shells = {1: [(1, 0, 0), (L - 1, 0, 0), (0, 1, 0), (0, L - 1, 0), (0, 0, 1), (0, 0, L - 1)],
              3: [(a, b, c) for a in (1, L - 1) for b in (1, L - 1) for c in (1, L - 1)],
              2: [v for v in [(a, b, 0) for a in (1, L - 1) for b in (1, L - 1)] +
                  [(a, 0, c) for a in (1, L - 1) for c in (1, L - 1)] +
                  [(0, b, c) for b in (1, L - 1) for c in (1, L - 1)]]}
    for s in range(S):
        assert out["sums"][s, 0] == N
        assert int(out["sums"][s].sum()) == int(Q[s]) ** 2
        for r2, vecs in shells.items():
            assert out["counts"][r2] == len(vecs)
            assert out["sums"][s, r2] == int(ora.c4_at(ref["spins"][s], vecs).sum()), (s, r2)
    j.close()


@pytest.mark.parametrize("L,tws,n,pick", [(64, [0, 1, 3], 3, [0, 1]), (128, [0, 2], 2, [1])])
def test_c4_sums_sides_64_128(J, L, tws, n, pick):
    """The four-point sums of the sides whose lanes all lie along z (their own kernel):
    every axis and shift of the picked samples against the oracle."""
    seed, p_neg, T = 71, 0.5, 0.7
    j = J.EAJob(L, p_neg, seed, 2)
    j.set_schedule(tws, [0])
    j.quench(T)
    j.sweep(n)
    ref = ora.run_job(L, p_neg, seed, 2, T, 0, tws, [0], n, samples=pick)
    for tw in tws:
        g = j.measure(tw, 0)["G"]
        assert np.array_equal(g[pick], ref["G"][tw]), tw
    j.close()


# ----------------------------------------------------------------------------------
# scheduled observables
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("L,p_neg,T,S", [(16, 0.5, 0.7, 4), (8, 0.2, 0.6, 3), (12, 0.5, 1.0, 2)])
def test_observables_match_oracle(J, L, p_neg, T, S):
    t_w, t, n = [0, 1, 2, 4, 8], [0, 1, 2, 4, 8, 16], 30
    j = gpu_run(J, L, p_neg, 5, S, T, 0, t_w, t, n)
    out = ora.run_job(L, p_neg, 5, S, T, 0, t_w, t, n)
    compare_job(j, out, L, list(range(S)), t_w, t, n)
    j.close()


@pytest.mark.parametrize("L,S", [(8, 2), (64, 1)])
def test_dense_schedule_more_snapshots_than_one_pass(J, L, S):
    """Every sweep a waiting time and a lag: up to 23 autocorrelations fall due at one
    time, more than one pass over the state holds (16), so a time takes two."""
    t_w = list(range(0, 23))
    t = list(range(0, 23))
    n = 22
    j = gpu_run(J, L, 0.5, 9, S, 0.8, 0, t_w, t, n)
    out = ora.run_job(L, 0.5, 9, S, 0.8, 0, t_w, t, n)
    compare_job(j, out, L, list(range(S)), t_w, t, n)
    j.close()


def test_tiny_workload_full_length(J):
    w = workloads.TINY
    j = gpu_run(J, w["L"], w["p_neg"], w["seed"], w["n_samples"], w["T"], 0, w["t_w"], w["t"],
                w["sweeps"])
    out = ora.run_job(w["L"], w["p_neg"], w["seed"], w["n_samples"], w["T"], 0, w["t_w"],
                      w["t"], w["sweeps"], keep_spins=True)
    compare_job(j, out, w["L"], [0], w["t_w"], w["t"], w["sweeps"])
    assert np.array_equal(j.all_spins(0), out["spins"][0])
    # C(t_w, t_w) = 1
    assert j.measure(8, 0)["C"] == 1.0
    j.close()


def test_small_workload_sampled(J):
    """Side 32, 64 samples: the GPU runs all samples, the oracle three of them."""
    w = workloads.SMALL[0]
    n = 16
    t_w, t = [0, 2, 8], [0, 1, 4, 8]
    j = gpu_run(J, w["L"], w["p_neg"], w["seed"], w["n_samples"], w["T"], 0, t_w, t, n)
    pick = [0, 31, 63]
    out = ora.run_job(w["L"], w["p_neg"], w["seed"], w["n_samples"], w["T"], 0, t_w, t, n,
                      samples=pick, keep_spins=True)
    compare_job(j, out, w["L"], pick, t_w, t, n)
    for i, s in enumerate(pick):
        assert np.array_equal(j.all_spins(s), out["spins"][i])
    j.close()


# ----------------------------------------------------------------------------------
# late times and the high bits of the sweep counter, from oracle-made states
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("L,t0", [(16, (1 << 32) - 2), (24, (1 << 40) + 12345), (32, 999_983)])
def test_late_time_from_oracle_state(J, L, t0):
    seed, p_neg, T = 31, 0.5, 0.7
    Jc = ora.init_couplings(L, p_neg, seed, 0)
    S0 = ora.init_spins(L, seed, 0)
    ora.sweeps(L, seed, 0, S0, Jc, T, 0, 0, 5)  # an oracle-made, non-trivial state
    ref = S0.copy()
    ora.sweeps(L, seed, 0, ref, Jc, T, 0, t0, 4)
    j = J.EAJob(L, p_neg, seed, 1)
    j.quench(T)
    j.set_couplings(0, Jc)
    j.set_spins(0, 0, S0[0])
    j.set_spins(0, 1, S0[1])
    j.set_time(t0)
    j.sweep(4)
    assert j.time == t0 + 4
    assert np.array_equal(j.all_spins(0), ref)
    j.close()


# ----------------------------------------------------------------------------------
# full size (side 128, the benchmark's launch configuration), sampled
# ----------------------------------------------------------------------------------
def test_paper_scale_sampled(J):
    """All 80 samples of the five p_neg jobs run on the GPU; the oracle runs sample 0
    of the first and last job for three sweeps."""
    jobs = workloads.PAPER_SCALE
    n = 3
    handles = []
    for w in jobs:
        j = J.EAJob(w["L"], w["p_neg"], w["seed"], w["n_samples"])
        j.quench(w["T"])
        handles.append(j)
    for j in handles:
        j.sweep(n)
    for k in (0, len(jobs) - 1):
        w = jobs[k]
        out = ora.run_job(w["L"], w["p_neg"], w["seed"], w["n_samples"], w["T"], 0, [], [], n,
                          samples=[0], keep_spins=True)
        assert np.array_equal(handles[k].all_spins(0), out["spins"][0])
    for j in handles:
        j.close()


def test_gauge_covariance_full_size(J):
    """Property at any size: J' = e_i e_j J, S'(0) = e S(0) gives S'(t) = e S(t)."""
    L, seed = 128, 3
    rng = np.random.default_rng(9)
    eps = rng.choice(np.array([-1, 1], dtype=np.int8), size=(L, L, L))
    Jc = ora.init_couplings(L, 0.5, seed, 0)
    S0 = ora.init_spins(L, seed, 0)
    Jg = np.empty_like(Jc)
    for d, ax in ((0, 2), (1, 1), (2, 0)):
        Jg[d] = Jc[d] * eps * np.roll(eps, -1, axis=ax)
    a = J.EAJob(L, 0.5, seed, 1)
    b = J.EAJob(L, 0.5, seed, 1)
    for j, JJ, SS in ((a, Jc, S0), (b, Jg, (S0 * eps[None]).astype(np.int8))):
        j.quench(0.7)
        j.set_couplings(0, JJ)
        j.set_spins(0, 0, SS[0])
        j.set_spins(0, 1, SS[1])
        j.sweep(50)
    assert np.array_equal(b.all_spins(0), a.all_spins(0) * eps[None])
    a.close()
    b.close()


def test_infinite_temperature_full_size(J):
    L = 128
    j = J.EAJob(L, 0.5, 4, 2)
    j.quench(float("inf"))
    s0 = [j.all_spins(s) for s in range(2)]
    j.sweep(3)
    for s in range(2):
        assert np.array_equal(j.all_spins(s), -s0[s])
    j.close()


def test_largest_side(J):
    """The largest side the library takes (1024: 2^30 sites, 671 MB of state per
    sample, the general tile kernel), by properties that hold at any size: at T = inf
    every spin flips every sweep; the ferromagnet at T = 0 from all spins up stays put;
    the overlap and energy sums agree with the spins read back."""
    L = 1024
    j = J.EAJob(L, 0.5, 8, 1)
    j.set_schedule([0, 1], [0])
    j.quench(float("inf"))
    s0 = j.spins(0, 0)
    j.sweep(1)
    assert np.array_equal(j.spins(0, 0), -s0)
    m = j.measure(1, 0)
    assert m["Q"][0] == int(np.sum(j.spins(0, 0) * j.spins(0, 1), dtype=np.int64))
    assert m["A"][0, 0] == L ** 3  # C(t_w, t_w) = 1
    j.close()
    f = J.EAJob(L, 0.0, 9, 1)
    f.quench(0.0)
    up = np.ones((L, L, L), dtype=np.int8)
    f.set_spins(0, 0, up)
    f.set_spins(0, 1, up)
    f.sweep(1)
    assert np.array_equal(f.spins(0, 0), up) and np.array_equal(f.spins(0, 1), up)
    f.close()


# ----------------------------------------------------------------------------------
# state handling and errors
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("L,rule,exact", [(16, 0, False), (64, 1, False), (32, 0, True)])
def test_checkpoint_restore_continues_bit_exact(J, tmp_path, L, rule, exact):
    S = 2
    t_w, t = [0, 4, 8], [0, 2, 8]
    if exact:  # couplings with an exact count, which the restore must carry over
        a = J.EAJob(L, 0.5, 12, S, exact_count=True)
        a.set_schedule(t_w, t)
        a.quench(0.7, rule)
        a.sweep(10)
    else:
        a = gpu_run(J, L, 0.5, 12, S, 0.7, rule, t_w, t, 10)
    path = str(tmp_path / "job.ckpt")
    a.checkpoint(path)
    a.sweep(9)
    b = J.EAJob.restore(path)
    assert b.time == 10
    b.sweep(9)
    for s in range(S):
        assert np.array_equal(a.all_spins(s), b.all_spins(s))
    for tw in t_w:
        for lag in t:
            ma, mb = a.measure(tw, lag), b.measure(tw, lag)
            for k in ("A", "Q", "E", "G"):
                assert np.array_equal(ma[k], mb[k])
        assert np.array_equal(a.c4_radial(tw)["sums"], b.c4_radial(tw)["sums"])
    for s in range(S):
        assert np.array_equal(a.couplings(s), b.couplings(s))
    a.close()
    b.close()


def test_thresholds_in_use_match_oracle(J):
    j = J.EAJob(8, 0.5, 1, 1)
    j.quench(0.55, 1)
    thr, alw = j.thresholds()
    t2, a2 = ora.thresholds(0.55, 1)
    assert np.array_equal(thr, t2) and np.array_equal(alw, a2)
    j.close()


def test_error_statuses(J):
    from paper_1411_5512_gb300 import _lib
    j = J.EAJob(8, 0.5, 1, 2)
    with pytest.raises(_lib.EAError) as e:
        j.sweep(1)
    assert e.value.status == _lib.EA_ERR_STATE
    j.set_schedule([0, 2], [0, 1])
    j.quench(0.7)
    with pytest.raises(_lib.EAError) as e:
        j.set_schedule([0], [0])
    assert e.value.status == _lib.EA_ERR_STATE
    with pytest.raises(_lib.EAError) as e:
        j.measure(2, 1)  # not reached yet
    assert e.value.status == _lib.EA_ERR_NO_SNAPSHOT
    j.sweep(3)
    j.measure(2, 1)
    with pytest.raises(_lib.EAError) as e:
        j.measure(1, 1)  # 1 is not a waiting time
    assert e.value.status == _lib.EA_ERR_NO_SNAPSHOT
    with pytest.raises(_lib.EAError) as e:
        j.spins(2, 0)
    assert e.value.status == _lib.EA_ERR_INVALID_ARG
    bad = np.zeros((8, 8, 8), dtype=np.int8)
    with pytest.raises(_lib.EAError):
        j.set_spins(0, 0, bad)
    j.close()


def test_torch_allocator_route(J):
    import torch
    J.use_torch_allocator()
    try:
        before = torch.cuda.memory_allocated()
        j = gpu_run(J, 16, 0.5, 2, 2, 0.7, 0, [0, 1], [0, 1], 3)
        assert torch.cuda.memory_allocated() > before
        ref = ora.run_job(16, 0.5, 2, 2, 0.7, 0, [0, 1], [0, 1], 3, keep_spins=True)
        assert np.array_equal(j.all_spins(1), ref["spins"][1])
        j.close()
        assert torch.cuda.memory_allocated() == before
    finally:
        J.use_cuda_allocator()


# ----------------------------------------------------------------------------------
# couplings with an exact count of negative bonds
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("L,p_neg,S", [(2, 0.5, 3), (4, 0.3, 2), (6, 0.137, 2), (16, 0.5, 3),
                                       (16, 0.0, 1), (16, 1.0, 1), (32, 0.21, 2), (128, 0.1, 1)])
def test_exact_count_couplings(J, L, p_neg, S):
    seed = 300 + L
    j = J.EAJob(L, p_neg, seed, S, exact_count=True)
    K = int(math.floor(p_neg * 3 * L ** 3 + 0.5))
    for s in range(S):
        Jg = j.couplings(s)
        assert int(np.sum(Jg == -1)) == K
        assert np.array_equal(Jg, ora.init_couplings_exact(L, p_neg, seed, s)), s
    j.close()


def test_exact_count_job_runs_like_the_oracle(J):
    """A job on exact-count couplings sweeps as the oracle does on the same couplings."""
    L, p_neg, seed, S, T, n = 16, 0.5, 77, 2, 0.7, 10
    j = J.EAJob(L, p_neg, seed, S, exact_count=True)
    j.quench(T)
    j.sweep(n)
    for s in range(S):
        Jc = ora.init_couplings_exact(L, p_neg, seed, s)
        Sref = ora.init_spins(L, seed, s)
        ora.sweeps(L, seed, s, Sref, Jc, T, 0, 0, n)
        assert np.array_equal(j.all_spins(s), Sref), s
    j.close()


def test_coupling_words_move_whole_disorder(J):
    """The packed couplings of one job set into another reproduce every bond; words with
    bits outside their lanes (side 6: one site per word) are refused."""
    from paper_1411_5512_gb300 import _lib
    a = J.EAJob(16, 0.3, 5, 2)
    b = J.EAJob(16, 0.3, 99, 2)
    words = a.coupling_words()
    assert words.size == 2 * 3 * (16 ** 3 // 32)
    b.set_coupling_words(words)
    for s in range(2):
        assert np.array_equal(a.couplings(s), b.couplings(s))
        assert np.array_equal(b.couplings(s), ora.init_couplings(16, 0.3, 5, s))
    c = J.EAJob(6, 0.5, 1, 1)
    w6 = c.coupling_words()
    w6[3] |= np.uint32(2)
    with pytest.raises(_lib.EAError):
        c.set_coupling_words(w6)
    for j in (a, b, c):
        j.close()


# ----------------------------------------------------------------------------------
# sample ranges: a context holding samples [lo, hi) of a job
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("L,S,lo,hi,G,rule,batch",
                         [(16, 5, 2, 5, 1, 0, False), (32, 6, 1, 4, 2, 0, True),
                          (64, 4, 1, 3, 1, 1, True), (128, 5, 3, 5, 1, 0, True),
                          (128, 4, 1, 3, 2, 1, False)])
def test_sample_range_matches_whole_job(J, L, S, lo, hi, G, rule, batch):
    """Samples lo .. hi-1 of a job created on their own (their job-local indices key
    every random number, share groups included) equal those samples of the whole job
    bit for bit: spins, couplings and every integer sum; one of them also equals the
    oracle."""
    seed, p_neg, T, n = 40 + L, 0.4, 0.8, 4
    t_w, t = [0, 2], [0, 1, 2]
    whole = J.EAJob(L, p_neg, seed, S, rng_group=G)
    part = J.EAJob(L, p_neg, seed, hi - lo, rng_group=G, first_sample=lo)
    for j in (whole, part):
        j.set_schedule(t_w, t)
        j.quench(T, rule)
        if batch:
            b = J.EABatch()
            b.add(j)
            b.sweep(n)
            b.close()
        else:
            j.sweep(n)
    for i, s in enumerate(range(lo, hi)):
        assert np.array_equal(part.couplings(i), whole.couplings(s)), s
        assert np.array_equal(part.all_spins(i), whole.all_spins(s)), s
    for tw in t_w:
        for lag in t:
            a, b_ = part.measure(tw, lag), whole.measure(tw, lag)
            for k in ("A", "Q", "E", "G"):
                assert np.array_equal(a[k], b_[k][lo:hi]), (k, tw, lag)
    ref = ora.run_job(L, p_neg, seed, S, T, rule, [], [], n, samples=[hi - 1], keep_spins=True,
                      rng_group=G)
    assert np.array_equal(part.all_spins(hi - lo - 1), ref["spins"][0])
    whole.close()
    part.close()


def test_sample_range_rejects_bad_ranges(J):
    from paper_1411_5512_gb300 import _lib
    for first, n in ((-1, 2), (65534, 2), (0, 0)):
        with pytest.raises(_lib.EAError) as e:
            J.EAJob(16, 0.5, 1, n, first_sample=first)
        assert e.value.status == _lib.EA_ERR_INVALID_ARG
