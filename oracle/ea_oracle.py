"""CPU oracle for the 3D +-J Edwards-Anderson ageing simulation (arXiv 1411.5512).

TEST INFRASTRUCTURE ONLY: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA library and never imports it.

The Markov chain itself (Philox draws, thresholds, initial state, checkerboard
Metropolis / heat-bath sweep) is plain C in ``ea_oracle.c``; this module wraps it
with ctypes and computes the observables from int8 spin arrays with numpy:

* overlap            q = (1/N) sum_i S^a_i S^b_i                  (Sec. II, Eq. 2)
* four-point         C4(r, t_w) = (1/N) sum_i q_i q_{i+r}         (Sec. II, Eq. 3)
                     along the axes, and over every displacement vector binned by
                     r^2 (the larger point set of the Sec. IV error bars)
* integral estimator I_k = int_0^{L/2} r^k C4 dr, xi_k = I_{k+1}/I_k, k = 1
                                                                  (Sec. II, Eqs. 5-6)
* autocorrelation    C(t, t_w) = (1/N) sum_i S_i(t_w) S_i(t_w+t)  (Sec. II, Eq. 7)
* energy             H = -sum_<ij> J_ij S_i S_j                   (Sec. II, Eq. 1)

Arrays use index order [z][y][x] (x fastest), spins S[a] for replicas a = 0, 1
and couplings J[d] for d = x, y, z, J[d] linking a site to its +e_d neighbour.

Readings of the paper taken here (the paper is silent on them):
* C(t, t_w) is averaged over both replicas and all samples.
* C4 is the non-connected correlation along the three lattice axes, r = 0..L/2,
  averaged over axes and samples; its error is the standard error of the mean
  over samples of the per-sample axis average.
* xi_1 uses rectangle sums over integer r = 1..r_c.  r_c is the last r before the
  first r >= 1 at which C4(r) < 3 * error (Sec. IV: the integral is cut where C4
  first falls below three times its error); r_c = L/2 if there is no such r or
  fewer than two samples.  The fitted tail correction is not applied.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    """Load (building if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i8p = ctypes.POINTER(ctypes.c_int8)
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.ora_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.ora_philox4x32_10.restype = None
        L.ora_geometry.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.ora_geometry.restype = ctypes.c_int
        L.ora_site_to_word.argtypes = [ctypes.c_int] * 4 + [u32p, ctypes.POINTER(ctypes.c_int)]
        L.ora_site_to_word.restype = ctypes.c_int
        L.ora_thresholds.argtypes = [ctypes.c_double, ctypes.c_int, u64p, u8p]
        L.ora_thresholds.restype = ctypes.c_int
        L.ora_init_couplings.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                         ctypes.c_uint32, i8p]
        L.ora_init_couplings.restype = ctypes.c_int
        L.ora_init_couplings_exact.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                               ctypes.c_uint32, i8p]
        L.ora_init_couplings_exact.restype = ctypes.c_int
        L.ora_init_spins.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, i8p]
        L.ora_init_spins.restype = ctypes.c_int
        L.ora_sweeps.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, i8p, i8p,
                                 ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                 i64p]
        L.ora_sweeps.restype = ctypes.c_int
        L.ora_half_step.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, i8p, i8p,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                    i64p]
        L.ora_half_step.restype = ctypes.c_int
        L.ora_geo_table.argtypes = [ctypes.c_double, u64p]
        L.ora_geo_table.restype = ctypes.c_int
        L.ora_draw64.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                 ctypes.c_int, ctypes.c_uint64] + [ctypes.c_int] * 5 + [u64p]
        L.ora_draw64.restype = ctypes.c_int
        L.ora_coin_word.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                    ctypes.c_uint64] + [ctypes.c_int] * 3 + [u32p]
        L.ora_coin_word.restype = ctypes.c_int
        L.ora_class_flips.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                      ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_uint32, u32p]
        L.ora_class_flips.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle: %s rejected its arguments" % what)


# ----------------------------------------------------------------------------------
# thin wrappers over the C chain
# ----------------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().ora_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                            _ptr(out, ctypes.c_uint32))
    return out


def geometry(L):
    """(kx, ky, kz, L/kx, L/ky, L/kz) of the random-number word-site mapping."""
    g = (ctypes.c_int * 6)()
    _check(lib().ora_geometry(L, g), "geometry(L=%d)" % L)
    return tuple(g)


def site_to_word(L, x, y, z):
    w = ctypes.c_uint32()
    b = ctypes.c_int()
    _check(lib().ora_site_to_word(L, x, y, z, ctypes.byref(w), ctypes.byref(b)), "site_to_word")
    return w.value, b.value


def thresholds(T, rule=0):
    """(thr[7], always[7]) for dE = -12, -8, ..., +12 (index k = (dE + 12) / 4)."""
    thr = np.zeros(7, dtype=np.uint64)
    alw = np.zeros(7, dtype=np.uint8)
    _check(lib().ora_thresholds(float(T), int(rule), _ptr(thr, ctypes.c_uint64),
                                _ptr(alw, ctypes.c_uint8)), "thresholds(T=%r)" % T)
    return thr, alw


def init_couplings(L, p_neg, seed, s):
    J = np.zeros((3, L, L, L), dtype=np.int8)
    _check(lib().ora_init_couplings(L, float(p_neg), seed, s, _ptr(J, ctypes.c_int8)),
           "init_couplings")
    return J


def init_couplings_exact(L, p_neg, seed, s):
    """Couplings with exactly floor(p_neg 3N + 1/2) negative bonds, the subset uniform."""
    J = np.zeros((3, L, L, L), dtype=np.int8)
    _check(lib().ora_init_couplings_exact(L, float(p_neg), seed, s, _ptr(J, ctypes.c_int8)),
           "init_couplings_exact")
    return J


def init_spins(L, seed, s):
    S = np.zeros((2, L, L, L), dtype=np.int8)
    _check(lib().ora_init_spins(L, seed, s, _ptr(S, ctypes.c_int8)), "init_spins")
    return S


def sweeps(L, seed, s, S, J, T, rule, t0, n):
    """Run sweeps t0 .. t0+n-1 in place on S; return the accepted dE per replica.

    ``s`` keys the sweep random numbers: the sample index, or sample // G when
    G samples share their random numbers.
    """
    assert S.dtype == np.int8 and S.shape == (2, L, L, L) and S.flags.c_contiguous
    J = np.ascontiguousarray(J, dtype=np.int8)
    dE = np.zeros(2, dtype=np.int64)
    _check(lib().ora_sweeps(L, seed, s, _ptr(S, ctypes.c_int8), _ptr(J, ctypes.c_int8),
                            float(T), int(rule), t0, n, _ptr(dE, ctypes.c_int64)), "sweeps")
    return dE


def half_step(L, seed, s, S, J, T, rule, t, h):
    """Half-step h of sweep t in place on S; return the accepted dE per replica."""
    assert S.dtype == np.int8 and S.shape == (2, L, L, L) and S.flags.c_contiguous
    J = np.ascontiguousarray(J, dtype=np.int8)
    dE = np.zeros(2, dtype=np.int64)
    _check(lib().ora_half_step(L, seed, s, _ptr(S, ctypes.c_int8), _ptr(J, ctypes.c_int8),
                               float(T), int(rule), t, h, _ptr(dE, ctypes.c_int64)), "half_step")
    return dE


def geo_table(p):
    """C[g] = floor(2^64 (1 - (1 - p)^g)), g = 0..32: the geometric-gap table."""
    C = np.zeros(33, dtype=np.uint64)
    _check(lib().ora_geo_table(float(p), _ptr(C, ctypes.c_uint64)), "geo_table(p=%r)" % p)
    return C


def draw64(rule, L, seed, s, a, t, word_site, u, d):
    """The 64-bit uniform number of draw d of class u at word-site (x', y', z'),
    replica a, sweep t (the draw contract stated beside draw64 in ea_oracle.c)."""
    xw, yw, zw = word_site
    out = ctypes.c_uint64()
    _check(lib().ora_draw64(int(rule), L, seed, s, int(a), t, xw, yw, zw, int(u), int(d),
                            ctypes.byref(out)), "draw64")
    return out.value


def coin_word(L, seed, s, a, t, word_site):
    """The heat bath's coin word of a word-site: bit b decides lane b of class dE = 0."""
    xw, yw, zw = word_site
    out = ctypes.c_uint32()
    _check(lib().ora_coin_word(L, seed, s, int(a), t, xw, yw, zw, ctypes.byref(out)),
           "coin_word")
    return out.value


def class_flips(rule, L, T, seed, s, a, t0, n_t, word_site, u, lanes):
    """The lanes (bit mask) of class u that flip, among the lanes `lanes` of one
    word-site, at sweeps t0 .. t0 + n_t - 1: the half-step's decision for that class."""
    xw, yw, zw = word_site
    out = np.zeros(n_t, dtype=np.uint32)
    _check(lib().ora_class_flips(int(rule), L, float(T), seed, s, int(a), t0, n_t, xw, yw, zw,
                                 int(u), int(lanes), _ptr(out, ctypes.c_uint32)), "class_flips")
    return out


# ----------------------------------------------------------------------------------
# observables: exact integer sums (int64)
# ----------------------------------------------------------------------------------
_AXIS = {0: 2, 1: 1, 2: 0}  # direction d = x, y, z -> numpy axis of a [z][y][x] array


def autocorr_sum(S_tw, S_now):
    """sum_i S_i(t_w) S_i(t_w + t) for each replica (Eq. 7 without the 1/N)."""
    return np.array([int(np.sum(S_tw[a].astype(np.int64) * S_now[a])) for a in range(2)],
                    dtype=np.int64)


def overlap_sum(S):
    """sum_i S^0_i S^1_i (Eq. 2 without the 1/N)."""
    return np.int64(np.sum(S[0].astype(np.int64) * S[1]))


def c4_sums(S):
    """G[d][r] = sum_i q_i q_{i + r e_d} for d = x, y, z and r = 0..L/2 (Eq. 3)."""
    L = S.shape[1]
    q = S[0].astype(np.int64) * S[1]
    G = np.zeros((3, L // 2 + 1), dtype=np.int64)
    for d in range(3):
        for r in range(L // 2 + 1):
            G[d, r] = np.sum(q * np.roll(q, -r, axis=_AXIS[d]))
    return G


def c4_full_sums(S):
    """G[dz, dy, dx] = sum_i q_i q_{i + (dx, dy, dz)} for every displacement vector of the
    periodic lattice (Eq. 3 with i + r any site at vector distance r from i), by brute
    force over the vectors."""
    L = S.shape[1]
    q = S[0].astype(np.int64) * S[1]
    G = np.empty((L, L, L), dtype=np.int64)
    for dz in range(L):
        qz = np.roll(q, -dz, axis=0)
        for dy in range(L):
            qzy = np.roll(qz, -dy, axis=1)
            for dx in range(L):
                G[dz, dy, dx] = np.sum(q * np.roll(qzy, -dx, axis=2))
    return G


def c4_at(S, vectors):
    """sum_i q_i q_{i + v} for a list of displacement vectors v = (dx, dy, dz)."""
    q = S[0].astype(np.int64) * S[1]
    return np.array([np.sum(q * np.roll(q, (-dz, -dy, -dx), axis=(0, 1, 2)))
                     for dx, dy, dz in vectors], dtype=np.int64)


def radial_index(L):
    """r^2 of the shortest periodic image of each displacement vector, [dz, dy, dx]:
    sum over the axes of min(d, L - d)^2, in 0 .. 3 (L/2)^2."""
    d = np.arange(L)
    m2 = np.minimum(d, L - d) ** 2
    return m2[:, None, None] + m2[None, :, None] + m2[None, None, :]


def c4_radial_sums(G):
    """(sums, counts): the sums G(v) over the vectors of each r^2 = 0 .. 3 (L/2)^2, and
    how many vectors each r^2 holds."""
    L = G.shape[0]
    r2 = radial_index(L).ravel()
    n_bins = 3 * (L // 2) ** 2 + 1
    sums = np.zeros(n_bins, dtype=np.int64)
    np.add.at(sums, r2, G.ravel())
    counts = np.bincount(r2, minlength=n_bins).astype(np.int64)
    return sums, counts


def energy(S, J):
    """H = -sum_{i,d} J_d(i) S_i S_{i+e_d} for each replica (Eq. 1)."""
    E = np.zeros(2, dtype=np.int64)
    for a in range(2):
        s = S[a].astype(np.int64)
        tot = 0
        for d in range(3):
            tot += np.sum(J[d].astype(np.int64) * s * np.roll(s, -1, axis=_AXIS[d]))
        E[a] = -tot
    return E


# ----------------------------------------------------------------------------------
# FP64 derived quantities
# ----------------------------------------------------------------------------------
def autocorrelation(A, N):
    """C(t, t_w) from A[s][a]: average over samples and replicas of A / N."""
    A = np.asarray(A, dtype=np.int64)
    return float(A.sum()) / float(N * A.size)


def overlaps(Q, N):
    """q_s = Q_s / N per sample."""
    return np.asarray(Q, dtype=np.float64) / float(N)


def c4_curve(G, N):
    """(C4[r], sem[r]) from G[s][d][r]: axis and sample average, SEM over samples."""
    G = np.asarray(G, dtype=np.int64)
    S = G.shape[0]
    per_sample = G.sum(axis=1).astype(np.float64) / (3.0 * N)  # [s][r]
    c4 = G.sum(axis=(0, 1)).astype(np.float64) / (3.0 * N * S)
    if S >= 2:
        sem = per_sample.std(axis=0, ddof=1) / np.sqrt(S)
    else:
        sem = np.full(c4.shape, np.nan)
    return c4, sem


def cutoff(c4, sem):
    """r_c: last r before the first r >= 1 with C4(r) < 3 sem(r); else r_max."""
    rmax = len(c4) - 1
    if np.all(np.isnan(sem)):
        return rmax
    for r in range(1, rmax + 1):
        if c4[r] < 3.0 * sem[r]:
            return r - 1
    return rmax


def xi1(c4, r_c):
    """xi_1 = I_2 / I_1 with I_k = sum_{r=1}^{r_c} r^k C4(r) (Eqs. 5-6, k = 1)."""
    I1 = 0.0
    I2 = 0.0
    for r in range(1, r_c + 1):
        I1 += r * c4[r]
        I2 += r * r * c4[r]
    if r_c < 1 or I1 == 0.0:
        return float("nan")
    return I2 / I1


# ----------------------------------------------------------------------------------
# a whole job: couplings, quench, sweeps with scheduled measurements
# ----------------------------------------------------------------------------------
def measurement_times(t_w, t, n_sweeps):
    times = set(int(x) for x in t_w if x <= n_sweeps)
    for a in t_w:
        for b in t:
            if a + b <= n_sweeps:
                times.add(int(a + b))
    return sorted(times)


def run_job(L, p_neg, seed, n_samples, T, rule, t_w, t, n_sweeps, samples=None,
            keep_spins=False, rng_group=1):
    """Run one job and return its integer observables.

    Returns a dict with
      'A'  {(t_w, t): int64 [S][2]}     autocorrelation sums
      'Q'  {m: int64 [S]}               overlap sums at every measurement time m
      'E'  {m: int64 [S][2]}            energies at every measurement time m
      'G'  {t_w: int64 [S][3][L/2+1]}   four-point sums at each t_w
      'dE' int64 [S][2]                 accepted energy changes over the run
      'spins' int8 [S][2][L][L][L]      final spins (if keep_spins)
    ``samples`` selects a subset of the sample indices 0..n_samples-1.  Samples
    s and s' with s // rng_group == s' // rng_group share their sweep random
    numbers (disorder and initial spins stay per sample).
    """
    t_w = sorted(set(int(x) for x in t_w))
    t = sorted(set(int(x) for x in t))
    samples = list(range(n_samples)) if samples is None else list(samples)
    times = measurement_times(t_w, t, n_sweeps)
    S_count = len(samples)
    out = {"A": {}, "Q": {}, "E": {}, "G": {},
           "dE": np.zeros((S_count, 2), dtype=np.int64)}
    for m in times:
        out["Q"][m] = np.zeros(S_count, dtype=np.int64)
        out["E"][m] = np.zeros((S_count, 2), dtype=np.int64)
    for a in t_w:
        if a <= n_sweeps:
            out["G"][a] = np.zeros((S_count, 3, L // 2 + 1), dtype=np.int64)
        for b in t:
            if a + b <= n_sweeps:
                out["A"][(a, b)] = np.zeros((S_count, 2), dtype=np.int64)
    finals = []
    for si, s in enumerate(samples):
        J = init_couplings(L, p_neg, seed, s)
        S = init_spins(L, seed, s)
        snaps = {}
        now = 0
        for m in times + [n_sweeps]:
            if m > now:
                out["dE"][si] += sweeps(L, seed, s // rng_group, S, J, T, rule, now, m - now)
                now = m
            if m not in out["Q"]:
                continue
            out["Q"][m][si] = overlap_sum(S)
            out["E"][m][si] = energy(S, J)
            if m in out["G"]:
                snaps[m] = S.copy()
                out["G"][m][si] = c4_sums(S)
            for a in t_w:
                if a <= m and (a, m - a) in out["A"]:
                    out["A"][(a, m - a)][si] = autocorr_sum(snaps[a], S)
        if keep_spins:
            finals.append(S.copy())
    if keep_spins:
        out["spins"] = np.stack(finals) if finals else np.zeros((0, 2, L, L, L), np.int8)
    return out


def derived(out, L, t_w, t):
    """FP64 derived quantities of one (t_w, t) pair of a run_job result."""
    N = L ** 3
    res = {"C": autocorrelation(out["A"][(t_w, t)], N),
           "q": overlaps(out["Q"][t_w + t], N)}
    c4, sem = c4_curve(out["G"][t_w], N)
    rc = cutoff(c4, sem)
    res.update({"C4": c4, "C4_sem": sem, "r_cut": rc, "xi1": xi1(c4, rc)})
    return res
