"""The host analysis of Sec. IV (C4 multifit, xi_1 with the fitted tail, z, x,
collapse) recovers the parameters of synthetic data built from the very forms it
fits; on the GPU it runs on measured curves."""
import numpy as np
import pytest

pytest.importorskip("scipy")

import oracle as ora
from paper_1411_5512_gb300 import analysis as an


def model_curves(alpha, beta, xis, As, L=64, rel_err=1e-3):
    r = np.arange(0, L // 2 + 1, dtype=np.float64)
    curves = []
    for xi, A in zip(xis, As):
        c = np.ones_like(r)
        c[1:] = an.c4_model(r[1:], A, alpha, xi, beta)
        curves.append((r, c, rel_err * np.abs(c) + 1e-12))
    return curves


def test_c4_model_hand_values():
    """Eq. 4 with a stretched exponential, A r^-alpha exp(-(r / xi)^beta), at points
    worked by hand."""
    assert abs(an.c4_model(1.0, 1.0, 0.5, 2.0, 1.0) - np.exp(-0.5)) < 1e-15
    assert abs(an.c4_model(4.0, 2.0, 0.5, 2.0, 2.0) - np.exp(-4.0)) < 1e-15  # 2 * 4^-1/2 * e^-(2^2)
    assert abs(an.c4_model(2.0, 3.0, 1.0, 2.0, 1.0) - 1.5 * np.exp(-1.0)) < 1e-15


def test_multifit_uses_points_from_r_min_on():
    """Sec. IV fits r >= 3: a wrong point at r = 2 changes nothing, one at r = 3 does."""
    alpha, beta = 0.45, 1.45
    xis, As = [2.0, 3.1, 4.7], [0.9, 0.85, 0.8]
    for r_bad, moves in ((2, False), (3, True)):
        curves = model_curves(alpha, beta, xis, As)
        for r, c, _ in curves:
            c[r == r_bad] *= 1.5
        fit = an.multifit_c4(curves, r_min=3)
        assert (abs(fit["alpha"] - alpha) > 1e-4) == moves, (r_bad, fit["alpha"])


def test_multifit_recovers_exact_parameters():
    alpha, beta = 0.45, 1.45
    xis, As = [2.0, 3.1, 4.7, 7.5], [0.9, 0.85, 0.8, 0.78]
    fit = an.multifit_c4(model_curves(alpha, beta, xis, As), r_min=3)
    assert abs(fit["alpha"] - alpha) < 1e-6 and abs(fit["beta"] - beta) < 1e-6
    assert np.allclose(fit["xi"], xis, rtol=1e-6) and np.allclose(fit["A"], As, rtol=1e-6)
    assert fit["chi2_dof"] < 1e-10


def test_multifit_with_noise_within_errors():
    alpha, beta = 0.5, 1.5
    xis, As = [2.5, 4.0, 6.0], [1.0, 1.0, 1.0]
    rng = np.random.default_rng(3)
    noisy = []
    for r, c, e in model_curves(alpha, beta, xis, As, rel_err=0.01):
        noisy.append((r, c + e * rng.standard_normal(len(c)), e))
    fit = an.multifit_c4(noisy, r_min=3)
    assert abs(fit["alpha"] - alpha) < 5 * fit["alpha_err"] + 1e-3
    assert abs(fit["beta"] - beta) < 5 * fit["beta_err"] + 1e-3
    assert np.all(np.abs(fit["xi"] - xis) < 5 * fit["xi_err"] + 1e-3)
    assert 0.5 < fit["chi2_dof"] < 2.0


def test_xi1_tail_continues_the_measured_sums():
    L = 64
    params = (0.9, 0.5, 4.0, 1.5)
    r = np.arange(0, L // 2 + 1, dtype=np.float64)
    c = np.ones_like(r)
    c[1:] = an.c4_model(r[1:], *params)
    full = an.xi1_with_tail(r, c, L // 2, L)
    # a cutoff continued with the same form gives the uncut value
    for r_c in (3, 7, 20):
        assert abs(an.xi1_with_tail(r, c, r_c, L, fit=params) - full) < 1e-12 * full
    # without a tail: the oracle's rectangle-sum estimator with the same cutoff
    for r_c in (5, 11):
        assert abs(an.xi1_with_tail(r, c, r_c, L) - ora.xi1(c, r_c)) < 1e-12


def test_fit_z_recovers_power_law_with_constant():
    t_w = np.logspace(1, 6, 16)
    xi = 1.3 * t_w ** (1 / 10.0) - 0.4
    res = an.fit_z(t_w, xi)
    assert abs(res["z"] - 10.0) < 1e-6 and abs(res["c"] + 0.4) < 1e-6


def test_fit_x_and_mean_over_windows():
    t = 2.0 ** np.arange(0, 21)
    assert abs(an.fit_x(t, 0.8 * t ** -0.019, 100, 1e4) - 0.019) < 1e-12
    curves = [(t_w, t, 0.7 * t ** -0.019) for t_w in (1e6, 4e6, 2e7)]
    assert abs(an.fit_x_mean(curves) - 0.019) < 1e-12
    assert np.isnan(an.fit_x_mean([(1e4, t, t ** -0.1)]))  # window [100, 10] is empty
    # Sec. IV's window ends at t_w / 1000: a curve that bends right after it still gives x
    bent = []
    for t_w in (1e6, 4e6):
        end = t_w / 1000.0
        bent.append((t_w, t, 0.7 * t ** -0.019 * np.exp(-np.maximum(t / end - 1.0, 0.0))))
    assert abs(an.fit_x_mean(bent) - 0.019) < 1e-12


def test_collapse_finds_the_exponent():
    # with a constant term, as Sec. IV fits xi(t_w): then xi(t_w + t) / xi(t_w) is not a
    # function of t / t_w alone, and only the right scaling variable collapses the curves
    def xi_of_t(t):
        return 1.2 * np.asarray(t, dtype=np.float64) ** 0.1 + 0.5

    x_true = 0.016
    t = np.unique(np.round(np.logspace(0, 6, 60)))
    curves = []
    for t_w in (1e3, 1e4, 1e5):
        u = xi_of_t(t_w + t) / xi_of_t(t_w)
        C = t ** -x_true * np.exp(-3.0 * (u - 1.0))
        curves.append((t_w, t, C))
    x, cost = an.collapse_x(curves, xi_of_t)
    assert abs(x - x_true) < 1e-9 and cost < 1e-6  # what is left is interpolation error
    # a wrong exponent spreads the curves apart
    _, cost_off = an.collapse_x(curves, xi_of_t, x_grid=np.array([x_true + 0.01]))
    assert cost_off > 100 * cost


def test_overlap_histogram():
    N = 16 ** 3
    Q = np.array([N, -N, 0, 0, N // 2, -N // 2, 0, 0])  # q = 1, -1, 0, 0, 0.5, -0.5, 0, 0
    edges, p, n = an.overlap_histogram(Q, N, bins=4)
    assert n == 8 and np.allclose(edges, [-1, -0.5, 0, 0.5, 1])
    width = 0.5
    # bins [-1,-.5) [-.5,0) [0,.5) [.5,1]: counts 1, 1, 4, 2
    assert np.allclose(p * width * n, [1, 1, 4, 2])
    assert abs(np.sum(p) * width - 1.0) < 1e-12


@pytest.mark.gpu
def test_pipeline_on_measured_curves():
    """A side-32 run: the measured C4 curves feed the multifit, and the library's
    xi_1 equals the host estimator without tail on the same curve."""
    from paper_1411_5512_gb300 import build, job
    build.build()
    L, S = 32, 64
    tws = [16, 32, 64, 128]
    j = job.EAJob(L, 0.5, 21, S)
    j.set_schedule(tws, [0])
    j.quench(0.7)
    j.sweep(max(tws))
    curves = []
    r = np.arange(0, L // 2 + 1, dtype=np.float64)
    for tw in tws:
        m = j.measure(tw, 0)
        curves.append((r, m["C4"], m["C4_sem"]))
        assert abs(an.xi1_with_tail(r, m["C4"], m["r_cut"], L) - m["xi1"]) < 1e-9 * abs(m["xi1"])
    fit = an.multifit_c4(curves, r_min=3)
    assert np.isfinite(fit["alpha"]) and np.isfinite(fit["beta"])
    assert np.all(np.isfinite(fit["xi"])) and np.all(fit["xi"] > 0)
    # the error bars of Sec. IV from the all-vector point set of the same snapshots
    allv = []
    for tw in tws:
        rad = j.c4_radial(tw)
        keep = rad["r"] <= L // 2
        allv.append((rad["r"][keep], rad["C4"][keep], rad["C4_sem"][keep]))
        # the axis points are among the vectors: the r = 1 shell is the axis r = 1 mean
        m = j.measure(tw, 0)
        assert abs(rad["C4"][1] - m["C4"][1]) < 1e-12
    e = an.multifit_error(curves, allv)
    assert np.isfinite(e["alpha_err"]) and np.isfinite(e["beta_err"])
    assert np.all(np.isfinite(e["xi_err"]))
    j.close()


def test_multifit_error_combines_both_point_sets():
    """Both point sets built from the same form: the error is the sum of the two fits'
    statistical errors (the difference vanishes); a shifted second set adds the shift."""
    alpha, beta = 0.5, 1.4
    xis, As = [2.5, 3.5, 5.0], [1.0, 1.0, 1.0]
    axis = model_curves(alpha, beta, xis, As, rel_err=1e-3)
    # the all-vector set: irrational distances sqrt(r^2) of the same form
    r = np.sqrt(np.arange(0, 3 * 32 ** 2 + 1, dtype=np.float64))[:400]
    allv = []
    for xi, A in zip(xis, As):
        c = np.ones_like(r)
        c[1:] = an.c4_model(r[1:], A, alpha, xi, beta)
        allv.append((r, c, 1e-3 * np.abs(c) + 1e-12))
    e = an.multifit_error(axis, allv)
    assert abs(e["alpha"] - alpha) < 1e-6 and abs(e["beta"] - beta) < 1e-6
    fa, fb = e["fit_axis"], e["fit_all"]
    assert abs(e["alpha_err"] - (fa["alpha_err"] + fb["alpha_err"])) < 1e-6
    # a second set from a different alpha: the error covers the difference
    allv2 = [(r, an.c4_model(np.maximum(r, 1), A, alpha + 0.05, xi, beta), e_)
             for (r, _, e_), xi, A in zip(allv, xis, As)]
    e2 = an.multifit_error(axis, allv2)
    assert e2["alpha_err"] >= abs(e2["fit_all"]["alpha"] - alpha) - 1e-6
    # a second set with 5% longer xi: each xi error covers its difference
    allv3 = [(r, an.c4_model(np.maximum(r, 1), A, alpha, 1.05 * xi, beta), e_)
             for (r, _, e_), xi, A in zip(allv, xis, As)]
    e3 = an.multifit_error(axis, allv3)
    fa3, fb3 = e3["fit_axis"], e3["fit_all"]
    dxi = np.abs(fa3["xi"] - fb3["xi"])
    assert np.allclose(dxi, 0.05 * np.array(xis), rtol=1e-3)
    assert np.all(dxi > fa3["xi_err"] + fb3["xi_err"])  # the shift dominates the fit errors
    assert np.allclose(e3["xi_err"], dxi + fa3["xi_err"] + fb3["xi_err"], rtol=1e-12)
    assert abs(e2["fit_all"]["alpha"] - (alpha + 0.05)) < 1e-4


def test_pscan_analysis_on_synthetic_curves():
    """The p-scan's analysis recovers alpha, beta, z and x from curves built from the
    forms it fits, on the axis points and on every displacement vector."""
    from paper_1411_5512_gb300 import pscan
    L = 64
    alpha, beta, z_true, x_true = 0.45, 1.4, 8.0, 0.02
    r = np.arange(0, L // 2 + 1, dtype=np.float64)
    r_all = np.sqrt(np.arange(0, 3 * (L // 2) ** 2 + 1, dtype=np.float64))
    r_all = r_all[r_all <= L // 2]
    tws = [2 ** k for k in range(4, 20)]  # x needs t_w / 1000 above 100
    c4, c4_all, C = {}, {}, {}
    for tw in tws:
        xi = 1.1 * tw ** (1.0 / z_true)
        cur = np.ones_like(r)
        cur[1:] = an.c4_model(r[1:], 0.9, alpha, xi, beta)
        c4[tw] = (cur, 1e-3 * cur + 1e-9, L // 2)
        ca = np.ones_like(r_all)
        ca[1:] = an.c4_model(r_all[1:], 0.9, alpha, xi, beta)
        c4_all[tw] = (r_all, ca, 1e-3 * ca + 1e-9)
        for j in range(0, 20):
            C[(tw, 2 ** j)] = 0.7 * (2.0 ** j) ** (-x_true)
    rows = pscan.analyse(L, [{"pneg": 0.3, "c4": c4, "c4_all": c4_all, "C": C}])
    row = rows[0]
    assert row["pneg"] == 0.3 and abs(row["p"] - 0.7) < 1e-15  # the paper's p = 1 - p_neg
    assert abs(row["alpha"] - alpha) < 1e-4 and abs(row["beta"] - beta) < 1e-4
    assert abs(row["z_fit"] - z_true) < 1e-3
    assert abs(row["xi_fit_last"] - 1.1 * tws[-1] ** (1.0 / z_true)) < 1e-3  # the latest t_w
    assert abs(row["x"] - x_true) < 1e-9
    assert np.isfinite(row["alpha_err"]) and row["alpha_err"] < 1e-2
