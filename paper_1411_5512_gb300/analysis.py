"""Host FP64 analysis of the ageing observables (Sec. II, Sec. IV).

Everything here works on the exact integer sums that the library measures
(C4 curves with their errors, autocorrelations C(t, t_w)); it needs numpy and
scipy and runs on the host only.

- c4_model, multifit_c4: the functional form of the four-point correlation,
  C4(r, t_w) = A(t_w) r^-alpha exp(-(r / xi(t_w))^beta) (Eq. 4 with a stretched
  exponential g), fitted to the curves of all waiting times t_w >= 10 at once
  with common alpha and beta and one xi and amplitude per t_w (Sec. IV).
- xi1_with_tail: the integral estimator xi_1 = I_2 / I_1 (Eqs. 5-6, k = 1),
  summed over r = 1..r_c and continued beyond r_c up to L/2 with the fitted
  form, as Sec. IV does past the point where C4 falls below three errors.
- fit_z: xi(t_w) = a t_w^(1/z) + c, the power law with a constant term that
  Sec. IV fits.
- fit_x: C(t, t_w) proportional to t^-x on t in [t_min, t_w / 1000] (Eq. 8),
  averaged over t_w (Sec. IV).
- collapse_x: the x for which t^x C(t, t_w) plotted against
  xi(t_w + t) / xi(t_w) falls on one curve for all t_w (the multiplicative
  decomposition of Sec. II, tested in Sec. IV).
- overlap_histogram: P(q), the distribution of the replica overlap q = Q / N
  (Eq. 2) over samples and times.
- multifit_error: the error bars of Sec. IV: the same multifit on the axis
  points and on every displacement vector with r >= r_min (ea_c4_radial); the
  error of alpha, beta and each xi is the difference of the two results plus
  both statistical errors.
"""
import numpy as np


def c4_model(r, A, alpha, xi, beta):
    """A r^-alpha exp(-(r / xi)^beta)."""
    r = np.asarray(r, dtype=np.float64)
    return A * r ** (-alpha) * np.exp(-(r / xi) ** beta)


def multifit_c4(curves, r_min=3.0, alpha0=0.5, beta0=1.5):
    """Fit c4_model to several C4 curves at once, with common alpha and beta.

    curves: list of (r, C4, err) arrays, one per waiting time.  Points with
    r >= r_min and a positive error enter the weighted least squares.
    Returns a dict with alpha, beta, xi (per curve), A (per curve), their
    standard errors from the Jacobian at the optimum, and chi2 / dof.
    """
    from scipy.optimize import least_squares

    data = []
    for r, c, e in curves:
        r = np.asarray(r, dtype=np.float64)
        c = np.asarray(c, dtype=np.float64)
        e = np.asarray(e, dtype=np.float64)
        keep = (r >= r_min) & (e > 0) & np.isfinite(c)
        data.append((r[keep], c[keep], e[keep]))
    n = len(data)
    if n == 0 or any(len(d[0]) < 2 for d in data):
        raise ValueError("every curve needs at least two points with r >= r_min")

    # start: xi from where each curve falls to 1/e of its first point
    p0 = [alpha0, beta0]
    for r, c, _ in data:
        A0 = max(c[0], 1e-12) * r[0] ** alpha0
        below = np.nonzero(c < c[0] / np.e)[0]
        xi0 = r[below[0]] if len(below) else r[-1]
        p0 += [np.log(A0), np.log(max(xi0, 0.5))]

    def resid(p):
        alpha, beta = p[0], p[1]
        out = []
        for i, (r, c, e) in enumerate(data):
            A, xi = np.exp(p[2 + 2 * i]), np.exp(p[3 + 2 * i])
            out.append((c4_model(r, A, alpha, xi, beta) - c) / e)
        return np.concatenate(out)

    lo = [-5.0, 0.05] + [-np.inf, np.log(1e-3)] * n
    hi = [5.0, 10.0] + [np.inf, np.log(1e6)] * n
    res = least_squares(resid, np.array(p0), bounds=(lo, hi), x_scale="jac",
                        xtol=1e-14, ftol=1e-14, gtol=1e-14, max_nfev=20000)
    npts = sum(len(d[0]) for d in data)
    dof = max(npts - len(p0), 1)
    chi2 = float(np.sum(res.fun ** 2))
    try:
        cov = np.linalg.pinv(res.jac.T @ res.jac)
        se = np.sqrt(np.maximum(np.diag(cov), 0.0))
    except np.linalg.LinAlgError:
        se = np.full(len(p0), np.nan)
    p = res.x
    xi = np.exp(p[3::2])
    return {"alpha": float(p[0]), "beta": float(p[1]),
            "alpha_err": float(se[0]), "beta_err": float(se[1]),
            "xi": xi, "xi_err": xi * se[3::2],
            "A": np.exp(p[2::2]), "chi2_dof": chi2 / dof, "ok": bool(res.success)}


def xi1_with_tail(r, C4, r_c, L, fit=None):
    """xi_1 = I_2 / I_1 with I_k = sum_{r=1}^{r_c} r^k C4(r) + sum_{r=r_c+1}^{L/2} r^k
    C4_fit(r): the measured curve up to the cutoff r_c, the fitted form beyond it
    (fit = (A, alpha, xi, beta); None keeps the measured sums only)."""
    r = np.asarray(r, dtype=np.float64)
    C4 = np.asarray(C4, dtype=np.float64)
    inside = (r >= 1) & (r <= r_c)
    I1 = float(np.sum(r[inside] * C4[inside]))
    I2 = float(np.sum(r[inside] ** 2 * C4[inside]))
    if fit is not None and r_c < L // 2:
        rt = np.arange(int(r_c) + 1, L // 2 + 1, dtype=np.float64)
        ct = c4_model(rt, *fit)
        I1 += float(np.sum(rt * ct))
        I2 += float(np.sum(rt ** 2 * ct))
    return I2 / I1 if I1 != 0 else float("nan")


def fit_z(t_w, xi, xi_err=None):
    """xi(t_w) = a t_w^(1/z) + c; returns dict(z, a, c, z_err)."""
    from scipy.optimize import curve_fit

    t_w = np.asarray(t_w, dtype=np.float64)
    xi = np.asarray(xi, dtype=np.float64)
    sigma = None if xi_err is None else np.asarray(xi_err, dtype=np.float64)

    def f(t, a, inv_z, c):
        return a * t ** inv_z + c

    # start from the power law without constant through the end points
    inv_z0 = np.log(xi[-1] / xi[0]) / np.log(t_w[-1] / t_w[0]) if len(xi) > 1 else 0.1
    inv_z0 = float(np.clip(inv_z0, 1e-3, 2.0))
    a0 = xi[-1] / t_w[-1] ** inv_z0
    p, cov = curve_fit(f, t_w, xi, p0=[a0, inv_z0, 0.0], sigma=sigma,
                       absolute_sigma=sigma is not None, maxfev=20000)
    inv_z = p[1]
    inv_z_err = float(np.sqrt(cov[1, 1])) if np.all(np.isfinite(cov)) else float("nan")
    return {"z": float(1.0 / inv_z), "a": float(p[0]), "c": float(p[2]),
            "z_err": inv_z_err / inv_z ** 2}


def fit_x(t, C, t_min=100.0, t_max=None):
    """Power law C(t) proportional to t^-x on t_min <= t <= t_max (log-log line);
    returns x, or nan with fewer than two points in the window."""
    t = np.asarray(t, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    keep = (t >= t_min) & (C > 0)
    if t_max is not None:
        keep &= t <= t_max
    if np.count_nonzero(keep) < 2:
        return float("nan")
    slope, _ = np.polyfit(np.log(t[keep]), np.log(C[keep]), 1)
    return float(-slope)


def fit_x_mean(curves, t_min=100.0):
    """Mean of fit_x over waiting times, each on t in [t_min, t_w / 1000]
    (Sec. IV); curves: list of (t_w, t, C).  Waiting times whose window holds
    fewer than two points are skipped."""
    xs = [fit_x(t, C, t_min, t_w / 1000.0) for t_w, t, C in curves]
    xs = [x for x in xs if np.isfinite(x)]
    return float(np.mean(xs)) if xs else float("nan")


def collapse_x(curves, xi_of_t, x_grid=None):
    """The exponent x of the multiplicative decomposition C = C_eq(t) C_age with
    C_eq = t^-x and C_age a function of xi(t_w + t) / xi(t_w) alone: the x for
    which the curves t^x C(t, t_w) against log(xi(t_w + t) / xi(t_w)) collapse
    best (smallest spread between curves, by linear interpolation on their common
    range).  curves: list of (t_w, t, C); xi_of_t: callable.  Returns (x, cost)."""
    if x_grid is None:
        x_grid = np.linspace(0.0, 0.1, 1001)
    prepared = []
    for t_w, t, C in curves:
        t = np.asarray(t, dtype=np.float64)
        C = np.asarray(C, dtype=np.float64)
        keep = (t > 0) & (C > 0)
        u = np.log(xi_of_t(t_w + t[keep]) / xi_of_t(t_w))
        order = np.argsort(u)
        prepared.append((u[order], t[keep][order], C[keep][order]))

    def cost(x):
        ys = [(u, np.log(C) + x * np.log(t)) for u, t, C in prepared]
        total, count = 0.0, 0
        for i in range(len(ys)):
            for j in range(i + 1, len(ys)):
                ui, yi = ys[i]
                uj, yj = ys[j]
                lo, hi = max(ui[0], uj[0]), min(ui[-1], uj[-1])
                if hi <= lo:
                    continue
                grid = np.linspace(lo, hi, 32)
                d = np.interp(grid, ui, yi) - np.interp(grid, uj, yj)
                total += float(np.sum(d * d))
                count += len(grid)
        return total / count if count else float("inf")

    costs = np.array([cost(x) for x in x_grid])
    k = int(np.argmin(costs))
    return float(x_grid[k]), float(costs[k])


def overlap_histogram(Q, N, bins=2 * 16):
    """P(q) of the overlaps q = Q / N (Eq. 2): Q holds the exact integer overlaps of
    any set of samples and times.  Returns (bin edges on [-1, 1], density, count)."""
    q = np.asarray(Q, dtype=np.float64).ravel() / float(N)
    hist, edges = np.histogram(q, bins=bins, range=(-1.0, 1.0), density=True)
    return edges, hist, int(q.size)


def multifit_error(axis_curves, all_curves, r_min=3.0):
    """Sec. IV error estimate: fit the axis curves and the all-vector curves (each a
    list of (r, C4, err) per waiting time), then
    err(v) = |v_axis - v_all| + se_axis(v) + se_all(v) for alpha, beta and xi.
    Returns {"alpha", "beta", "xi": values of the axis fit, and their "*_err"}."""
    fa = multifit_c4(axis_curves, r_min=r_min)
    fb = multifit_c4(all_curves, r_min=r_min)
    out = {"alpha": fa["alpha"], "beta": fa["beta"], "xi": fa["xi"]}
    for k in ("alpha", "beta"):
        out[k + "_err"] = abs(fa[k] - fb[k]) + fa[k + "_err"] + fb[k + "_err"]
    out["xi_err"] = np.abs(fa["xi"] - fb["xi"]) + fa["xi_err"] + fb["xi_err"]
    out["fit_axis"], out["fit_all"] = fa, fb
    return out
