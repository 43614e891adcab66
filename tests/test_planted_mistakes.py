"""The pins catch plausible mistakes.  Each case plants one mistake in a copy of the
code under test, on the CPU: a dropped term, a wrong sign, index, operand or
constant.  The tests that pin that code then run against the copy and must fail;
the unchanged copy must pass.  Two groups:

- the oracle (its C chain and its numpy observables) against the oracle's pins;
  the mistakes lie in the arithmetic the paper fixes (Eqs. 1-3, 5-7 and 9, the
  checkerboard of Sec. III, the heat-bath rule and the gap construction that
  realises both rules) and in the way the random-number mapping spends its bits
  (a lead shared by two classes or two words, overlapping bit fields, colliding
  or reused calls, a shifted coin), which must still give independent flips;
- the host analysis of Sec. IV (``analysis.py``) and the p-scan table built on it
  (``pscan.py``) against their tests.

Every copy lives in a temporary directory; the files under test are never modified.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")
PKG = os.path.join(ROOT, "paper_1411_5512_gb300")
ANALYSIS_PINS = os.path.join(ROOT, "tests", "test_analysis.py")

# (name, file in oracle/, text, replacement): the text must occur exactly once.
MUTANTS = [
    # Philox4x32-10 (SC'11): multiplier, key schedule, round count
    ("philox_multiplier", "ea_oracle.c", "0xD2511F53u * (uint64_t)c[0]", "0xD2511F55u * (uint64_t)c[0]"),
    ("philox_key_bump", "ea_oracle.c", "k[1] += 0xBB67AE85u;", "k[1] += 0xBB67AE86u;"),
    ("philox_nine_rounds", "ea_oracle.c", "for (int r = 0; r < 10; r++)", "for (int r = 0; r < 9; r++)"),
    # word-site geometry
    ("geometry_kz_cap", "ea_oracle.c", "int kz = p2 < 32 ? p2 : 32;", "int kz = p2 < 16 ? p2 : 16;"),
    ("geometry_block_origin", "ea_oracle.c", "sy[b] = ((b / kx) % ky) * Ly + yw;",
     "sy[b] = (((b / kx) % ky) * Ly + yw + 1) % L;"),
    # Eq. 9 and the heat-bath rule
    ("metropolis_sign", "ea_oracle.c", "P = exp(-(double)dE / T);", "P = exp((double)dE / T);"),
    ("metropolis_temperature_scale", "ea_oracle.c", "P = exp(-(double)dE / T);",
     "P = exp(-(double)dE / (2.0 * T));"),
    ("metropolis_dE_zero", "ea_oracle.c", "            if (dE <= 0)\n                P = 1.0;",
     "            if (dE < 0)\n                P = 1.0;"),
    ("heatbath_sign", "ea_oracle.c", "P = 1.0 / (1.0 + exp((double)dE / T));",
     "P = 1.0 / (1.0 + exp(-(double)dE / T));"),
    ("heatbath_gap_probability", "ea_oracle.c", "p = 1.0 / (1.0 + exp((double)(12 - 4 * u) / T));",
     "p = 1.0 / (1.0 + exp((double)(12 - 4 * u) / (2.0 * T)));"),
    # the local field dE = 2 S_i sum_j J_ij S_j
    ("field_drops_a_bond", "ea_oracle.c", "J[2 * N + izm] * Sa[izm];", "0;"),
    ("field_backward_bond_index", "ea_oracle.c", "J[0 * N + ixm] * Sa[ixm]", "J[0 * N + i] * Sa[ixm]"),
    ("field_direction_swap", "ea_oracle.c", "J[1 * N + i] * Sa[iyp]", "J[2 * N + i] * Sa[iyp]"),
    ("field_sign", "ea_oracle.c", "return 2 * Sa[i] * h_loc;", "return -2 * Sa[i] * h_loc;"),
    # the checkerboard of Sec. III
    ("colour_two_axes", "ea_oracle.c", "if (((xw + yw + zw) & 1) != (h ^ a))", "if (((xw + yw) & 1) != (h ^ a))"),
    # gaps: P(G >= g) = (1 - p)^g and the selection that follows
    ("gap_table_exponent", "ea_oracle.c", "double q = -expm1((double)g * log1p(-p));",
     "double q = -expm1((double)(g + 1) * log1p(-p));"),
    ("gap_skips_a_site", "ea_oracle.c", "start += G + 1;", "start += G + 2;"),
    ("gap_none_test", "ea_oracle.c", "if (V >= C[rem])", "if (V >= C[rem - 1])"),
    ("heatbath_coin_always", "ea_oracle.c", "return lanes & coin;", "return lanes;"),
    ("heatbath_keep_inverted", "ea_oracle.c", "return u < 3 ? mark : (lanes & ~mark);", "return mark;"),
    ("heatbath_wrong_pair", "ea_oracle.c", "int j = u < 3 ? u : 6 - u;", "int j = u < 3 ? u : u - 4;"),
    # the draw contract (draw64): how the random bits are spent must still give
    # independent fair bits and independent flips
    ("draw_lead_shared", "ea_oracle.c", "((uint64_t)((lead >> 10) & 0x3FFu) << 54)",
     "((uint64_t)((lead >> 22) & 0x3FFu) << 54)"),
    ("draw_quad_output", "ea_oracle.c", "uint32_t lead = out[ox + 2 * oz];", "uint32_t lead = out[ox + oz];"),
    ("draw_extension_overlap", "ea_oracle.c", "(join64(out[0], out[1]) >> 12)",
     "(join64(out[0], out[1]) >> 11)"),
    ("draw_continuation_off_by_one", "ea_oracle.c", "t, 1 + u + 3 * ((d - 1) / 2), out);",
     "t, u + 3 * ((d - 1) / 2), out);"),
    ("draw_continuation_drops_class", "ea_oracle.c", "t, 1 + u + 3 * ((d - 1) / 2), out);",
     "t, 1 + 3 * ((d - 1) / 2), out);"),
    ("draw_continuation_reused", "ea_oracle.c",
     "int e = (d - 1) % 2;\n            flip_call(STREAM_METROPOLIS",
     "int e = 0;\n            flip_call(STREAM_METROPOLIS"),
    ("coin_lane_shift", "ea_oracle.c", "return lanes & coin;", "return lanes & (coin >> 1);"),
    ("heat_pair_shared_lead", "ea_oracle.c", "uint32_t word = out[3 - pair];",
     "uint32_t word = out[1 + (pair & 1)];"),
    ("heat_keep_same_half", "ea_oracle.c", "uint64_t lead = u < 3 ? (word >> 16) : (word & 0xFFFFu);",
     "uint64_t lead = word >> 16;"),
    ("heat_continuation_drops_class", "ea_oracle.c", "1 + u + 7 * ((d - 1) / 2)", "1 + 7 * ((d - 1) / 2)"),
    ("energy_change_sign", "ea_oracle.c", "dE_acc[a] += dE[b];", "dE_acc[a] -= dE[b];"),
    # initial state
    ("couplings_inverted", "ea_oracle.c", "J[d * N + i] = ((uint64_t)out[d] < thr) ? (int8_t)-1 : (int8_t)1;",
     "J[d * N + i] = ((uint64_t)out[d] < thr) ? (int8_t)1 : (int8_t)-1;"),
    ("exact_count_truncated", "ea_oracle.c", "floor(p_neg * 3.0 * (double)N + 0.5)", "floor(p_neg * 3.0 * (double)N)"),
    ("replicas_share_start", "ea_oracle.c", "S[a * N + i] = (out[a] >> 31)", "S[a * N + i] = (out[0] >> 31)"),
    # observables (Eqs. 1-3, 5-7)
    ("overlap_one_replica", "ea_oracle.py", "np.sum(S[0].astype(np.int64) * S[1]))",
     "np.sum(S[0].astype(np.int64) * S[0]))"),
    ("autocorr_other_replica", "ea_oracle.py", "S_tw[a].astype(np.int64) * S_now[a]",
     "S_tw[a].astype(np.int64) * S_now[1 - a]"),
    ("axis_map_transposed", "ea_oracle.py", "_AXIS = {0: 2, 1: 1, 2: 0}", "_AXIS = {0: 0, 1: 1, 2: 2}"),
    ("energy_sign", "ea_oracle.py", "E[a] = -tot", "E[a] = tot"),
    ("c4_full_shift_axis", "ea_oracle.py", "qzy = np.roll(qz, -dy, axis=1)", "qzy = np.roll(qz, -dy, axis=0)"),
    ("radial_unfolded", "ea_oracle.py", "m2 = np.minimum(d, L - d) ** 2", "m2 = d ** 2"),
    ("c4_curve_sample_norm", "ea_oracle.py", "/ (3.0 * N * S)", "/ (3.0 * N)"),
    ("c4_sem_ddof", "ea_oracle.py", "std(axis=0, ddof=1)", "std(axis=0, ddof=0)"),
    ("cutoff_two_sigma", "ea_oracle.py", "if c4[r] < 3.0 * sem[r]:", "if c4[r] < 2.0 * sem[r]:"),
    ("xi1_moment", "ea_oracle.py", "I2 += r * r * c4[r]", "I2 += r * c4[r]"),
]

# Mistakes in the analysis of Sec. IV and the p-scan table built on it:
# (name, file in the package, text, replacement).
ANALYSIS_MUTANTS = [
    ("model_alpha_sign", "analysis.py", "r ** (-alpha)", "r ** (alpha)"),
    ("model_ratio_inverted", "analysis.py", "np.exp(-(r / xi) ** beta)", "np.exp(-(xi / r) ** beta)"),
    ("model_beta_dropped", "analysis.py", "np.exp(-(r / xi) ** beta)", "np.exp(-(r / xi))"),
    ("multifit_r_min_exclusive", "analysis.py", "keep = (r >= r_min) & (e > 0)", "keep = (r > r_min) & (e > 0)"),
    ("multifit_unweighted", "analysis.py", "out.append((c4_model(r, A, alpha, xi, beta) - c) / e)",
     "out.append((c4_model(r, A, alpha, xi, beta) - c))"),
    ("xi1_second_moment", "analysis.py", "I2 = float(np.sum(r[inside] ** 2 * C4[inside]))",
     "I2 = float(np.sum(r[inside] * C4[inside]))"),
    ("xi1_tail_repeats_r_c", "analysis.py", "rt = np.arange(int(r_c) + 1, L // 2 + 1", "rt = np.arange(int(r_c), L // 2 + 1"),
    ("xi1_tail_short", "analysis.py", "rt = np.arange(int(r_c) + 1, L // 2 + 1", "rt = np.arange(int(r_c) + 1, L // 2"),
    ("xi1_tail_moment", "analysis.py", "I2 += float(np.sum(rt ** 2 * ct))", "I2 += float(np.sum(rt * ct))"),
    ("z_without_constant", "analysis.py", "return a * t ** inv_z + c", "return a * t ** inv_z"),
    ("z_inverted", "analysis.py", 'return {"z": float(1.0 / inv_z)', 'return {"z": float(inv_z)'),
    ("x_sign", "analysis.py", "return float(-slope)", "return float(slope)"),
    ("x_window", "analysis.py", "fit_x(t, C, t_min, t_w / 1000.0)", "fit_x(t, C, t_min, t_w / 100.0)"),
    ("collapse_sign", "analysis.py", "np.log(C) + x * np.log(t)", "np.log(C) - x * np.log(t)"),
    ("collapse_variable", "analysis.py", "u = np.log(xi_of_t(t_w + t[keep]) / xi_of_t(t_w))",
     "u = np.log(xi_of_t(t[keep]) / xi_of_t(t_w))"),
    ("overlap_norm", "analysis.py", "q = np.asarray(Q, dtype=np.float64).ravel() / float(N)",
     "q = np.asarray(Q, dtype=np.float64).ravel() / float(2 * N)"),
    ("error_without_difference", "analysis.py", 'out[k + "_err"] = abs(fa[k] - fb[k]) + fa[k + "_err"] + fb[k + "_err"]',
     'out[k + "_err"] = fa[k + "_err"] + fb[k + "_err"]'),
    ("error_one_fit_only", "analysis.py", 'out[k + "_err"] = abs(fa[k] - fb[k]) + fa[k + "_err"] + fb[k + "_err"]',
     'out[k + "_err"] = abs(fa[k] - fb[k]) + fa[k + "_err"]'),
    ("xi_error_without_difference", "analysis.py", 'out["xi_err"] = np.abs(fa["xi"] - fb["xi"]) + fa["xi_err"] + fb["xi_err"]',
     'out["xi_err"] = fa["xi_err"] + fb["xi_err"]'),
    # the p-scan table built on the analysis
    ("pscan_p_convention", "pscan.py", '"p": 1.0 - cur["pneg"], "alpha": fit["alpha"]',
     '"p": cur["pneg"], "alpha": fit["alpha"]'),
    ("pscan_first_xi", "pscan.py", '"xi_fit_last": float(xi_fit[-1])', '"xi_fit_last": float(xi_fit[0])'),
    ("pscan_z_from_xi1", "pscan.py", 'zf = an.fit_z(np.array(tws, dtype=np.float64), xi_fit)["z"]',
     'zf = an.fit_z(np.array(tws, dtype=np.float64), xi_int)["z"]'),
]

_DRIVER = r"""
import sys
sys.path.insert(0, sys.argv[1])
import oracle
assert oracle.__file__.startswith(sys.argv[1]), oracle.__file__
oracle.lib()
import pytest
sys.exit(pytest.main([sys.argv[2], "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]))
"""


_ANALYSIS_DRIVER = r"""
import importlib.util
import os
import sys
sys.path.insert(0, sys.argv[3])
import paper_1411_5512_gb300 as pkg
for name in ("analysis", "pscan"):
    path = os.path.join(sys.argv[1], name + ".py")
    spec = importlib.util.spec_from_file_location("paper_1411_5512_gb300." + name, path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod
    spec.loader.exec_module(mod)
    setattr(pkg, name, mod)
import pytest
sys.exit(pytest.main([sys.argv[2], "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]))
"""


def _copy(dst, mutant):
    os.makedirs(os.path.join(dst, "oracle"))
    for f in ("__init__.py", "build.py", "ea_oracle.c", "ea_oracle.py"):
        shutil.copy(os.path.join(ORACLE, f), os.path.join(dst, "oracle", f))
    if mutant is None:
        return
    _, fname, old, new = mutant
    path = os.path.join(dst, "oracle", fname)
    with open(path) as f:
        src = f.read()
    assert src.count(old) == 1, "the planted text of %s must occur once" % mutant[0]
    with open(path, "w") as f:
        f.write(src.replace(old, new))


def _copy_analysis(dst, mutant):
    os.makedirs(dst)
    for fname in ("analysis.py", "pscan.py"):
        with open(os.path.join(PKG, fname)) as f:
            src = f.read()
        if mutant is not None and mutant[1] == fname:
            _, _, old, new = mutant
            assert src.count(old) == 1, "the planted text of %s must occur once" % mutant[0]
            src = src.replace(old, new)
        with open(os.path.join(dst, fname), "w") as f:
            f.write(src)
    return dst


def _run(args, cwd):
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    try:
        p = subprocess.run([sys.executable, "-c"] + args, cwd=cwd, env=env,
                           capture_output=True, text=True, timeout=300)
    except subprocess.TimeoutExpired:
        return None, "timed out"
    return p.returncode, p.stdout + p.stderr


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    base = tmp_path_factory.mktemp("oracle_mutants")
    jobs = {}
    for name, m in [("unchanged", None)] + [(m[0], m) for m in MUTANTS]:
        d = str(base / ("oracle_" + name))
        _copy(d, m)
        jobs["oracle:" + name] = ([_DRIVER, d, PINS], d)
    for name, m in [("unchanged", None)] + [(m[0], m) for m in ANALYSIS_MUTANTS]:
        d = str(base / ("analysis_" + name))
        path = _copy_analysis(d, m)
        jobs["analysis:" + name] = ([_ANALYSIS_DRIVER, path, ANALYSIS_PINS, ROOT], d)
    workers = max(1, min(8, (os.cpu_count() or 1)))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        futs = {key: ex.submit(_run, *job) for key, job in jobs.items()}
        return {key: f.result() for key, f in futs.items()}


def _failed_tests(log):
    return [ln.split(" ")[1] for ln in log.splitlines() if ln.startswith("FAILED ")]


@pytest.mark.parametrize("group", ["oracle", "analysis"])
def test_unchanged_copy_passes_the_pins(outcomes, group):
    rc, log = outcomes[group + ":unchanged"]
    assert rc == 0, log[-3000:]


@pytest.mark.parametrize("name", ["oracle:" + m[0] for m in MUTANTS] +
                         ["analysis:" + m[0] for m in ANALYSIS_MUTANTS])
def test_planted_mistake_fails_a_pin(outcomes, name):
    rc, log = outcomes[name]
    assert rc is not None, "%s: the pins did not finish" % name
    # exit status 1: tests ran and at least one failed (not a collection or usage error)
    assert rc == 1, "%s survived the pins (status %r)\n%s" % (name, rc, log[-3000:])
    assert _failed_tests(log), log[-3000:]
