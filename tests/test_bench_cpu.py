"""The benchmark's reference arm runs on the host (the CPU oracle on a bounded sample,
one process per sample on the host's cores) and prints the one JSON line of the
benchmark contract; the roofline helper reports the lower roof."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3", "--ref-sweeps", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "flips/ns" and d["higher_is_better"] is True
    assert d["config"]["workload"] == "L128_p0.5-0.1_S16x5_T0.7"
    cb = d["cpu_baseline"]
    n_cores = len(os.sched_getaffinity(0))
    assert cb["kind"] == "oracle" and cb["value"] == d["value"]
    assert cb["cores"] == min(n_cores, 16) and cb["host"]["nproc"] == n_cores
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_roofline_reports_the_lower_roof():
    sys.path.insert(0, ROOT)
    import bench
    pk, _ = bench.peaks()
    flips, launch_s = 167772160, 30e-6
    ipk = {"lop3": 18.7e12, "imad": 9e12, "philox": 5e11}
    r = bench.roofline((flips, launch_s), 1.4, ipk, None, 0.28)
    hbm_roof = pk["hbm_gbs"] * 1e9 / bench.BYTES_PER_FLIP
    alu_roof = ipk["lop3"] / 1.4
    assert r["bound"] == ("hbm" if hbm_roof <= alu_roof else "alu")
    assert abs(r["frac"] - (flips / launch_s) / min(hbm_roof, alu_roof)) < 1e-12
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    assert r["other"]["bound"] != r["bound"]
    assert abs(r["half_step_traffic"]["bytes_per_flip"] - 0.75) < 1e-15
    assert abs(bench.BYTES_PER_FLIP - 0.4375) < 1e-15


def test_heat_bath_alu_roof():
    """(20 + 90 c) / 32 ops per flip with the heat bath's own Philox calls per word c,
    priced at the measured lop3 rate."""
    sys.path.insert(0, ROOT)
    import bench
    ipk = {"lop3": 19.7e12, "imad": 19.9e12, "philox": 4.4e11}
    prof = {"words": 1000, "philox_calls": 1110}
    r = bench.heat_alu_roof(4633.0, prof, ipk)
    ops = (20 + 90 * 1.11) / 32
    assert abs(r["ops_per_flip"] - ops) < 1e-12
    assert abs(r["roof_flips_per_ns"] - 19.7e12 / ops / 1e9) < 1e-9
    assert abs(r["frac"] - 4633.0 / r["roof_flips_per_ns"]) < 1e-12
