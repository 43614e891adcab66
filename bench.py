"""Throughput benchmark: checkerboard Metropolis sweeps of the 3D +-J EA model.

Workload (paper scale): L = 128 (N = 2,097,152), five jobs with p_neg in
{0.5, 0.4, 0.3, 0.2, 0.1} of 16 samples each, two replicas per sample, T = 0.7,
logarithmic measurement schedule.  A step is one window of sweeps over all 80
samples (both replicas), with the scheduled measurements that fall inside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  Under torchrun each rank runs its own
independent copy of the workload (weak scaling, no collective on the data path).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "spin flips/ns (ps/flip) at L=128 + % of roofline; batched vs plain; p50/p99"
UNIT = "flips/ns"
WORKLOAD = "L128_p0.5-0.1_S16x5_T0.7"


# ----------------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------------
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms.  Started ahead of
    the timed region; mark() and stop() bound the window whose samples count."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []       # (host time, fields)
        self.proc = None
        self.thread = None
        self.t0 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 9:
                self.rows.append((time.perf_counter(), parts))

    def mark(self):
        """The timed region starts now."""
        self.t0 = time.perf_counter()

    def stop(self):
        self.t1 = time.perf_counter()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        t0 = self.t0 if self.t0 is not None else float("-inf")
        t1 = getattr(self, "t1", float("inf"))
        rows = [r for t, r in self.rows if t0 <= t <= t1]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------------
# the CPU oracle on the host's cores (reference arm and cpu_baseline leg)
# ----------------------------------------------------------------------------------
def host_cpu():
    """(cores this process may use, CPU model name)."""
    try:
        n = len(os.sched_getaffinity(0))
    except Exception:
        n = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return n, model


def _oracle_worker(conn, cases):
    """One host process: the oracle's state of its samples, swept on request."""
    sys.path.insert(0, ROOT)
    import oracle as ora
    state = []
    for L, p_neg, seed, s, T, rule in cases:
        state.append([L, seed, s, ora.init_spins(L, seed, s), ora.init_couplings(L, p_neg, seed, s),
                      T, rule, 0])
    conn.send("ready")
    while True:
        n = conn.recv()
        if n is None:
            break
        for st in state:
            L, seed, s, S, J, T, rule, t = st
            ora.sweeps(L, seed, s, S, J, T, rule, t, n)
            st[7] = t + n
        conn.send(True)
    conn.close()


class OraclePool:
    """The oracle's samples spread over `procs` host processes (spawned), each
    sweeping its own samples; sweep(n) returns the wall time of the slowest."""

    def __init__(self, cases, procs):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        procs = max(1, min(procs, len(cases)))
        self.flips_per_sweep = sum(2 * c[0] ** 3 for c in cases)
        self.procs = procs
        self.conns, self.workers = [], []
        for k in range(procs):
            a, b = ctx.Pipe()
            w = ctx.Process(target=_oracle_worker, args=(b, cases[k::procs]), daemon=True)
            w.start()
            self.conns.append(a)
            self.workers.append(w)
        for c in self.conns:
            assert c.recv() == "ready"

    def sweep(self, n):
        t0 = time.perf_counter()
        for c in self.conns:
            c.send(n)
        for c in self.conns:
            c.recv()
        return time.perf_counter() - t0

    def close(self):
        for c in self.conns:
            c.send(None)
        for w in self.workers:
            w.join(timeout=30)


def _oracle_rate(cases, procs, sweeps):
    """flips/ns of the oracle over `cases` on `procs` processes: one untimed sweep,
    then `sweeps` timed ones."""
    pool = OraclePool(cases, procs)
    try:
        pool.sweep(1)
        dt = pool.sweep(sweeps)
    finally:
        pool.close()
    flips = pool.flips_per_sweep * sweeps
    return {"value": flips / (dt * 1e9), "ps_per_flip": dt * 1e12 / flips, "flips": flips,
            "seconds": dt, "cores": pool.procs}


def cpu_oracle_baseline(l128_sweeps=10, c2_sweeps=100):
    """The oracle timed on the host: single-thread and one process per sample on all
    cores, at side 128 (the 16 samples of the p_neg = 0.5 job) and at side 32 (the
    64 samples of the T = 0.6 job)."""
    from paper_1411_5512_gb300 import workloads

    n_cores, model = host_cpu()
    w = workloads.PAPER_SCALE[0]
    l128 = [(w["L"], w["p_neg"], w["seed"], s, w["T"], 0) for s in range(w["n_samples"])]
    c = workloads.SMALL[0]
    c2 = [(c["L"], c["p_neg"], c["seed"], s, c["T"], 0) for s in range(c["n_samples"])]
    all_128 = _oracle_rate(l128, n_cores, l128_sweeps)
    one_128 = _oracle_rate(l128, 1, l128_sweeps)
    all_c2 = _oracle_rate(c2, n_cores, c2_sweeps)
    one_c2 = _oracle_rate(c2[:8], 1, c2_sweeps)
    desc = "%d samples x 2 replicas of the L=%d p_neg=%.1f job (T=%.1f), %d sweeps"
    return {"value": all_128["value"], "unit": UNIT, "cores": all_128["cores"], "kind": "oracle",
            "ps_per_flip": all_128["ps_per_flip"],
            "sample": (desc % (w["n_samples"], w["L"], w["p_neg"], w["T"], l128_sweeps)) +
                      ", one process per sample on all host cores",
            "host": {"nproc": n_cores, "model": model},
            "single_thread": dict(one_128, sample=desc % (w["n_samples"], w["L"], w["p_neg"],
                                                           w["T"], l128_sweeps)),
            "c2": {"all_cores": dict(all_c2, sample=desc % (c["n_samples"], c["L"], c["p_neg"],
                                                            c["T"], c2_sweeps)),
                   "single_thread": dict(one_c2, sample=desc % (8, c["L"], c["p_neg"], c["T"],
                                                                c2_sweeps))}}


def run_reference(args, world, rank):
    """The oracle as it stands on the host's cores: each step one sweep of the 16
    samples of the side-128 p_neg = 0.5 job, one process per sample."""
    if rank != 0:
        return 0
    from paper_1411_5512_gb300 import workloads

    n_cores, model = host_cpu()
    w = workloads.PAPER_SCALE[0]
    cases = [(w["L"], w["p_neg"], w["seed"], s, w["T"], 0) for s in range(w["n_samples"])]
    per_step = max(1, args.ref_sweeps)
    pool = OraclePool(cases, n_cores)
    try:
        for _ in range(args.warmup):
            pool.sweep(per_step)
        times = [pool.sweep(per_step) for _ in range(args.steps)]
    finally:
        pool.close()
    tot = sum(times)
    flips = pool.flips_per_sweep * per_step * args.steps
    value = flips / (tot * 1e9)
    sample = ("%d steps x %d sweep(s) of the %d samples x 2 replicas of the L=128 p_neg=0.5 "
              "job, one process per sample on %d host cores" %
              (args.steps, per_step, w["n_samples"], pool.procs))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "L": 128,
                       "jobs": [x["p_neg"] for x in workloads.PAPER_SCALE], "samples": 80,
                       "replicas": 2, "rule": "metropolis", "rng_group": 1,
                       "sweeps_per_step": per_step,
                       "path": "the CPU oracle on the host's cores, each step a bounded sample "
                               "of the workload (cpu_baseline.sample)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                             "sample": sample, "host": {"nproc": n_cores, "model": model}},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------
# The roofline of the method, per flip (one attempted update of one site of one
# replica of one sample):
# - memory: a sweep must move the state across memory at least once: read 2
#   spin bits and 3 coupling bits, write 2 spin bits per site and sample, 7
#   bits per 2 flips = 0.4375 B/flip.  A pair of half-step kernels moves 12 bits
#   per 2 flips (0.75 B/flip); reported beside it.
# - integer ops: about 20 bit-logic ops per 32-site word (bond bits, bit-sliced
#   count, accept mask, flip) and about 90 per Philox4x32-10 call (ten rounds of
#   two wide multiplies, two three-input XORs and the key schedule), with the
#   calls per word counted on the live state; every op is priced at the measured
#   lop3.b32 rate of this GPU (ea_int_throughput).
# Thread instructions the side-128 tile kernel executes per attempted flip, from
# the ncu capture of profiles/metro_tile_kernel_L128_S128.md
# (sass__thread_inst_executed_true_per_opcode total 825.3 M over 268.4 M flips):
# what the kernel spends against the algorithmic ops of the ALU roof.
NCU_THREAD_INST_PER_FLIP = 825.3e6 / (128 * 128 ** 3)
BYTES_PER_FLIP = 7.0 / 16.0
BYTES_PER_FLIP_HALF_STEPS = 12.0 / 16.0
OPS_LOGIC_PER_WORD = 20
OPS_PER_PHILOX = 90
# DRAM bytes (read + write) of one batched half-step of this workload (the sum
# over its launches, one per stream group), keyed by (launch shape, streams):
# rows per thread 4, 8, 16 <-> --cpt 1, 2, 4.  From an ncu capture of this
# command with that fixed shape and stream count, taken with the caches warm as
# they are inside a step (--cache-control none, one pass: dram__bytes_read.sum +
# dram__bytes_write.sum, mean over consecutive half-steps).  Take them again
# (or drop the entry) when the kernel changes.
TRAFFIC_BYTES_PER_HALF_STEP = {(1, 1): 76.7e6 + 22.3e6, (2, 1): 80.0e6 + 25.5e6,
                               (4, 1): 83.8e6 + 29.2e6}
# With stream groups (streams > 1) the launches overlap, and ncu, which runs them
# one at a time, cannot capture their traffic: no entry, `traffic` is null.
# The same for the heat-bath tile kernel on the heat-bath leg.
HEAT_TRAFFIC_BYTES_PER_HALF_STEP = {(1, 1): 78.7e6 + 26.6e6, (2, 1): 79.3e6 + 26.4e6}


def timed_steps(stream, n_steps, step_fn, flush):
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(n_steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(n_steps)]
    for k in range(n_steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
            starts[k].record(stream)
            step_fn()
            ends[k].record(stream)
    stream.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)]


def pct(v, q):
    v = sorted(v)
    if not v:
        return None
    i = min(len(v) - 1, max(0, int(round(q / 100.0 * (len(v) - 1)))))
    return v[i]


def value_per_half_step(flips_per_half_step, kernel_ms):
    """flips and seconds per batched half-step (all samples; one launch per stream
    group, the groups side by side)."""
    return flips_per_half_step, kernel_ms * 1e-3


def traffic_bytes(args, batch_cfg):
    if args.traffic_bytes is not None:
        return args.traffic_bytes
    return TRAFFIC_BYTES_PER_HALF_STEP.get((batch_cfg[0], batch_cfg[2]))


def roofline(per_half_step, ops_per_flip, ipk, traffic, calls_per_word):
    """The binding roof of the half-step kernel and the others beside it.  HBM at the
    algorithmic 0.4375 B/flip against the measured copy bandwidth; integer ALU at
    the algorithmic ops per flip against the measured lop3.b32 rate."""
    flips, launch_s = per_half_step
    pk, pk_kind = peaks()
    rate = flips / launch_s  # flips/s
    hbm_roof = pk["hbm_gbs"] * 1e9 / BYTES_PER_FLIP
    alu_peak = ipk["lop3"]
    alu_roof = alu_peak / ops_per_flip
    hbm = {"bound": "hbm", "achieved": rate * BYTES_PER_FLIP / 1e9, "peak": pk["hbm_gbs"],
           "unit": "GB/s", "frac": rate / hbm_roof, "roof_flips_per_ns": hbm_roof / 1e9,
           "bytes_per_flip": BYTES_PER_FLIP,
           "peak_kind": "%s copy bandwidth (MEASURED_PEAKS.json)" % pk_kind}
    alu = {"bound": "alu", "achieved": rate * ops_per_flip / 1e12, "peak": alu_peak / 1e12,
           "unit": "Tops/s", "frac": rate / alu_roof, "roof_flips_per_ns": alu_roof / 1e9,
           "ops_per_flip": ops_per_flip, "philox_calls_per_word": calls_per_word,
           "ncu_thread_inst_per_flip": NCU_THREAD_INST_PER_FLIP,
           "peak_kind": "measured lop3.b32 rate of this GPU (ea_int_throughput)",
           "measured_rates": {"lop3_tops": ipk["lop3"] / 1e12, "imad_tops": ipk["imad"] / 1e12,
                              "philox_gcalls": ipk["philox"] / 1e9}}
    half = {"bound": "hbm", "bytes_per_flip": BYTES_PER_FLIP_HALF_STEPS,
            "achieved": rate * BYTES_PER_FLIP_HALF_STEPS / 1e9, "peak": pk["hbm_gbs"],
            "unit": "GB/s", "frac": rate * BYTES_PER_FLIP_HALF_STEPS / 1e9 / pk["hbm_gbs"],
            "roof_flips_per_ns": pk["hbm_gbs"] / BYTES_PER_FLIP_HALF_STEPS,
            "what": "the traffic of a pair of half-step kernels, for comparison"}
    primary, other = (hbm, alu) if hbm_roof <= alu_roof else (alu, hbm)
    roof = dict(primary)
    roof.update({"kernel": "metro_tile_kernel", "flips_per_half_step": flips,
                 "traffic": traffic,
                 "traffic_over_algorithmic": (None if traffic is None else
                                              traffic / (flips * BYTES_PER_FLIP)),
                 "binding": "%s roof %.0f flips/ns (HBM %.0f, integer ALU %.0f); with the "
                            "caches warm a half-step launch moves about 105 MB of DRAM" %
                            (primary["bound"], min(hbm_roof, alu_roof) / 1e9, hbm_roof / 1e9,
                             alu_roof / 1e9),
                 "other": other, "half_step_traffic": half})
    return roof


def run_ours(args, world, rank, local):
    import torch

    from paper_1411_5512_gb300 import job, shard, workloads

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    job.use_torch_allocator()
    stream = torch.cuda.Stream()
    specs = workloads.PAPER_SCALE
    L = specs[0]["L"]
    N = L ** 3
    sps = args.sweeps_per_step
    total_sweeps = (2 * args.warmup + 2 * args.steps + 64) * sps
    t_w = workloads.pow2_times(total_sweeps)
    t_lag = workloads.pow2_times(total_sweeps)

    jobs = []
    for w in specs:
        j = job.EAJob(w["L"], w["p_neg"], w["seed"] + 1000 * rank, w["n_samples"], stream=stream)
        j.set_schedule(t_w, t_lag)
        j.quench(w["T"])
        jobs.append(j)
    samples = sum(w["n_samples"] for w in specs)
    flips_per_step = sps * samples * 2 * N
    # L2 flush buffer (larger than the 126 MB L2), written between steps
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def plain_step():
        for j in jobs:
            j.sweep(sps)

    batch = job.EABatch(stream=stream)
    for j in jobs:
        batch.add(j)
    if args.cpt:
        batch.configure(args.cpt, args.graph_sweeps)
        if args.streams:
            batch.set_streams(args.streams)
        batch_cfg = (args.cpt, args.graph_sweeps, batch.streams())
    else:
        batch_cfg = tuple(batch.autotune(trial_sweeps=64)) + (batch.streams(),)

    def batched_step():
        batch.sweep(sps)

    sampler = ClockSampler(local)
    sampler.start()  # running before the timed region starts
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            batched_step()
    stream.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.mark()
    n_launch0 = job.launch_count()
    wall0 = time.perf_counter()
    step_ms = timed_steps(stream, args.steps, batched_step, flush)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    # the library's kernels enqueued in the timed region: sweep launches, the
    # time-advance kernel of each graph replay and the scheduled observables
    gpu_launches = job.launch_count() - n_launch0
    if world > 1:
        torch.distributed.barrier()
    sampler.stop()
    t_ms = shard.max_over_ranks(sum(step_ms), device="cuda")
    value = world * flips_per_step * args.steps / (t_ms * 1e6)
    # batched half-steps: each covers all 80 samples, in one launch per stream group
    launches = args.steps * 2 * sps
    kernel_ms = t_ms / launches  # incl. the rare observable and time-advance kernels

    # plain: the same work as separate per-job launch sequences (the paper's two
    # launches per sweep, one job at a time)
    batch.close()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            plain_step()
    plain_ms = timed_steps(stream, args.steps, plain_step, flush)
    plain_value = flips_per_step * args.steps / (sum(plain_ms) * 1e6)

    # Philox calls per word, counted on the live state by the counting variant
    batch = job.EABatch(stream=stream)
    for j in jobs:
        batch.add(j)
    prof = batch.profile(sweeps=4)
    batch.close()
    calls_per_word = prof["philox_calls"] / max(1, prof["words"])
    ops_per_flip = (OPS_LOGIC_PER_WORD + OPS_PER_PHILOX * calls_per_word) / 32.0
    ipk = job.int_throughput(stream)  # measured integer rates of this GPU
    roof = roofline(value_per_half_step(samples * N, kernel_ms), ops_per_flip, ipk,
                    traffic_bytes(args, batch_cfg), calls_per_word)
    roof["us_per_half_step"] = kernel_ms * 1e3
    roof["launches_per_half_step"] = min(batch_cfg[2], len(jobs))  # one per stream group

    # the paper's plain path: one sample per launch sequence, two launches per
    # sweep, over every sample of the workload
    plain1 = None
    if not args.no_plain_single:
        plain1 = run_plain_single(args, job, workloads, stream, flush, t_w, t_lag,
                                  jobs[0].time)

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, job, workloads, stream, rank, world, batch_cfg)
    serving = None
    if not args.no_serve:
        serving = run_serving(args, job, workloads, stream)
    mixed = None
    if not args.no_mixed:
        mixed = run_mixed(args, job, workloads, stream, flush)
    side32 = None
    if not args.no_mixed:
        side32 = run_side32(args, job, workloads, stream, flush)
    heat = None
    if not args.no_heat:
        heat = run_heat(args, job, workloads, stream, flush, ipk)
    c4r = None
    if not args.no_heat:
        c4r = run_c4_radial(args, job, workloads, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_oracle_baseline(args.cpu_l128_sweeps, args.cpu_c2_sweeps)

    for j in jobs:
        j.close()
    clocks = sampler.summary()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "ps_per_flip": 1e3 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "L": L,
                       "jobs": [w["p_neg"] for w in specs], "samples": samples, "replicas": 2,
                       "sweeps_per_step": sps, "rule": "metropolis", "rng_group": 1,
                       "path": "batched: each half-step of all 5 jobs is one launch per "
                               "stream group (the jobs split into batch_config.streams groups "
                               "on streams of their own)",
                       "batch_config": {"cols_per_thread": batch_cfg[0],
                                        "graph_sweeps": batch_cfg[1],
                                        "streams": batch_cfg[2]},
                       "l2": "flushed between steps (256 MiB write); inside a step nothing is "
                             "flushed, and a half-step still re-reads most of the 105 MB state "
                             "from DRAM (warm L2 sector hit rate 44%)"},
            "step_ms": {"p50": pct(step_ms, 50), "p99": pct(step_ms, 99)},
            "plain": {"value": plain_value, "unit": UNIT,
                      "path": "per-job launch sequences (16 samples per launch), 2 launches "
                              "per sweep per job",
                      "step_ms": {"p50": pct(plain_ms, 50), "p99": pct(plain_ms, 99)}},
            "batched_over_plain": value / plain_value,
            "roofline": roof, "clocks": clocks, "gpu_launches": gpu_launches, "wall_s": wall}
    if plain1 is not None:
        line["plain_single"] = plain1
        line["batched_over_plain_single"] = value / plain1["value"]
    if e2e is not None:
        line["e2e"] = e2e
    if serving is not None:
        line["serving"] = serving
    if mixed is not None:
        line["mixed_l"] = mixed
    if side32 is not None:
        line["side32"] = side32
    if heat is not None:
        line["heat_bath"] = heat
    if c4r is not None:
        line["c4_radial"] = c4r
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_plain_single(args, job, workloads, stream, flush, t_w, t_lag, t_now):
    """Every sample of the workload in a context of its own (its job's sample s,
    ea_create_samples_range), each swept by its own launch sequence, two launches per
    sweep: the paper's plain path.  The contexts are first brought to the batched
    jobs' time, so both see a lattice of the same age."""
    specs = workloads.PAPER_SCALE
    ctxs = []
    for w in specs:
        for s in range(w["n_samples"]):
            j = job.EAJob(w["L"], w["p_neg"], w["seed"], 1, stream=stream, first_sample=s)
            j.set_schedule(t_w, t_lag)
            j.quench(w["T"])
            ctxs.append(j)
    b = job.EABatch(stream=stream)
    for j in ctxs:
        b.add(j)
    b.sweep(t_now)
    b.close()
    sps = args.sweeps_per_step

    def step():
        for j in ctxs:
            j.sweep(sps)

    step()
    ms = timed_steps(stream, 3, step, flush)
    for j in ctxs:
        j.close()
    flips = sps * sum(2 * w["n_samples"] * w["L"] ** 3 for w in specs)
    m = statistics.median(ms)
    return {"value": flips / (m * 1e6), "unit": UNIT, "ms_per_step": m,
            "path": "one sample per launch sequence (80 contexts), 2 launches per sweep each"}


def run_side32(args, job, workloads, stream, flush):
    """The side-32 configuration (two jobs of 64 samples, T = 0.6 and 0.8) in one
    batch: sample-resident (one block per sample in shared memory, up to 1024 sweeps
    per launch) against one launch per half-step, median of three steps."""
    specs = workloads.SMALL
    jobs = []
    for w in specs:
        j = job.EAJob(w["L"], w["p_neg"], w["seed"], w["n_samples"], stream=stream)
        j.quench(w["T"])
        jobs.append(j)
    flips = args.side32_sweeps * sum(2 * w["n_samples"] * w["L"] ** 3 for w in specs)
    out = {"workload": "L32_S64x2_T0.6,0.8", "sweeps": args.side32_sweeps}
    for name, res in (("resident", 32), ("per_half_step", 0)):
        b = job.EABatch(stream=stream)
        for j in jobs:
            b.add(j)
        b.configure(0, 16)
        b.set_resident(res)
        b.sweep(4)
        ms = timed_steps(stream, 3, lambda: b.sweep(args.side32_sweeps), flush)
        b.close()
        m = statistics.median(ms)
        out[name] = {"value": flips / (m * 1e6), "unit": UNIT, "ms": m}
    for j in jobs:
        j.close()
    out["resident_over_per_half_step"] = out["resident"]["value"] / out["per_half_step"]["value"]
    return out


def run_mixed(args, job, workloads, stream, flush):
    """Mixed-L batch (364 single-sample jobs over L in {24, 48, 64, 96, 128}): the
    same sweeps as one batched launch per half-step vs per-job launch sequences."""
    import torch

    specs = workloads.mixed_l_jobs()
    jobs = []
    for w in specs:
        j = job.EAJob(w["L"], w["p_neg"], w["seed"], w["n_samples"], stream=stream)
        j.quench(w["T"])
        jobs.append(j)
    flips_per_sweep = sum(2 * w["n_samples"] * w["L"] ** 3 for w in specs)
    b = job.EABatch(stream=stream)
    for j in jobs:
        b.add(j)
    cfg = b.autotune(trial_sweeps=64)
    b_streams = b.streams()
    n_b = args.mixed_sweeps
    b.sweep(4)
    ms_b = timed_steps(stream, 3, lambda: b.sweep(n_b), flush)
    b.close()
    n_p = max(1, n_b // 8)

    def plain():
        for j in jobs:
            j.sweep(n_p)

    plain()
    ms_p = timed_steps(stream, 3, plain, flush)
    for j in jobs:
        j.close()
    mb, mp = statistics.median(ms_b), statistics.median(ms_p)
    vb = flips_per_sweep * n_b / (mb * 1e6)
    vp = flips_per_sweep * n_p / (mp * 1e6)
    return {"workload": workloads.MIXED_L["name"], "jobs": len(specs),
            "flips_per_sweep": flips_per_sweep,
            "batched": {"value": vb, "unit": UNIT, "sweeps": n_b, "ms": mb,
                        "cols_per_thread": cfg[0], "graph_sweeps": cfg[1],
                        "streams": b_streams},
            "plain": {"value": vp, "unit": UNIT, "sweeps": n_p, "ms": mp},
            "batched_over_plain": vb / vp}


def heat_alu_roof(value, prof, ipk):
    c = prof["philox_calls"] / max(prof["words"], 1)
    ops = (OPS_LOGIC_PER_WORD + OPS_PER_PHILOX * c) / 32.0
    roof = ipk["lop3"] / ops / 1e9  # flips/ns
    return {"ops_per_flip": ops, "roof_flips_per_ns": roof, "frac": value / roof,
            "peak_kind": "measured lop3.b32 rate of this GPU (ea_int_throughput)"}


def run_heat(args, job, workloads, stream, flush, ipk):
    """The heat-bath variant on the paper-scale workload (side 128, five jobs of 16
    samples, T = 0.7): batched, median of 3 steps of 64 sweeps, L2 flushed between.
    Its integer-ALU roof takes the same (20 + 90 c) / 32 ops per flip as the
    Metropolis one, with c its own Philox calls per word (one main call per word
    where the Metropolis path shares one per four)."""
    specs = workloads.PAPER_SCALE
    jobs = []
    for w in specs:
        j = job.EAJob(w["L"], w["p_neg"], w["seed"], w["n_samples"], stream=stream)
        j.quench(w["T"], 1)
        jobs.append(j)
    b = job.EABatch(stream=stream)
    for j in jobs:
        b.add(j)
    if args.cpt:  # a fixed launch shape (for a traffic capture of that shape)
        b.configure(args.cpt, args.graph_sweeps)
        if args.streams:
            b.set_streams(args.streams)
        cfg = (args.cpt, args.graph_sweeps, b.streams())
    else:
        cfg = tuple(b.autotune(trial_sweeps=64)) + (b.streams(),)
    prof = b.profile(sweeps=4)
    n = args.sweeps_per_step
    b.sweep(n)
    ms = timed_steps(stream, 3, lambda: b.sweep(n), flush)
    b.close()
    for j in jobs:
        j.close()
    flips = n * sum(2 * w["n_samples"] * w["L"] ** 3 for w in specs)
    m = statistics.median(ms)
    return {"workload": "L128_p0.5-0.1_S16x5_T0.7 heat bath", "value": flips / (m * 1e6),
            "unit": UNIT, "ms_per_step": m, "cols_per_thread": cfg[0], "graph_sweeps": cfg[1],
            "streams": cfg[2],
            "philox_calls_per_word": prof["philox_calls"] / max(prof["words"], 1),
            "alu_roof": heat_alu_roof(flips / (m * 1e6), prof, ipk),
            "hbm_frac_of_measured": flips / (m * 1e6) * 0.75 / peaks()[0]["hbm_gbs"],
            "traffic_per_half_step": HEAT_TRAFFIC_BYTES_PER_HALF_STEP.get((cfg[0], cfg[2])),
            "algorithmic_bytes_per_half_step":
                0.75 * sum(w["n_samples"] * w["L"] ** 3 for w in specs)}


def run_c4_radial(args, job, workloads, stream):
    """The four-point sums over every displacement vector of a side-128 job of 16
    samples (one snapshot): wall time of the synchronous call, per sample."""
    w = workloads.PAPER_SCALE[0]
    j = job.EAJob(w["L"], w["p_neg"], w["seed"], w["n_samples"], stream=stream)
    j.set_schedule([0], [0])
    j.quench(w["T"])
    j.c4_radial(0)  # warm-up
    reps = []
    for _ in range(3):
        t0 = time.perf_counter()
        j.c4_radial(0)
        reps.append(time.perf_counter() - t0)
    j.close()
    ms = statistics.median(reps) * 1e3
    return {"workload": "L128_S16 one snapshot", "ms": ms, "ms_per_sample": ms / w["n_samples"]}


def run_serving(args, job, workloads, stream):
    """Continuous batching of a seeded Poisson stream of ageing jobs (rate 50/s,
    L in {16, 32, 64, 128}, p_neg in [0.1, 0.5], T in [0.5, 1.0], sweeps
    log-uniform in [1e3, 1e6]), admitted by footprint.  Latency = completion
    (results read back on the host) minus the job's scheduled arrival."""
    import numpy as np
    import torch

    specs = workloads.serving_stream(args.serve_jobs)
    srv = job.EAServer(budget_bytes=args.serve_budget_gb << 30, max_running=256,
                       chunk_sweeps=args.serve_chunk, stream=stream)
    t_sched = [0, 1, 2, 4, 8, 16, 32, 64, 128, 256, 512]
    arrival = {}
    sweeps_of = {}
    lat = []
    lat_k = []  # completion latency per 10^3 sweeps of the job
    flips = 0
    nxt = 0
    open_ids = []
    t0 = time.perf_counter()
    while len(lat) < len(specs):
        now = time.perf_counter() - t0
        while nxt < len(specs) and specs[nxt]["arrival"] <= now:
            sp = specs[nxt]
            jid = srv.submit(sp["L"], sp["p_neg"], sp["seed"], sp["n_samples"], sp["T"],
                             sp["sweeps"], t_w=t_sched, t=t_sched)
            arrival[jid] = sp["arrival"]
            sweeps_of[jid] = sp["sweeps"]
            flips += sp["sweeps"] * 2 * sp["n_samples"] * sp["L"] ** 3
            open_ids.append(jid)
            nxt += 1
        st = srv.stats()
        if st["running"] == 0 and st["queued"] == 0:
            if nxt < len(specs):
                time.sleep(max(0.0, specs[nxt]["arrival"] - now))
            continue
        srv.step()
        still = []
        for jid in open_ids:
            state, _ = srv.state(jid)
            if state == 2:
                srv.job(jid).measure(0, 512)  # reads the results back (synchronises)
                lat.append(time.perf_counter() - t0 - arrival[jid])
                lat_k.append(lat[-1] / (sweeps_of[jid] / 1e3))
                srv.release(jid)
            else:
                still.append(jid)
        open_ids = still
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    srv.close()
    lat = np.array(lat)
    lat_k = np.array(lat_k)
    return {"workload": workloads.SERVING["name"], "jobs": len(specs),
            "rate_per_s": workloads.SERVING["rate"], "chunk_sweeps": args.serve_chunk,
            "latency_s": {"p50": float(np.percentile(lat, 50)),
                          "p99": float(np.percentile(lat, 99)),
                          "max": float(lat.max())},
            "latency_s_per_1e3_sweeps": {"p50": float(np.percentile(lat_k, 50)),
                                         "p99": float(np.percentile(lat_k, 99))},
            "flips": int(flips), "wall_s": wall, "value": flips / (wall * 1e9), "unit": UNIT}


def run_e2e(args, job, workloads, stream, rank, world, batch_cfg):
    """Whole jobs through the public API with their inputs from host memory: create,
    the couplings of every sample uploaded from a pinned host buffer (the packed
    layout), the schedule from host arrays, quench, sweeps of all five jobs together
    in one batch, and every scheduled observable read back to host."""
    import numpy as np
    import torch

    specs = workloads.PAPER_SCALE
    n = args.e2e_sweeps
    t_w = workloads.pow2_times(n)
    t_lag = workloads.pow2_times(n)
    # the inputs, prepared once outside the timed region: each job's couplings
    # (drawn from its seed) in pinned host memory
    inputs = []
    for w in specs:
        j = job.EAJob(w["L"], w["p_neg"], w["seed"] + 7 + 1000 * rank, w["n_samples"],
                      stream=stream)
        words = j.coupling_words()
        pinned = torch.empty(words.size, dtype=torch.int32, pin_memory=True)
        pinned.numpy().view(np.uint32)[:] = words
        inputs.append(pinned)
        j.close()
    h2d = sum(4 * x.numel() for x in inputs) + 8 * (len(t_w) + len(t_lag)) * len(specs)
    d2h = 0

    def one():
        nonlocal d2h
        d2h = 0
        jobs = []
        for w, words in zip(specs, inputs):
            j = job.EAJob(w["L"], w["p_neg"], w["seed"] + 7 + 1000 * rank, w["n_samples"],
                          stream=stream)
            j.set_coupling_words(words)
            j.set_schedule(t_w, t_lag)
            j.quench(w["T"])
            jobs.append(j)
        b = job.EABatch(stream=stream)  # the jobs' sweeps share launches
        # the launch configuration the batched leg's autotuner found for these jobs
        b.configure(batch_cfg[0], batch_cfg[1])
        b.set_streams(batch_cfg[2])
        for j in jobs:
            b.add(j)
        b.sweep(n)
        b.close()
        for j in jobs:
            for a in t_w:
                for c in t_lag:
                    if a + c <= n:
                        m = j.measure(a, c)
                        d2h += sum(m[k].nbytes for k in ("A", "Q", "E", "G"))
            j.close()

    one()  # warm
    torch.cuda.synchronize()
    reps = max(1, args.e2e_steps)
    t0 = time.perf_counter()
    for _ in range(reps):
        one()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    samples = sum(w["n_samples"] for w in specs)
    flips = reps * n * samples * 2 * 128 ** 3
    return {"value": world * flips / (dt * 1e9), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "sweeps_per_step": n, "steps": reps,
            "includes": "create, couplings H2D from pinned host memory, schedule H2D, quench, "
                        "batched sweeps, all observables D2H, destroy"}


def run_case(args):
    """A small, self-contained run of the sweep kernels, for profiling: one job of
    --case-samples samples at side --case-L (p_neg = 0.5, T = --case-T), quenched
    and swept --case-sweeps times through a one-job batch with launch shape --cpt
    (or the plain path with --case-plain).  At side 128 and 128 samples the state
    is 168 MB, above the 126 MB L2, so DRAM counters stay meaningful while the
    device footprint stays small."""
    import torch

    from paper_1411_5512_gb300 import job

    torch.cuda.set_device(0)
    j = job.EAJob(args.case_L, 0.5, 100, args.case_samples)
    if args.case_measure:
        j.set_schedule([0, 1, 2, 4], [0, 1, 2, 4])
    elif args.case_c4_radial:
        j.set_schedule([args.case_sweeps], [0])
    j.quench(args.case_T, args.case_rule)
    if args.case_plain:
        j.sweep(args.case_sweeps)
    else:
        b = job.EABatch()
        b.configure(args.cpt, 0)
        if args.case_variant >= 0:
            b.set_variant(args.case_variant)
        if args.case_resident >= 0:
            b.set_resident(args.case_resident)
        b.add(j)
        b.sweep(args.case_sweeps)
        b.close()
    if args.case_c4_radial:
        j.c4_radial(args.case_sweeps)
    torch.cuda.synchronize()
    print("case ok: L=%d S=%d t=%d" % (args.case_L, args.case_samples, j.time))
    j.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sweeps-per-step", type=int, default=64)
    ap.add_argument("--e2e-sweeps", type=int, default=1024)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-l128-sweeps", type=int, default=10)
    ap.add_argument("--cpu-c2-sweeps", type=int, default=100)
    ap.add_argument("--ref-sweeps", type=int, default=1)
    ap.add_argument("--no-plain-single", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpt", type=int, default=0, choices=[0, 1, 2, 4],
                    help="fixed launch shape of the batched path instead of the autotuned one")
    ap.add_argument("--graph-sweeps", type=int, default=8)
    ap.add_argument("--streams", type=int, default=0, choices=[0, 1, 2, 3, 4, 5],
                    help="with --cpt: the batch's stream groups (0: the library's default)")
    ap.add_argument("--traffic-bytes", type=float, default=None,
                    help="DRAM bytes per half-step launch from an ncu capture of this command")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-heat", action="store_true")
    ap.add_argument("--mixed-sweeps", type=int, default=64)
    ap.add_argument("--side32-sweeps", type=int, default=512)
    ap.add_argument("--serve-jobs", type=int, default=200)
    ap.add_argument("--serve-chunk", type=int, default=1024)
    ap.add_argument("--serve-budget-gb", type=int, default=64)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--case", action="store_true",
                    help="a small profiling run of the sweep kernels instead of the benchmark")
    ap.add_argument("--case-L", type=int, default=128)
    ap.add_argument("--case-samples", type=int, default=128)
    ap.add_argument("--case-sweeps", type=int, default=4)
    ap.add_argument("--case-rule", type=int, default=0)
    ap.add_argument("--case-T", type=float, default=0.7)
    ap.add_argument("--case-plain", action="store_true")
    ap.add_argument("--case-c4-radial", action="store_true")
    ap.add_argument("--case-measure", action="store_true",
                    help="schedule t_w = t = {0, 1, 2, 4} (the observable kernels fire)")
    ap.add_argument("--case-variant", type=int, default=-1,
                    help="side-128 Metropolis kernel: 0 tile, 1 staged (-1: the default)")
    ap.add_argument("--case-resident", type=int, default=-1,
                    help="largest side run sample-resident (-1: the default)")
    args = ap.parse_args()
    if args.case:
        return run_case(args)
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
