"""Benchmark of the multi-spin Ising Metropolis path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Workload (default): the large-lattice configuration, L = 16384 (2.7e8 spins,
~103 MB packed), T = 2.269, hot start with seed 3, E and M recorded every 10
sweeps.  One step = 10 sweeps (20 half-sweep launches) + one E/M record read
back to the host; 100 steps = the configuration's 1000 sweeps.  The packed
lattice fits in L2 (129 MB), so L2 is flushed (a 256 MB write) between timed
steps, outside the per-step CUDA events.

The JSON line (rank 0) reports spin-updates/ns: `value` from per-step CUDA
events on the lattice's stream with the lattice resident in HBM, `e2e` from
wall-clock steps through the C ABI that upload the spins from pinned host
memory (ising_set_spins) and read E/M back, `roofline` for the half-sweep
kernel, and `cpu_baseline` = the oracle on a bounded sample.

N > 1: one process per GPU, each an independent replica (own seed); the
path has no exchange step on one GPU's lattice, so there is no collective on
the data path (weak scaling).

--impl reference times the oracle (plain single-threaded C) on the host on a
bounded sample of the same workload: each step is one sweep of an L = 2048
lattice at the same temperature (the oracle's cost per update does not depend
on L, and the run stays within minutes for any --steps value).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L_LARGE = 16384
SEED_LARGE = 3
BETA = 1.0 / 2.269
SWEEPS_PER_STEP = 10
METRIC = "spin-updates/ns"
NOMINAL_SM_MAX_MHZ = 2070.0     # used only if neither nvidia-smi nor MEASURED_PEAKS.json gives the clock
# DRAM bytes (read + write) per half-sweep launch of the current kernel at
# L = 16384, from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum);
# None for other sizes and the 7-round scheme.
MEASURED_TRAFFIC = {16384: 1.103e8}
MULWIDE_PER_SITE = 4            # Philox4x32-10 with the counter-independent rounds hoisted:
                                # 16 multiplies per call, one call per 4 sites (10 per call,
                                # 2.5 per site, for the opt-in 7-round scheme)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-csv", default=None, help="directory for the raw nvidia-smi clock samples")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the plain-vs-batched comparison")
    ap.add_argument("--tiling", default=None, help="rows,block_words,block_groups")
    ap.add_argument("--L", type=int, default=L_LARGE, help="lattice side (profiling of a smaller case)")
    ap.add_argument("--workload", default="large",
                    choices=["large", "plain", "scan", "batched", "serving", "paper", "midsize"],
                    help="large (default): L=16384 roofline config; plain: L=64 x 1000 sweeps; "
                         "scan: L=1024 x 26 temperatures; batched: 512 uneven replicas vs per-instance launches; "
                         "paper: the paper's three test cases (Table 2) in both word layouts; "
                         "midsize: L = 296 .. 1008 on the cluster path and on the graph replays")
    ap.add_argument("--sweeps", type=int, default=None, help="override the workload's sweep count")
    ap.add_argument("--rng", type=int, default=10, choices=[10, 7],
                    help="Philox rounds of the sweep draws: 10 (default scheme) or the opt-in 7")
    ap.add_argument("--rate", type=float, default=200.0,
                    help="serving: mean arrival rate of the Poisson request stream (req/s)")
    ap.add_argument("--instances", type=int, default=None,
                    help="batched: compare with per-instance launches on the first N replicas only")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    # where the raw samples go: --clocks-csv DIR, else the system temp directory
    csv_dir = None

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        import tempfile
        d = ClockSampler.csv_dir or tempfile.gettempdir()
        os.makedirs(d, exist_ok=True)
        self.path = os.path.join(d, f"clocks_rank{self.gpu}.csv")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(L: int, sweeps: int, beta: float, seed: int):
    """Time `sweeps` oracle sweeps of an L x L hot-start lattice (init excluded)."""
    import oracle
    oracle.build()
    s = oracle.init_hot(L, seed)
    t0 = time.perf_counter()
    oracle.run(s, seed, beta, 0, sweeps, sweeps)
    dt = time.perf_counter() - t0
    return sweeps * L * L / (dt * 1e9), dt


def host_cpu() -> str:
    """CPU model and logical core count of this host, for the baseline lines."""
    import platform
    import subprocess
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return f"{model or platform.processor() or platform.machine()} x {os.cpu_count()}"


def _oracle_worker(job):
    """One host core: `sweeps` oracle sweeps of one lattice, E/M every sweep
    (init excluded); returns (spin updates, seconds)."""
    L, seed, beta, hot, sweeps = job
    import oracle
    s = oracle.init_hot(L, seed) if hot else oracle.init_cold(L, 1)
    t0 = time.perf_counter()
    oracle.run(s, seed, beta, 0, sweeps, 1)
    return L * L * sweeps, time.perf_counter() - t0


def oracle_all_cores(jobs):
    """The oracle on all host cores at once, one independent lattice per core
    (a spawn-context pool: no worker inherits the parent's CUDA state).
    Returns the aggregate rate (sum of the concurrent per-core rates) and the
    per-core mean, in spin-updates/ns."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = pool.map(_oracle_worker, jobs)
    rates = [u / (dt * 1e9) for u, dt in res]
    return sum(rates), sum(rates) / len(rates)


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build()
    L = 2048          # a bounded sample: ~0.13 s of oracle work per step
    s = oracle.init_hot(L, SEED_LARGE)
    t = 0
    for _ in range(args.warmup):
        t += 1
        oracle.sweep(s, SEED_LARGE, t, BETA)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        t += 1
        oracle.sweep(s, SEED_LARGE, t, BETA)
    dt = time.perf_counter() - t0
    value = args.steps * L * L / (dt * 1e9)
    sample = f"one oracle sweep of an L={L} hot-start lattice (seed {SEED_LARGE}, T=2.269) per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": "large: L=16384 periodic Ising, T=2.269, hot start seed 3, E/M every 10 sweeps",
                   "reference_step": sample},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample,
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def splitmix64(x: int) -> int:
    """SplitMix64 output for state x (Steele, Lea, Flood 2014): per-replica seeds."""
    z = (x + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


def batched_replicas(n=512, seed=11):
    """The batched configuration: L uniform on {32..2048} (powers of two), T
    uniform on [1.5, 3.5] (numpy default_rng(seed)), hot starts with seed
    SplitMix64(seed * 2^32 + r)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    Ls = rng.choice([32, 64, 128, 256, 512, 1024, 2048], size=n).astype(np.int32)
    Ts = rng.uniform(1.5, 3.5, size=n)
    seeds = np.array([splitmix64((seed << 32) + r) for r in range(n)], dtype=np.uint64)
    return Ls, 1.0 / Ts, seeds


def max_over_ranks(values, world, device="cuda"):
    """Element-wise maximum of per-rank timings (seconds) over all ranks; the
    whole-job time of a weak-scaling run is the slowest rank's."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_rate(units_per_rank, world, seconds):
    """Units per nanosecond of the whole job: every rank did units_per_rank in
    at most `seconds`."""
    return world * units_per_rank / (seconds * 1e9)


def emit(line):
    print(json.dumps(line), flush=True)


def batched_summary(ising, sweeps=5000, instances=32):
    """The batched configuration in one batch, and the same replicas (first
    `instances`) as per-instance ising_sweep_record calls, bit-compared."""
    import numpy as np
    import torch
    Ls, betas, seeds = batched_replicas()
    n = len(Ls)
    with ising.Batch([32], [0.4], [1], [1]) as warm:
        warm.sweep([10], every=1)
    b = ising.Batch(Ls, betas, seeds, np.ones(n, dtype=np.uint8))
    from paper_1811_04384_gb300 import tuning
    tuning.apply_batch(b, "batched512")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    E, M = b.sweep(sweeps, every=1)
    dt_b = time.perf_counter() - t0
    b.close()
    exact = True
    upd_k = 0.0
    t0 = time.perf_counter()
    for r in range(instances):
        with ising.Lattice(int(Ls[r]), int(seeds[r])) as lat:
            lat.init_hot()
            lat.set_beta(float(betas[r]))
            Ep, Mp = lat.sweep_record(sweeps, 1)
        exact &= bool(np.array_equal(Ep, E[r]) and np.array_equal(Mp, M[r]))
        upd_k += float(Ls[r]) ** 2 * sweeps
    dt_p = time.perf_counter() - t0
    v_b = float(np.sum(Ls.astype(np.float64) ** 2)) * sweeps / (dt_b * 1e9)
    v_p = upd_k / (dt_p * 1e9)
    return {"value": v_b, "unit": METRIC, "replicas": n, "sweeps": sweeps,
            "per_instance_value": v_p, "per_instance_replicas": instances,
            "batched_over_per_instance": v_b / v_p, "bit_exact": exact,
            "timing": "wall clock around ising_batch_sweep / each ising_sweep_record (both synchronise)"}


BATCH_LANES = 4      # ising_batch default: independent graph branches


def batch_launches(n_replicas: int, sweeps: int, chunk: int = 50) -> int:
    """Kernels one ising_batch_sweep launches: two half-sweeps per sweep per
    non-empty lane, one chunk-counter advance per replayed graph."""
    lanes = min(BATCH_LANES, n_replicas)
    return 2 * sweeps * lanes + (sweeps + chunk - 1) // chunk


def run_batched(args, ising, local):
    import numpy as np
    import torch
    from paper_1811_04384_gb300 import tuning
    Ls, betas, seeds = batched_replicas()
    n = len(Ls)
    sweeps = args.sweeps or 5000
    with ising.Batch([32], [0.4], [1], [1]) as warm:      # loads the kernels, captures a graph once
        warm.sweep([10], every=1)
    b = ising.Batch(Ls, betas, seeds, np.ones(n, dtype=np.uint8))
    tuned = tuning.apply_batch(b, "batched512")
    updates = float(np.sum(Ls.astype(np.float64) ** 2)) * sweeps
    with ClockSampler(local) as clocks:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        E, M = b.sweep(sweeps, every=1)
        torch.cuda.synchronize()
        dt_b = time.perf_counter() - t0
    k = args.instances or n
    t0 = time.perf_counter()
    exact = True
    upd_k = 0.0
    for r in range(k):
        with ising.Lattice(int(Ls[r]), int(seeds[r])) as lat:
            lat.init_hot()
            lat.set_beta(float(betas[r]))
            Ep, Mp = lat.sweep_record(sweeps, 1)
        exact &= bool(np.array_equal(Ep, E[r]) and np.array_equal(Mp, M[r]))
        upd_k += float(Ls[r]) ** 2 * sweeps
    dt_p = time.perf_counter() - t0
    b.close()
    cpu = None
    if not args.no_cpu_baseline:
        cores = min(os.cpu_count() or 1, n)
        jobs = [(int(Ls[r]), int(seeds[r]), float(betas[r]), True, max(1, int(round(1e8 / float(Ls[r]) ** 2))))
                for r in range(cores)]
        cpu_rate, cpu_core = oracle_all_cores(jobs)
        cpu = {"value": cpu_rate, "unit": METRIC, "cores": cores, "kind": "oracle", "per_core": cpu_core,
               "host": host_cpu(),
               "sample": f"replicas 0..{cores - 1} of the batch, one per host core, concurrently, about 1e8 "
                         "spin updates each (E/M every sweep)"}
    emit({"metric": METRIC, "value": updates / (dt_b * 1e9), "unit": METRIC, "n_gpus": 1, "steps": 1,
          "warmup": 1, "ms_per_step": dt_b * 1e3, "higher_is_better": True, "scaling": "weak",
          "vs_baseline": None, "dtype": "u64", "data": "synthetic",
          "config": {"workload": f"batched: {n} replicas, L uniform on {{32..2048}}, T uniform [1.5,3.5] "
                                 f"(seed 11), hot starts, {sweeps} sweeps, E/M every sweep",
                     "replica_updates": updates,
                     "tiles": "autotuned (tuned.json batch/batched512)" if tuned else "library defaults"},
          "per_instance": {"value": upd_k / (dt_p * 1e9), "unit": METRIC, "replicas": k,
                           "path": "one ising_lattice per replica, ising_sweep_record(sweeps, 1)",
                           "bit_exact_vs_batched": exact},
          "batched_over_per_instance": (updates / dt_b) / (upd_k / dt_p),
          "cpu_baseline": cpu, "clocks": clocks.summary(), "gpu_launches": batch_launches(n, sweeps)})


def run_scan(args, ising, local):
    import numpy as np
    import torch
    from math import pi  # noqa: F401
    Ts = np.array([(10 + k) / 10.0 for k in range(26)])
    L = 1024
    n = len(Ts)
    therm = 2000
    meas = args.sweeps or 10000
    b = ising.Batch([L] * n, 1.0 / Ts, [7] * n, np.zeros(n, dtype=np.uint8))
    with ClockSampler(local) as clocks:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.sweep(therm, every=therm)
        E, M = b.sweep(meas, every=1)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    b.close()
    per_T = []
    for r in range(n):
        e, m = ising.means(E[r], M[r], L)
        per_T.append({"T": float(Ts[r]), "E_per_spin": e, "absM_per_spin": m})
    cpu = None
    if not args.no_cpu_baseline:
        cores = min(os.cpu_count() or 1, n)
        cpu_rate, cpu_core = oracle_all_cores([(L, 7, float(1.0 / Ts[k]), False, 100) for k in range(cores)])
        cpu = {"value": cpu_rate, "unit": METRIC, "cores": cores, "kind": "oracle", "per_core": cpu_core,
               "host": host_cpu(),
               "sample": f"{cores} of the scan's lattices (L={L}, cold start, seed 7, T={Ts[0]}..{Ts[cores - 1]}), "
                         "100 sweeps each with E/M every sweep, one per host core, concurrently"}
    emit({"metric": METRIC, "value": n * L * L * (therm + meas) / (dt * 1e9), "unit": METRIC, "n_gpus": 1,
          "steps": 1, "warmup": 0, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
          "vs_baseline": None, "dtype": "u64", "data": "synthetic",
          "config": {"workload": f"scan: L={L}, T=1.0..3.5 step 0.1 ({n} replicas in one batch), cold start, "
                                 f"seed 7, {therm}+{meas} sweeps, E/M every measured sweep"},
          "per_T": per_T, "cpu_baseline": cpu, "clocks": clocks.summary(),
          "gpu_launches": batch_launches(n, therm) + batch_launches(n, meas)})


def run_serving(args, ising, local):
    import numpy as np
    from paper_1811_04384_gb300 import serving
    n = args.instances or 400
    stream = serving.poisson_stream(n, rate=args.rate, seed=13)
    budget = 4 << 30
    with ClockSampler(local) as clocks:
        reqs, stats = serving.serve_stream(stream, budget, max_jobs=256, epoch_sweeps=50, every=1)
    lat = np.array([r.result.done_s - r.result.submit_s for r in reqs])
    wait = np.array([r.result.start_s - r.result.submit_s for r in reqs])
    ok = all(r.result.status == 0 for r in reqs)
    updates = float(sum(r.L * r.L * r.sweeps for r in reqs))
    # bit-exact: every 10th job again, alone, through the single-lattice path
    exact = True
    checked = 0
    for r in reqs[::10]:
        with ising.Lattice(r.L, r.seed) as lat1:
            lat1.init_hot()
            lat1.set_beta(r.beta)
            E, M = lat1.sweep_record(r.sweeps, 1)
        exact &= bool(np.array_equal(E, r.E) and np.array_equal(M, r.M))
        checked += 1
    span = max(r.result.done_s for r in reqs) - min(r.result.submit_s for r in reqs)
    emit({"metric": METRIC, "value": updates / (span * 1e9), "unit": METRIC, "n_gpus": 1, "steps": 1,
          "warmup": 0, "ms_per_step": span * 1e3, "higher_is_better": True, "scaling": "weak",
          "vs_baseline": None, "dtype": "u64", "data": "synthetic",
          "config": {"workload": f"serving: {n} Poisson arrivals ({args.rate:g} req/s, seed 13), L in {{64..4096}}, "
                                 "T in [1.5,3.5], sweeps log-uniform 100..10000, hot starts, E/M every sweep",
                     "rate_req_per_s": args.rate, "hbm_budget_bytes": budget, "max_jobs": 256, "epoch_sweeps": 50},
          "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                        "mean": float(lat.mean()), "queue_wait_p50": float(np.percentile(wait, 50))},
          "offered_updates_per_ns": updates / (stream[-1][0] * 1e9),
          "offered_over_achieved": (updates / stream[-1][0]) / (updates / span),
          "device_busy_updates_per_ns": stats["spin_updates"] / (stats["busy_s"] * 1e9),
          "epochs": stats["epochs"], "all_ok": ok,
          "alone_vs_mix": {"jobs_checked": checked, "bit_exact": exact},
          "clocks": clocks.summary()})


def run_plain(args, ising, local):
    """L = 64 is launch-latency bound: time ising_sweep_record(1000, 1) alone
    (wall clock around the call, which synchronises), lattice already created,
    on each execution path."""
    import numpy as np
    L, n = 64, args.sweeps or 1000
    results = {}
    series = {}
    for name, path in (("resident", ising.ISING_PATH_RESIDENT), ("launches", ising.ISING_PATH_LAUNCHES)):
        with ising.Lattice(L, 1) as lat:
            lat.set_path(path)
            lat.init_hot()
            lat.set_beta(BETA)
            lat.sweep_record(20, 1)                      # warm-up (module load)
            lat.init_hot()
            best = None
            for _ in range(3):
                lat.init_hot()
                t0 = time.perf_counter()
                E, M = lat.sweep_record(n, 1)
                dt = time.perf_counter() - t0
                best = dt if best is None else min(best, dt)
            results[name] = best
            series[name] = (E, M)
    with ising.Batch([L], [BETA], [1], [1]) as b:     # graph-captured launches
        b.sweep([20], every=1)
    with ising.Batch([L], [BETA], [1], [1]) as b:
        t0 = time.perf_counter()
        Eb, Mb = b.sweep([n], every=1)
        results["graph"] = time.perf_counter() - t0
    exact = all(np.array_equal(series[k][0], Eb[0]) and np.array_equal(series[k][1], Mb[0]) for k in series)
    rate = {k: L * L * n / (v * 1e9) for k, v in results.items()}
    emit({"metric": METRIC, "value": rate["resident"], "unit": METRIC, "n_gpus": 1, "steps": 1, "warmup": 1,
          "ms_per_step": results["resident"] * 1e3, "higher_is_better": True, "scaling": "weak",
          "vs_baseline": None, "dtype": "u64", "data": "synthetic",
          "config": {"workload": f"plain: L={L}, T=2.269, hot start seed 1, {n} sweeps, E/M every sweep; "
                                 "wall clock of ising_sweep_record(n, 1) (best of 3)"},
          "paths": {"resident_on_chip": rate["resident"], "launches": rate["launches"],
                    "graph_captured_batch": rate["graph"]},
          "bit_exact_across_paths": exact,
          "gpu_launches": 3})      # the timed on-chip call: mask draw, on-chip sweeps, sweep counter


# Mid-size lattices, between the on-chip range (L <= 292) and L = 1080:
# there the automatic path is the cluster path (one thread-block
# cluster keeps the lattice on chip over pieces of up to 256 sweeps).
MIDSIZE_L = [296, 400, 512, 700, 1008]


def cluster_launches(L: int, sweeps: int, every: int) -> int:
    """Kernel launches of ising_sweep_record(sweeps, every) on the cluster
    path: per chunk of 1024 records, a mask draw and a cluster launch per
    piece of sweeps (two mask buffers of at most 128 MB, 256 sweeps at most)
    and one sweep-counter advance."""
    W = -(-(L // 2) // 21)
    P = W + (W & 1)
    piece = max(1, min(256, (256 << 20) // (2 * 2 * L * P * 8)))
    launches, records, rest = 0, sweeps // every, sweeps % every
    while records > 0:
        chunk = min(records, 1024)
        launches += 2 * -(-(chunk * every) // piece) + 1
        records -= chunk
    if rest > 0:                       # the sweeps after the last record: one ising_sweep
        launches += 2 * -(-rest // piece) + 1
    return launches


def run_midsize(args, ising, local):
    """Each mid-size L on the automatic path (the cluster path) and on the
    graph replays (ISING_PATH_LAUNCHES), T = 2.269 from a hot start, E/M every
    10 sweeps, about 2e9 spin updates per L and path; CUDA events on the
    lattice's stream.  The two paths' E/M series must be identical."""
    import numpy as np
    import torch
    stream = torch.cuda.Stream()
    cases = []
    total_updates, total_s, launches = 0.0, 0.0, 0
    with ClockSampler(local) as clocks:
        for L in MIDSIZE_L:
            sweeps = args.sweeps or max(10, int(2e9 // (L * L)))
            sweeps -= sweeps % 10
            entry = {"L": L, "sweeps": sweeps}
            series = {}
            for name, path in (("cluster", ising.ISING_PATH_AUTO), ("graphs", ising.ISING_PATH_LAUNCHES)):
                with ising.Lattice(L, SEED_LARGE, stream=stream) as lat:
                    lat.set_path(path)
                    lat.init_hot()
                    lat.set_beta(BETA)
                    lat.sweep_record(40, 10)                     # warm-up (module load, graph capture)
                    lat.init_hot()
                    lat.t = 0
                    if name == "cluster":
                        assert lat.get_path() == ising.ISING_PATH_CLUSTER, L
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    E, M = lat.sweep_record(sweeps, 10)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    dt = e0.elapsed_time(e1) / 1e3
                series[name] = (E, M)
                entry[name] = L * L * sweeps / (dt * 1e9)
                if name == "cluster":
                    total_updates += L * L * sweeps
                    total_s += dt
                    launches += cluster_launches(L, sweeps, 10)
            entry["cluster_over_graphs"] = entry["cluster"] / entry["graphs"]
            entry["bit_exact_across_paths"] = bool(np.array_equal(series["cluster"][0], series["graphs"][0]) and
                                                   np.array_equal(series["cluster"][1], series["graphs"][1]))
            cases.append(entry)
    emit({"metric": METRIC, "value": total_updates / (total_s * 1e9), "unit": METRIC, "n_gpus": 1, "steps": 1,
          "warmup": 1, "ms_per_step": total_s * 1e3, "higher_is_better": True, "scaling": "weak",
          "vs_baseline": None, "dtype": "u64", "data": "synthetic",
          "config": {"workload": "midsize: L = " + ", ".join(map(str, MIDSIZE_L)) + ", T=2.269, hot start seed 3, "
                                 "about 2e9 spin updates per L, E/M every 10 sweeps; value = the automatic (cluster) "
                                 "path over all sizes (CUDA events); each size also on the graph replays"},
          "cases": cases, "clocks": clocks.summary(), "gpu_launches": launches})


# The paper's test cases (Table 2): lattice side and iterations; an iteration
# is 10 update attempts per spin, i.e. 10 sweeps of the checkerboard chain.
PAPER_CASES = [("case 1", 2016, 5000), ("case 2", 2016, 4500), ("case 3", 1008, 4500)]
PAPER_STRIPS = 72       # the paper's largest run: 9 nodes x 8 cores, one column strip each


def run_paper(args, ising, local):
    """The paper's three test cases as equal spin-update counts of the
    checkerboard chain, in the row-packed layout and in the paper's own
    column-interleaved layout; E/M once per iteration (every 10 sweeps)."""
    import numpy as np
    import torch
    stream = torch.cuda.Stream()
    cases = []
    total_updates, total_s = 0.0, 0.0
    with ClockSampler(local) as clocks:
        for name, L, iters in PAPER_CASES:
            sweeps = (args.sweeps or 10 * iters)
            sweeps -= sweeps % 10
            entry = {"case": name, "L": L, "iterations": sweeps // 10, "sweeps": sweeps}
            series = {}
            for lname, layout in (("row_packed", ising.ISING_LAYOUT_ROW_PACKED),
                                  ("column_interleaved", ising.ISING_LAYOUT_COLUMN_INTERLEAVED)):
                with ising.Lattice(L, SEED_LARGE, stream=stream, layout=layout) as lat:
                    lat.init_hot()
                    lat.set_beta(BETA)
                    lat.sweep_record(10, 10)                     # warm-up (module load)
                    lat.init_hot()
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    E, M = lat.sweep_record(sweeps, 10)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    dt = e0.elapsed_time(e1) / 1e3
                series[lname] = (E, M)
                entry[lname] = {"seconds": dt, "value": L * L * sweeps / (dt * 1e9)}
                if lname == "row_packed":
                    total_updates += L * L * sweeps
                    total_s += dt
            # the paper's own chain: random memory-word updates in two column phases,
            # 72 strips (the paper's largest run, 9 nodes x 8 cores), E/M every iteration
            with ising.Lattice(L, SEED_LARGE, stream=stream, layout=ising.ISING_LAYOUT_COLUMN_INTERLEAVED) as lat:
                lat.init_hot()
                lat.set_beta(BETA)
                lat.set_chain(ising.ISING_CHAIN_RANDOM_WORDS, PAPER_STRIPS)
                lat.sweep_record(2, 1)                           # warm-up (module load)
                lat.init_hot()
                lat.t = 0
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                Er, Mr = lat.sweep_record(sweeps // 10, 1)
                e1.record(stream)
                torch.cuda.synchronize()
                dt = e0.elapsed_time(e1) / 1e3
            entry["random_words"] = {"strips": PAPER_STRIPS, "iterations": sweeps // 10, "seconds": dt,
                                     "value": L * L * sweeps / (dt * 1e9),
                                     "E_per_spin_last": float(Er[-1]) / (L * L)}
            entry["bit_exact_across_layouts"] = bool(np.array_equal(series["row_packed"][0],
                                                                    series["column_interleaved"][0]) and
                                                     np.array_equal(series["row_packed"][1],
                                                                    series["column_interleaved"][1]))
            entry["E_per_spin_last"] = float(series["row_packed"][0][-1]) / (L * L)
            cases.append(entry)
    emit({"metric": METRIC, "value": total_updates / (total_s * 1e9), "unit": METRIC, "n_gpus": 1, "steps": 1,
          "warmup": 1, "ms_per_step": total_s * 1e3, "higher_is_better": True, "scaling": "weak",
          "vs_baseline": None, "dtype": "u64", "data": "synthetic",
          "config": {"workload": "paper: the three test cases of Table 2 (L = 2016, 2016, 1008; 5000, 4500, "
                                 "4500 iterations of 10 sweeps), T=2.269, hot start seed 3, E/M every iteration; "
                                 "value = row-packed layout over all three cases (CUDA events); each case also "
                                 "runs the paper's own random-word chain (72 strips) for the same iterations"},
          "cases": cases, "clocks": clocks.summary()})


def integer_peaks(ising, clocks_summary: dict) -> dict:
    """The integer peaks of this device: the SM count and the per-SM, per-clock
    rates of 32x32->64 multiply-adds, 32-bit multiply-adds and three-input
    XORs measured by ising_probe_int_pipes (the SM's cycle counter, so
    independent of the clock), times the maximum SM clock that nvidia-smi
    reported during the timed region (clocks.max.sm), else the measured
    MEASURED_PEAKS.json's sm_max_mhz, else the nominal 2070 MHz."""
    probe = ising.probe_int_pipes()
    mhz, src = clocks_summary.get("sm_max_mhz"), "nvidia-smi clocks.max.sm during the timed region"
    if not mhz:
        peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(peaks_path) and json.load(open(peaks_path)).get("sm_max_mhz"):
            mhz, src = float(json.load(open(peaks_path))["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
        else:
            mhz, src = NOMINAL_SM_MAX_MHZ, "nominal"
    return dict(probe, sm_max_mhz=float(mhz), clock_source=src)


def two_pipe_roofline(achieved_sites_per_ns: float, rng: int, peaks: dict) -> dict:
    """The two-pipe integer bound, beside the strict multiply-only one: the
    integer work per site over both pipes it can use.  Per site,
    FMA-heavy only: the Philox multiplies, 2 issue slots each (4 per site;
    2.5 with 7 rounds); ALU only: the Philox three-input XORs (4.5; 3 with
    7 rounds), the two threshold compares and the word logic (1.1, per
    site of a 21-field word); either pipe: the two accept-bit inserts.  With
    the inserts split to balance, each pipe (64 lanes / clock / SM) carries
    half of the total."""
    mul = MULWIDE_PER_SITE if rng == 10 else 2.5
    xors = 4.5 if rng == 10 else 3.0
    # issue slots in units of one 32-bit multiply-add (the FMA-heavy pipe's
    # lane rate); a 32x32->64 product takes mad32 / mulwide of them
    lanes = peaks["mad32_per_sm_clk"]
    fma_only = mul * lanes / peaks["mulwide_per_sm_clk"]
    alu_only = (xors + 2 + 1.1) * lanes / peaks["lop3_per_sm_clk"]
    either = 2.0
    slots = max(fma_only, alu_only, (fma_only + alu_only + either) / 2)
    peak = peaks["sm_count"] * lanes * peaks["sm_max_mhz"] * 1e6 / slots / 1e9
    return {"peak_spin_updates_per_ns": peak, "frac": achieved_sites_per_ns / peak,
            "slots_per_site_per_pipe": slots,
            "basis": (f"FMA-heavy only {mul} x mul.wide per site, ALU only Philox XORs + 2 compares + word logic, "
                      f"2 inserts on either pipe, balanced; {peaks['sm_count']} SMs x measured lane rates "
                      f"(mul.wide {peaks['mulwide_per_sm_clk']:.1f}, mad32 {peaks['mad32_per_sm_clk']:.1f}, "
                      f"lop3 {peaks['lop3_per_sm_clk']:.1f} per SM per clock, ising_probe_int_pipes) x "
                      f"{peaks['sm_max_mhz']:.0f} MHz ({peaks['clock_source']})")}


def main():
    args = parse()
    ClockSampler.csv_dir = args.clocks_csv
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload != "large":
        import torch
        torch.cuda.set_device(local)
        from paper_1811_04384_gb300 import build as lib_build
        lib_build.build()
        import paper_1811_04384_gb300 as ising
        if rank == 0:
            {"batched": run_batched, "scan": run_scan, "plain": run_plain,
             "serving": run_serving, "paper": run_paper, "midsize": run_midsize}[args.workload](args, ising, local)
        return

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1811_04384_gb300 import build as lib_build
    lib_build.build()
    import paper_1811_04384_gb300 as ising

    L = args.L
    seed = SEED_LARGE + 1000003 * rank        # replicas: independent seeds
    stream = torch.cuda.Stream()
    lat = ising.Lattice(L, seed, stream=stream)
    if args.tiling:
        lat.set_tiling(*[int(x) for x in args.tiling.split(",")])
    if args.rng == 7:
        lat.set_rng(ising.ISING_RNG_PHILOX4X32_7)
    lat.init_hot()
    lat.set_beta(BETA)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
        lat.sweep_record(SWEEPS_PER_STEP, SWEEPS_PER_STEP)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    E_series, M_series = [], []
    with ClockSampler(local) as clocks:
        barrier()
        w0 = time.perf_counter()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            starts[k].record(stream)
            E, M = lat.sweep_record(SWEEPS_PER_STEP, SWEEPS_PER_STEP)
            ends[k].record(stream)
            E_series.append(int(E[0]))
            M_series.append(int(M[0]))
        barrier()
        wall = time.perf_counter() - w0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    dev_s = sum(step_ms) / 1e3
    dev_s, wall = max_over_ranks([dev_s, wall], world)

    updates_per_rank = args.steps * SWEEPS_PER_STEP * L * L
    value = whole_job_rate(updates_per_rank, world, dev_s)
    launches_per_step = 2 * SWEEPS_PER_STEP + 1     # half-sweeps + counter advance
    half_sweep_s = dev_s / (args.steps * 2 * SWEEPS_PER_STEP)

    # roofline of the half-sweep kernel: the 32x32->64 multiplies of Philox4x32-10
    sites_per_launch = L * L // 2
    mul_per_site = MULWIDE_PER_SITE if args.rng == 10 else 2.5
    achieved_mul = sites_per_launch * mul_per_site / half_sweep_s / 1e12
    cs = clocks.summary()
    peaks = integer_peaks(ising, cs)
    peak_mul = peaks["sm_count"] * peaks["mulwide_per_sm_clk"] * peaks["sm_max_mhz"] * 1e6 / 1e12
    W = (L // 2 + 20) // 21
    P = W + (W & 1)
    hbm_bytes_per_launch = 3 * L * P * 8          # read own + write own + read other colour
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm_peak = json.load(open(peaks_path))["hbm_gbs"] if os.path.exists(peaks_path) else 6800.0

    # e2e: every step's spins come from pinned host memory and its E/M record
    # goes back to the host, through ising_run_states (the copy of step k+1
    # overlaps the sweeps of step k); the one-call-per-step form is reported
    # beside it
    e2e = None
    if not args.no_e2e:
        hosts = [torch.empty((L, L), dtype=torch.int8, pin_memory=True) for _ in range(2)]
        spins = lat.get_spins()
        for hb in hosts:
            hb.numpy()[:] = spins
        n_e2e = max(3, min(args.steps, 50))
        states = [hosts[k % 2].numpy() for k in range(n_e2e)]
        lat.run_states(states[:2], SWEEPS_PER_STEP, SWEEPS_PER_STEP)       # warm-up (buffers, streams)
        barrier()
        e0 = time.perf_counter()
        lat.run_states(states, SWEEPS_PER_STEP, SWEEPS_PER_STEP)
        barrier()
        e_dt = time.perf_counter() - e0
        barrier()
        s0 = time.perf_counter()
        for k in range(n_e2e):
            lat.set_spins(states[k])
            lat.sweep_record(SWEEPS_PER_STEP, SWEEPS_PER_STEP)
        barrier()
        s_dt = time.perf_counter() - s0
        e_dt, s_dt = max_over_ranks([e_dt, s_dt], world)
        e2e = {"value": whole_job_rate(n_e2e * SWEEPS_PER_STEP * L * L, world, e_dt), "unit": METRIC,
               "h2d_bytes_per_step": L * L, "d2h_bytes_per_step": 32 * 16, "steps": n_e2e,
               "path": "ising_run_states: per step the pinned int8 L*L spins to the device (copy overlapping the "
                       "previous step's sweeps), 10 sweeps, E/M record back",
               "one_call_per_step": {"value": whole_job_rate(n_e2e * SWEEPS_PER_STEP * L * L, world, s_dt),
                                     "path": "ising_set_spins (pinned, read in place) + ising_sweep_record(10, 10)"}}

    # plain vs batched: the batched configuration (512 uneven replicas, one
    # launch per colour, CUDA graph) against per-instance calls on a sample
    batched = None
    if rank == 0 and world == 1 and not args.no_batched:
        batched = batched_summary(ising, sweeps=5000, instances=32)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt = oracle_sample(L, 1, BETA, SEED_LARGE)
        cpu = {"value": v, "unit": METRIC, "cores": 1, "kind": "oracle", "host": host_cpu(),
               "sample": f"1 sweep of the L={L} hot-start lattice (seed {SEED_LARGE}, T=2.269); init excluded; {dt:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": (f"large: L={L} periodic Ising (J=1, h=0), T=2.269, hot start seed 3, "
                                    "E/M every 10 sweeps; step = 10 sweeps + E/M record"),
                       "L": L, "sweeps_per_step": SWEEPS_PER_STEP, "parallelism": f"replicas x{world}",
                       "l2": "flushed between steps (256 MB write; lattice 103 MB < L2)",
                       "tiling": args.tiling or "default 4,0,128 (1-D items, 128 threads a block)",
                       "rng": f"Philox4x32-{args.rng}"},
            "wall_s": wall,
            "roofline": {"bound": "alu", "achieved": achieved_mul, "peak": peak_mul,
                         "unit": "T mul.wide.u32/s", "frac": achieved_mul / peak_mul,
                         "traffic": MEASURED_TRAFFIC.get(L) if args.rng == 10 else None,
                         "kernel": "half_sweep_kernel",
                         "achieved_spin_updates_per_ns": sites_per_launch / half_sweep_s / 1e9,
                         "peak_spin_updates_per_ns": peak_mul * 1e12 / mul_per_site / 1e9,
                         "peak_basis": (f"{peaks['sm_count']} SMs x {peaks['mulwide_per_sm_clk']:.1f} "
                                        "mul.wide.u32 per SM per clock (measured, ising_probe_int_pipes) x "
                                        f"{peaks['sm_max_mhz']:.0f} MHz ({peaks['clock_source']}); "
                                        f"{mul_per_site} per site (16 per Philox4x32-10 call after hoisting, "
                                        "4 sites per call)"),
                         "int_pipes": peaks,
                         "two_pipe": two_pipe_roofline(sites_per_launch / half_sweep_s / 1e9, args.rng, peaks),
                         "hbm_achieved_gbs": hbm_bytes_per_launch / half_sweep_s / 1e9,
                         "hbm_peak_gbs": hbm_peak,
                         "hbm_frac": hbm_bytes_per_launch / half_sweep_s / 1e9 / hbm_peak},
            "e2e": e2e,
            "cpu_baseline": cpu,
            "batched": batched,
            "clocks": cs,
            "gpu_launches": args.steps * launches_per_step,
            "E_last": E_series[-1], "M_last": M_series[-1],
        }
        print(json.dumps(line), flush=True)
    lat.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
