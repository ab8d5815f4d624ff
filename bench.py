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
bounded sample of the same workload: each step is one sweep of an L = 4096
lattice at the same temperature.
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
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
IMAD_PER_SM_CLK = 64            # 32-bit integer multiply results per SM per clock
MUL_RESULTS_PER_SITE = 10       # Philox4x32-10: 20 32x32->64 products per 4 sites


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tiling", default=None, help="rows,block_words,block_groups")
    ap.add_argument("--L", type=int, default=L_LARGE, help="lattice side (profiling of a smaller case)")
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

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        os.makedirs(os.path.join(ROOT, "gpurun_out"), exist_ok=True)
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{self.gpu}.csv")
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


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build()
    L = 4096
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
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
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
    if world > 1:
        t = torch.tensor([dev_s, wall], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        dev_s, wall = float(t[0]), float(t[1])

    updates_per_rank = args.steps * SWEEPS_PER_STEP * L * L
    value = world * updates_per_rank / (dev_s * 1e9)
    launches_per_step = 2 * SWEEPS_PER_STEP + 1     # half-sweeps + counter advance
    half_sweep_s = dev_s / (args.steps * 2 * SWEEPS_PER_STEP)

    # roofline of the half-sweep kernel: integer multiplies of Philox4x32-10
    sites_per_launch = L * L // 2
    achieved_imad = sites_per_launch * MUL_RESULTS_PER_SITE / half_sweep_s / 1e12
    peak_imad = SM_COUNT * IMAD_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12
    W = (L // 2 + 20) // 21
    P = W + (W & 1)
    hbm_bytes_per_launch = 3 * L * P * 8          # read own + write own + read other colour
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm_peak = json.load(open(peaks_path))["hbm_gbs"] if os.path.exists(peaks_path) else 6800.0

    # e2e: spins uploaded from pinned host memory each step, E/M read back
    e2e = None
    if not args.no_e2e:
        host = torch.empty((L, L), dtype=torch.int8, pin_memory=True)
        host_np = host.numpy()
        host_np[:] = lat.get_spins()
        n_e2e = max(3, min(args.steps, 50))
        lat.set_spins(host_np)
        lat.sweep_record(SWEEPS_PER_STEP, SWEEPS_PER_STEP)
        barrier()
        e0 = time.perf_counter()
        for _ in range(n_e2e):
            lat.set_spins(host_np)
            lat.sweep_record(SWEEPS_PER_STEP, SWEEPS_PER_STEP)
        barrier()
        e_dt = time.perf_counter() - e0
        if world > 1:
            t = torch.tensor([e_dt], dtype=torch.float64, device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e_dt = float(t[0])
        e2e = {"value": world * n_e2e * SWEEPS_PER_STEP * L * L / (e_dt * 1e9), "unit": METRIC,
               "h2d_bytes_per_step": L * L, "d2h_bytes_per_step": 32 * 16, "steps": n_e2e,
               "path": "ising_set_spins (pinned int8 L*L) + ising_sweep_record(10, 10) per step"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt = oracle_sample(L, 1, BETA, SEED_LARGE)
        cpu = {"value": v, "unit": METRIC, "cores": 1, "kind": "oracle",
               "sample": f"1 sweep of the L={L} hot-start lattice (seed {SEED_LARGE}, T=2.269); init excluded; {dt:.1f} s"}

    if rank == 0:
        cs = clocks.summary()
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": (f"large: L={L} periodic Ising (J=1, h=0), T=2.269, hot start seed 3, "
                                    "E/M every 10 sweeps; step = 10 sweeps + E/M record"),
                       "L": L, "sweeps_per_step": SWEEPS_PER_STEP, "parallelism": f"replicas x{world}",
                       "l2": "flushed between steps (256 MB write; lattice 103 MB < L2)",
                       "tiling": args.tiling or "default 4,32,4"},
            "wall_s": wall,
            "roofline": {"bound": "alu", "achieved": achieved_imad, "peak": peak_imad,
                         "unit": "T int32-mul/s", "frac": achieved_imad / peak_imad, "traffic": None,
                         "kernel": "half_sweep_kernel",
                         "achieved_spin_updates_per_ns": sites_per_launch / half_sweep_s / 1e9,
                         "peak_spin_updates_per_ns": peak_imad * 1e12 / MUL_RESULTS_PER_SITE / 1e9,
                         "peak_basis": "152 SMs x 64 int32 multiply results/clk x 2070 MHz; 10 per site",
                         "hbm_achieved_gbs": hbm_bytes_per_launch / half_sweep_s / 1e9,
                         "hbm_peak_gbs": hbm_peak,
                         "hbm_frac": hbm_bytes_per_launch / half_sweep_s / 1e9 / hbm_peak},
            "e2e": e2e,
            "cpu_baseline": cpu,
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
