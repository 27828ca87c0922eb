"""Benchmark: 2D heat, periodic 4096 x 4096 FP64, r = 0.2, 10,000 steps, by the
swept rule on one GB300 (and the naive one-kernel-per-step path beside it).

One bench step = one pass of the whole hot path over the workload: reset the
device state from a resident copy of the initial field (device to device) and
advance 10,000 time steps. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one process per GPU) every rank advances its own
independent grid ("replicas only": the method needs no collective on one
GPU), the timed region is bracketed by a barrier, the time is the max over
ranks and ``value`` is the cells all ranks advanced per second.

``--impl reference`` times the CPU oracle (plain FP64 step loop, all host
cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s swept vs naive per-step (same GB300), roofline %, error vs FP64"
UNIT = "Gcell-updates/s"
# Algorithmic FP64 pipe operations per heat update: the east+south pair sum of
# a point is the west+north pair sum of its south-east neighbour, so a point
# needs one pair sum of its own, one sum and two fused multiply-adds.
HEAT_FP64_OPS_PER_UPDATE = 4


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--grid", type=int, default=4096)
    p.add_argument("--nsteps", type=int, default=10_000)
    p.add_argument("--tile", type=int, default=32)
    p.add_argument("--r", type=float, default=0.2)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--no-naive", action="store_true", help="skip the naive comparison arm")
    p.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--profile-case", action="store_true",
                   help="short run of the same grid for ncu captures (no JSON timing claims)")
    return p.parse_args()


# --------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": smax, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- reference

def cpu_oracle_rate(u0, r, seconds):
    """Time the oracle as it stands on a bounded sample of the workload: the
    full grid for as many steps as fit in about ``seconds``."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.heat(u0, r, 1)
    t1 = (time.perf_counter() - t0)
    nsteps = max(1, int(seconds / max(t1, 1e-4)))
    t0 = time.perf_counter()
    oracle.heat(u0, r, nsteps)
    dt = time.perf_counter() - t0
    return u0.size * nsteps / dt / 1e9, nsteps, dt, oracle.num_threads()


def run_reference(args, rank):
    if rank != 0:
        return
    from paper_1602_07558_gb300 import inputs
    u0 = inputs.smooth_field(args.grid, args.grid, seed=args.seed)
    rates = []
    for i in range(args.warmup + args.steps):
        rate, nsteps, dt, cores = cpu_oracle_rate(u0, args.r, args.cpu_seconds / 2)
        if i >= args.warmup:
            rates.append((rate, nsteps, dt))
    value = statistics.mean(r[0] for r in rates)
    ms = statistics.mean(r[2] for r in rates) * 1e3
    sample = (f"{args.grid}x{args.grid} FP64 heat, {rates[-1][1]} of the {args.nsteps} steps "
              f"per bench step (bounded sample)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"heat {args.grid}x{args.grid} FP64 r={args.r} (CPU oracle)",
                   "grid": args.grid, "nsteps": args.nsteps},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------- ours

def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_1602_07558_gb300 import inputs
    from paper_1602_07558_gb300.swept2d import Swept2D, measure_fp64_rate

    N = args.grid
    cells = N * N
    stream = torch.cuda.Stream()
    u0_host = inputs.smooth_field(N, N, seed=args.seed + rank).reshape(1, N, N)
    u0_dev = torch.from_numpy(u0_host).to("cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()

    sw = Swept2D(N, N, op="heat", tile=args.tile, params=(args.r,), stream=stream)
    nv = Swept2D(N, N, op="heat", tile=0, params=(args.r,), stream=stream) if not args.no_naive else None

    if args.profile_case:
        # a short run of each path on the full grid, for ncu launch lists / captures
        with torch.cuda.stream(stream):
            for s in filter(None, (sw, nv)):
                s.set_state(u0_dev)
                s.advance(4 * args.tile, mode="swept" if s is sw else "naive")
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": True, "grid": N, "tile": args.tile}), flush=True)
        return

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_steps(s, mode, k, w):
        times = []
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        launches0 = s.query("launches")
        for i in range(w + k):
            if i == w:
                barrier()
                launches0 = s.query("launches")
            with torch.cuda.stream(stream):
                flush.zero_()                       # L2 flush outside the timed events
                start.record(stream)
                s.set_state(u0_dev)
                s.advance(args.nsteps, mode=mode)
                stop.record(stream)
            stop.synchronize()
            if i >= w:
                times.append(start.elapsed_time(stop))
        barrier()
        return times, int(s.query("launches") - launches0)

    with ClockSampler(local) as clocks:
        t_sw, launches = timed_steps(sw, "swept", args.steps, args.warmup)
        t_nv = timed_steps(nv, "naive", max(1, args.steps - 1), 1)[0] if nv else None
    ms_sw = statistics.mean(t_sw)
    ms_nv = statistics.mean(t_nv) if t_nv else None

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    ms_sw = max_over_ranks(ms_sw)
    value = world * cells * args.nsteps / (ms_sw * 1e-3) / 1e9
    naive_value = world * cells * args.nsteps / (max_over_ranks(ms_nv) * 1e-3) / 1e9 if ms_nv else None

    # swept == naive, bitwise, on the full run of the workload
    out_sw = sw.get_state()
    same = None
    if nv is not None:
        same = bool(np.array_equal(out_sw, nv.get_state()))

    # roofline of the dominant kernel: one timed pass with per-launch events
    fp64_rate = measure_fp64_rate(stream)
    sw.set_timing(True)
    with torch.cuda.stream(stream):
        sw.set_state(u0_dev)
        sw.advance(args.nsteps, mode="swept")
    kern = {k: sw.kernel_stats(k) for k in ("up", "bridge", "octahedron", "down", "naive")}
    sw.set_timing(False)
    n = args.tile
    h = n // 2
    tiles = (N // n) ** 2
    oct_cells = sum((2 * t) ** 2 for t in range(1, h + 1)) + sum((n - 2 * t) ** 2 for t in range(1, h))
    oct_launches, oct_ms = kern["octahedron"]
    oct_avg_ms = oct_ms / max(1, oct_launches)
    achieved = HEAT_FP64_OPS_PER_UPDATE * oct_cells * tiles / (oct_avg_ms * 1e-3) / 1e9
    peak = fp64_rate / 1e9
    total_kernel_ms = sum(v[1] for v in kern.values())

    roofline = {
        "bound": "alu", "unit": "Gop/s (FP64 pipe)", "kernel": "octahedron",
        "achieved": achieved, "peak": peak, "frac": achieved / peak,
        "peak_source": "measured in this run (swept2d_measure_fp64_rate: FP64 FMA chains)",
        "ops_per_update": HEAT_FP64_OPS_PER_UPDATE,
        "updates_per_launch": oct_cells * tiles,
        "avg_launch_ms": oct_avg_ms,
        "share_of_kernel_time": oct_ms / total_kernel_ms if total_kernel_ms else None,
        "hbm_bytes_per_launch": 2 * 4 * (n * n // 2 + n) * 8 * tiles,
        "traffic": None,
    }

    # error vs the FP64 oracle, and e2e through host buffers (rank 0)
    result = None
    if rank == 0:
        import oracle
        small = inputs.uniform(64, 64, seed=0)
        with Swept2D(64, 64, op="heat", tile=16, params=(args.r,), stream=stream) as s64:
            s64.set_state(small)
            s64.advance(512)
            e64 = float(np.max(np.abs(s64.get_state()[0] - oracle.heat(small, args.r, 512))))
        e_full = float(np.max(np.abs(sw_state_after(sw, u0_dev, 53, stream)[0]
                                     - oracle.heat(u0_host[0], args.r, 53))))
        # e2e: pinned host in, pinned host out, through the public API
        h_in = torch.from_numpy(u0_host.copy()).pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        e2e_t = []
        for i in range(1 + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sw.set_state(h_in)
            sw.advance(args.nsteps)
            sw.get_state(h_out)
            dt = time.perf_counter() - t0
            if i >= 1:
                e2e_t.append(dt)
        e2e_value = cells * args.nsteps / statistics.mean(e2e_t) / 1e9

        cpu = None
        if not args.no_cpu and world == 1:
            rate, nsteps_cpu, secs, cores = cpu_oracle_rate(u0_host[0], args.r, args.cpu_seconds)
            cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"{N}x{N} FP64 heat, {nsteps_cpu} steps ({secs:.1f} s)"}
        naive_rf = None
        if ms_nv:
            nk = sw_naive_kernel_ms(nv, u0_dev, stream)
            naive_rf = {"bound": "alu", "unit": "Gop/s (FP64 pipe)",
                        "achieved": HEAT_FP64_OPS_PER_UPDATE * cells / (nk * 1e-3) / 1e9,
                        "peak": peak,
                        "frac": HEAT_FP64_OPS_PER_UPDATE * cells / (nk * 1e-3) / 1e9 / peak,
                        "avg_launch_ms": nk,
                        "hbm_GBps_at_16B_per_update": 16 * cells / (nk * 1e-3) / 1e9}
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_sw,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"heat {N}x{N} FP64 r={args.r}, {args.nsteps} steps, "
                                   f"32-mode smooth field, swept tile {n}",
                       "grid": N, "nsteps": args.nsteps, "tile": n,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "flushed (256 MB write) between timed steps; state 134 MB"},
            "naive": {"value": naive_value, "unit": UNIT, "ms_per_step": ms_nv,
                      "roofline": naive_rf} if ms_nv else None,
            "speedup_vs_naive": (value / naive_value) if naive_value else None,
            "swept_equals_naive_bitwise": same,
            "error_vs_fp64_oracle": {"heat_64x64_512_steps_maxabs": e64,
                                     f"heat_{N}x{N}_53_steps_maxabs": e_full},
            "roofline": roofline,
            "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in kern.items()},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(u0_host.nbytes),
                    "d2h_bytes_per_step": int(u0_host.nbytes)},
            "gpu_launches": launches,
            "gpu_launches_per_step": launches // max(1, args.steps),
            "clocks": clocks.summary(),
        }
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if result is not None:
        print(json.dumps(result), flush=True)


def sw_state_after(s, u0_dev, nsteps, stream):
    import torch
    with torch.cuda.stream(stream):
        s.set_state(u0_dev)
        s.advance(nsteps)
    return s.get_state()


def sw_naive_kernel_ms(nv, u0_dev, stream):
    import torch
    nv.set_timing(True)
    with torch.cuda.stream(stream):
        nv.set_state(u0_dev)
        nv.advance(200, mode="naive")
    n, ms = nv.kernel_stats("naive")
    nv.set_timing(False)
    return ms / max(1, n)


if __name__ == "__main__":
    main()
