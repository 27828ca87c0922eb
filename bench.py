"""Benchmark of the swept rule on one GB300 (and the naive one-kernel-per-step
path beside it), printing one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload heat4096|heat64|heat2048_f32|heat2048_bf16|euler2048|
                              euler2048_f32|euler2048_bf16|wave1024|batch1024|
                              batch1024_euler]

The default workload is the headline one: 2D heat, periodic 4096 x 4096 FP64,
r = 0.2, 10,000 steps, smooth 32-mode initial field, tile 64 (512 threads). One bench step =
one pass of the whole hot path over the workload: reset the device state from a
resident copy of the initial field (device to device) and advance all steps.

Other workloads: heat64 (64 x 64 FP64, 512 steps, tile 16, U[0,1) field);
heat2048_f32 / heat2048_bf16 (2048 x 2048, binary32 arithmetic with Kahan-
compensated time update, binary32 / bfloat16 storage, 100,000 steps, error
against the FP64 solution reported); euler2048 (2048 x 2048 compressible Euler,
midpoint RK2, 5,000 steps, tile 32); euler2048_f32 / euler2048_bf16 (the
same in binary32 arithmetic with Kahan-compensated time update, binary32 /
bfloat16 storage, error against the FP64 solution reported); wave1024 (the paper's Section 6 wave
equation, leapfrog, Courant number 0.3, source at the centre, 1024 x 1024);
batch1024 (1,024 independent grids of uneven sizes, binary32 storage, one
graph-captured swept launch sequence for all of them, tile autotuned per size
class, against the batched naive path and against looping single-grid runs);
batch1024_euler (the same 1,024 grid sizes with the binary32 Euler form, each
grid's own time step, 2,000 steps).

The default run (headline workload, N = 1, no size flags) then measures the
other workloads, each in a child process with the same timing rules, and adds
their results to the line as ``secondary`` (``--no-secondary`` skips them).

With N > 1 (torchrun, one process per GPU) every rank advances its own
independent grid ("replicas only"), the timed region is bracketed by a barrier,
the time is the max over ranks and ``value`` counts the cells of all ranks.

``--impl reference`` times the CPU oracle (plain step loop, all host cores) on
a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time
from dataclasses import dataclass, field

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s swept vs naive per-step (same GB300), roofline %, error vs FP64"
UNIT = "Gcell-updates/s"
HBM_PEAK_GBPS = 6779.7          # MEASURED_PEAKS.json hbm_gbs (copy test on this pool)
GAMMA, CFL, KAPPA = 1.4, 0.3, 0.5


@dataclass
class Workload:
    op: str
    dtype: str
    grid: int
    nsteps: int
    tile: int
    params: tuple
    init: str
    seed: int
    describe: str = ""
    threads: int = 0                 # swept threads per block (0: the library's default)
    persistent: bool = False         # the swept arm's default form (measured fastest)
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    "heat4096": Workload("heat", "f64", 4096, 10_000, 64, (0.2,), "smooth", 1,
                         "heat 4096x4096 FP64 r=0.2, 10000 steps, 32-mode smooth field", 512),
    "heat64": Workload("heat", "f64", 64, 512, 16, (0.2,), "uniform", 0,
                       "heat 64x64 FP64 r=0.2, 512 steps, U[0,1) field (seed 0)"),
    "heat2048_f32": Workload("heat_kahan", "f32", 2048, 100_000, 64, (0.2,), "smooth", 1,
                             "heat 2048x2048, binary32 storage and arithmetic, Kahan-"
                             "compensated update, r=0.2, 100000 steps", persistent=True),
    "heat2048_bf16": Workload("heat_kahan", "bf16", 2048, 100_000, 64, (0.2,), "smooth", 1,
                              "heat 2048x2048, bfloat16 storage, binary32 arithmetic, Kahan-"
                              "compensated update, r=0.2, 100000 steps", persistent=True),
    "euler2048": Workload("euler_rk2", "f64", 2048, 5_000, 32, (GAMMA, CFL, KAPPA), "euler", 2,
                          "Euler 2048x2048 FP64, midpoint RK2, CFL 0.3, 5000 steps"),
    "euler2048_f32": Workload("euler_kahan", "f32", 2048, 5_000, 32, (GAMMA, CFL, KAPPA),
                              "euler", 2, "Euler 2048x2048, binary32 storage and arithmetic, "
                              "Kahan-compensated update, midpoint RK2, CFL 0.3, 5000 steps"),
    "euler2048_bf16": Workload("euler_kahan", "bf16", 2048, 5_000, 32, (GAMMA, CFL, KAPPA),
                               "euler", 2, "Euler 2048x2048, bfloat16 storage, binary32 "
                               "arithmetic, Kahan-compensated update, midpoint RK2, CFL 0.3, "
                               "5000 steps", 256),
    "batch1024": Workload("heat_kahan", "f32", 0, 20_000, 0, (0.2,), "batch", 3,
                          "1024 independent periodic grids, nx and ny uniform in {32,48,...,512} "
                          "(seed 3), heat with binary32 storage and Kahan-compensated update, "
                          "r=0.2, 20000 steps", persistent=True,
                          extra={"one_launch": True, "batch_tiles": "16,32"}),
    "batch1024_euler": Workload("euler_kahan", "f32", 0, 2_000, 0, (GAMMA, CFL, KAPPA), "batch",
                                3, "1024 independent periodic grids, nx and ny uniform in "
                                "{32,48,...,512} (seed 3), Euler with binary32 storage and "
                                "arithmetic, Kahan-compensated update, each grid's own CFL 0.3 "
                                "time step, 2000 steps"),
    "wave1024": Workload("wave", "f64", 1024, 10_000, 32, (0.3,), "source", 0,
                         "wave 1024x1024 FP64 leapfrog, Courant 0.3, Gaussian source at the "
                         "centre, 10000 steps"),
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="heat4096", choices=sorted(WORKLOADS))
    p.add_argument("--grid", type=int, default=None)
    p.add_argument("--nsteps", type=int, default=None)
    p.add_argument("--tile", type=int, default=None)
    p.add_argument("--no-naive", action="store_true", help="skip the naive comparison arm")
    p.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--quick-check", action="store_true",
                   help="compare with the oracle after 53 steps (20 for Euler), not all steps")
    p.add_argument("--oracle-steps", type=int, default=None,
                   help="compare with the CPU oracle after this many steps (default: all)")
    p.add_argument("--profile-case", action="store_true",
                   help="short run of the same grid for ncu captures (no timing claims)")
    p.add_argument("--threads", type=int, default=None, help="swept threads per block")
    p.add_argument("--stage", type=int, default=None, help="1: stage panels by TMA")
    p.add_argument("--autotune", action="store_true",
                   help="pick tile, threads and staging by timing short runs first")
    p.add_argument("--graph", action="store_true",
                   help="run each advance (swept and naive) as a captured CUDA graph")
    p.add_argument("--persistent", action="store_true",
                   help="swept arm: one persistent launch per advance")
    p.add_argument("--batch-tiles", default=None,
                   help="batches: candidate tile sides for the autotuner (default 16,32,64; "
                        "the heat batch's one-launch form: 16,32)")
    p.add_argument("--one-launch", action="store_true",
                   help="batches, with --persistent: one persistent launch for every tile class")
    p.add_argument("--no-secondary", action="store_true",
                   help="default run: skip the other workloads' lines (each measured in a "
                        "child process of its own)")
    p.add_argument("--launch-per-phase", action="store_true",
                   help="swept arm: one launch per phase (the default of most workloads)")
    a = p.parse_args()
    w = WORKLOADS[a.workload]
    if not a.persistent and not a.launch_per_phase:
        a.persistent = w.persistent
        # the workload's default form (the heat batch: one launch for every class)
        a.one_launch = a.one_launch or (a.persistent and w.extra.get("one_launch", False))
    if a.batch_tiles is None:
        a.batch_tiles = w.extra.get("batch_tiles", "16,32,64")
    for k in ("grid", "nsteps", "tile"):
        if getattr(a, k) is not None:
            setattr(w, k, getattr(a, k))
    return a, w


# --------------------------------------------------------------- inputs

def initial_state(w: Workload, rank: int = 0) -> np.ndarray:
    """Host copy of the initial state, (nvars, ny, nx) in the op's storage type."""
    from paper_1602_07558_gb300 import inputs
    N, seed = w.grid, w.seed + rank
    if w.op == "euler_rk2":
        U = inputs.euler_pulse(N, N, seed, gamma=GAMMA)
        return np.concatenate([U, U])
    if w.op == "euler_kahan":           # (U, U*, C) with C = 0
        U = to_storage(inputs.euler_pulse(N, N, seed, gamma=GAMMA).astype(np.float32), w.dtype)
        return np.concatenate([U, U, np.zeros_like(U)])
    if w.op == "wave":
        return inputs.wave_source(N, N)
    f = inputs.smooth_field(N, N, seed) if w.init == "smooth" else inputs.uniform(N, N, seed)
    if w.op == "heat":
        return f[None]
    u32 = to_storage(f.astype(np.float32), w.dtype)
    return np.stack([u32, np.zeros_like(u32)])


def to_storage(u32: np.ndarray, dtype: str) -> np.ndarray:
    """binary32 values -> the storage type (bfloat16 bits by torch's round to
    nearest even)."""
    if dtype != "bf16":
        return u32
    import torch
    return torch.from_numpy(np.ascontiguousarray(u32)).to(torch.bfloat16).view(torch.int16) \
        .numpy().view(np.uint16)


def storage_to_f64(a: np.ndarray, dtype: str) -> np.ndarray:
    if dtype == "bf16":
        return (a.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return a.astype(np.float64)


# --------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples go to $SWEPT2D_CLOCKS_DIR (default: the system's
        # temporary directory); their summary goes into the JSON line
        import tempfile
        out_dir = os.environ.get("SWEPT2D_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_rank{gpu_index}.csv")

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


# ------------------------------------------------------------ CPU oracle

def oracle_advance(w: Workload, state: np.ndarray, nsteps: int) -> np.ndarray:
    """The oracle on the same initial state (returns the state in the same layout)."""
    import oracle
    oracle.build()
    if w.op == "heat":
        return oracle.heat(state[0], w.params[0], nsteps)[None]
    if w.op == "heat_kahan":
        u, c = oracle.heat_kahan(state[0], state[1], w.params[0], nsteps, storage=w.dtype)
        return np.stack([u, c])
    if w.op == "euler_rk2":
        a, dt = oracle.euler_setup(state[:4], GAMMA, CFL)
        U = oracle.euler_rk2(state[:4], GAMMA, dt, KAPPA, a, nsteps)
        return U
    if w.op == "wave":
        u, uo = oracle.wave(state[0], state[1], w.params[0] * w.params[0], nsteps)
        return np.stack([u, uo])
    if w.op == "euler_kahan":
        a, dt = oracle.euler_setup(storage_to_f64(state[:4], w.dtype), GAMMA, CFL)
        return oracle.euler_kahan(state, GAMMA, dt, KAPPA, a, nsteps, storage=w.dtype)
    raise ValueError(w.op)


def cpu_oracle_rate(w: Workload, state, seconds):
    """Time the oracle as it stands on a bounded sample of the workload: the
    full grid for as many steps as fit in about ``seconds`` (at most the
    workload's own step count; a workload shorter than that is repeated).
    Returns (Gcell-updates/s, steps per run, runs, seconds, threads)."""
    import oracle
    oracle_advance(w, state, 1)                # first call: library load, page faults
    k = 1                                      # calibration: double until ~5% of the budget
    while True:
        t0 = time.perf_counter()
        oracle_advance(w, state, k)
        dt = time.perf_counter() - t0
        if dt >= 0.05 * seconds or k >= w.nsteps:
            break
        k *= 2
    t1 = max(dt / k, 1e-9)
    nsteps = max(1, min(w.nsteps, int(seconds / t1)))
    runs = max(1, int(seconds / (t1 * nsteps))) if nsteps == w.nsteps else 1
    t0 = time.perf_counter()
    for _ in range(runs):
        oracle_advance(w, state, nsteps)
    dt = time.perf_counter() - t0
    cells = state.shape[-1] * state.shape[-2]
    return cells * nsteps * runs / dt / 1e9, nsteps, runs, dt, oracle.num_threads()


def sample_text(N, w, nsteps, runs, secs):
    if runs > 1:
        return f"{N}x{N}, the full {w.nsteps} steps, {runs} runs ({secs:.1f} s)"
    return f"{N}x{N}, {nsteps} of {w.nsteps} steps ({secs:.1f} s)"


def run_reference(args, w, rank):
    if rank != 0:
        return
    state = initial_state(w)
    rates = []
    for i in range(args.warmup + args.steps):
        rate, nsteps, runs, dt, cores = cpu_oracle_rate(w, state, args.cpu_seconds / 2)
        if i >= args.warmup:
            rates.append((rate, nsteps, dt, runs))
    value = statistics.mean(r[0] for r in rates)
    ms = statistics.mean(r[2] for r in rates) * 1e3
    nlast, runs_last = rates[-1][1], rates[-1][3]
    sample = (f"{w.grid}x{w.grid} {w.describe}: "
              + (f"the full {w.nsteps} steps, {runs_last} runs" if runs_last > 1
                 else f"{nlast} of the {w.nsteps} steps")
              + " per bench step (bounded sample)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": w.dtype,
        "data": "synthetic",
        "config": {"workload": w.describe + " (CPU oracle)", "grid": w.grid, "nsteps": w.nsteps},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------- ranks

def aggregate_over_ranks(ms_local, cells_local, nsteps, dist=None, device="cpu"):
    """Replicas only: every rank advanced its own grid of ``cells_local`` points
    by ``nsteps`` steps in ``ms_local`` ms. The job's time is the slowest
    rank's; ``value`` counts the points of all ranks (Gcell-updates/s)."""
    if dist is None:
        return ms_local, cells_local * nsteps / (ms_local * 1e-3) / 1e9
    import torch
    t = torch.tensor([ms_local, float(cells_local)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    ms = float(tmax[0].item())
    return ms, float(t[1].item()) * nsteps / (ms * 1e-3) / 1e9


# ------------------------------------------------------------- rooflines

def octahedron_updates(n):
    h = n // 2
    return sum((2 * t) ** 2 for t in range(1, h + 1)) + sum((n - 2 * t) ** 2 for t in range(1, h))


def bridge_updates(n):
    h = n // 2
    return 2 * sum((n - 2 * k - 2) * (2 * k + 2) for k in range(h - 1))


# DRAM traffic (read + write bytes) per tile of one octahedron launch, from one
# ncu capture of the same kernel (the grid side it was taken on, 1024 or 2048),
# scaled to a launch by its number of tiles (reads equal the algorithmic panel
# bytes there; part of the writes may still be in L2 when the kernel ends).
# Kernels without a capture of their current version report None.
OCT_TRAFFIC_PER_TILE = {
    ("heat", "f64", 64): ((69.218e6 + 27.145e6) / 1024, 2048),
    ("heat_kahan", "f32", 64): ((69.242e6 + 21.500e6) / 1024, 2048),
    ("heat_kahan", "bf16", 64): ((34.622e6 + 0.215e6) / 1024, 2048),
    ("euler_rk2", "f64", 32): ((570.552e6 + 533.881e6) / 4096, 2048),
    ("euler_kahan", "f32", 32): ((428.327e6 + 394.044e6) / 4096, 2048),
    ("euler_kahan", "bf16", 32): ((213.992e6 + 160.476e6) / 4096, 2048),
    ("wave", "f64", 32): ((35.673e6 + 3.069e6) / 1024, 1024),
}

# Algorithmic work of one point update (one point advanced one sub-step),
# counted from the update formulas (a fused multiply-add or a division is one
# operation): FP64 operations, binary32 operations, and level-buffer accesses
# (every stored value the sub-step reads, read once, and every value it writes,
# written once: the shared-memory traffic of a walk that keeps each point's
# neighbours in registers).
#   heat FP64: own east+south pair sum, the sum of two pair sums, two FMAs = 4;
#     reads u, writes u = 2 accesses
#   wave FP64: the same Laplacian (3), 2u, 2u - u_old, one FMA = 6; reads and
#     writes (u, u_old) = 4
#   Euler FP64, per stage: one point's fluxes 15 (shared by its neighbours: 1/r,
#     u, v, ke 3, p 2, E+p, F and G 6), per conserved variable 12 = 63; stage 0
#     reads U writes U*, stage 1 reads U* and U writes U: 10 on average
#   heat binary32 + Kahan: 2 pair sums, sum, FMA, r d, - c, u + y, (u' - u) - y
#     = 9; reads and writes (u, c) = 4
#   Euler binary32 + Kahan: fluxes 15 and 12 per variable in stage 0, 16 per
#     variable in stage 1 (compensated update): 71 on average; stage 0 reads U
#     writes U*, stage 1 reads U*, U, C writes U, C: 14 on average
WORK = {
    ("heat", "f64"): (4, 0, 2),
    ("wave", "f64"): (6, 0, 4),
    ("euler_rk2", "f64"): (63, 0, 10),
    ("heat_kahan", "f32"): (0, 9, 4),
    ("heat_kahan", "bf16"): (0, 9, 4),
    ("euler_kahan", "f32"): (0, 71, 14),
    ("euler_kahan", "bf16"): (0, 71, 14),
}


def hbm_peak():
    """(GB/s, source): MEASURED_PEAKS.json's copy rate, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (copy test)"
    except (OSError, ValueError, KeyError):
        return HBM_PEAK_GBPS, "fallback 6779.7 GB/s (an earlier copy test on this pool)"


def bounds(w, esize, upd, hbm_bytes, seconds, peaks):
    """The slowest of the HBM, FP64, FP32 and shared-memory bounds for `upd`
    point updates moving `hbm_bytes` that took `seconds`."""
    fp64, fp32, acc = WORK.get((w.op, w.dtype), (0, 0, 0))
    wavefronts = acc * upd * max(1, esize // 4) / 32.0    # a warp access: 1 wavefront per 128 B
    hbm_gbs, hbm_src = hbm_peak()
    rows = {
        "hbm": (hbm_bytes / (hbm_gbs * 1e9), hbm_bytes / seconds / 1e9, hbm_gbs, "GB/s", hbm_src),
        "fp64": (fp64 * upd / peaks["fp64_ops_per_s"], fp64 * upd / seconds / 1e9,
                 peaks["fp64_ops_per_s"] / 1e9, "Gop/s (FP64 pipe)",
                 "measured in this run (FP64 FMA and add chains, maximum)"),
        "fp32": (fp32 * upd / peaks["fp32_ops_per_s"], fp32 * upd / seconds / 1e9,
                 peaks["fp32_ops_per_s"] / 1e9, "Gop/s (FP32 pipe)",
                 "measured in this run (FP32 FMA chains)"),
        "smem": (wavefronts / peaks["smem_wavefronts_per_s"], wavefronts / seconds / 1e9,
                 peaks["smem_wavefronts_per_s"] / 1e9, "G wavefronts/s (shared memory)",
                 "measured in this run (conflict-free 4-byte loads)"),
    }
    bound = max(rows, key=lambda k: rows[k][0])
    t, achieved, peak, unit, src = rows[bound]
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": t / seconds, "peak_source": src,
            "per_update": {"fp64_ops": fp64, "fp32_ops": fp32, "smem_accesses": acc,
                           "hbm_bytes": hbm_bytes / upd if upd else None},
            "all_bounds_frac": {k: v[0] / seconds for k, v in rows.items()}}


def roofline(w, kern, peaks, esize, nvars):
    """Roofline of the dominant swept kernel (the octahedron): its algorithmic
    work per launch over its CUDA-event launch time against the slowest of the
    HBM, FP64, FP32 and shared-memory bounds; the bridge's beside it."""
    n, N = w.tile, w.grid
    tiles = (N // n) ** 2
    launches, ms = kern["octahedron"]
    avg_ms = ms / max(1, launches)
    upd = octahedron_updates(n) * tiles            # point updates (sub-steps) per launch
    hbm_bytes = 2 * 4 * (n * n // 2 + n) * nvars * esize * tiles
    total_ms = sum(v[1] for v in kern.values())
    per_tile, cap_grid = OCT_TRAFFIC_PER_TILE.get((w.op, w.dtype, n), (None, None))
    out = {"kernel": "octahedron", "avg_launch_ms": avg_ms, "updates_per_launch": upd,
           "hbm_bytes_per_launch": hbm_bytes,
           "share_of_kernel_time": ms / total_ms if total_ms else None,
           "traffic": per_tile * tiles if per_tile else None,
           "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the same "
                              f"kernel at {cap_grid}x{cap_grid}, scaled by tiles")
           if per_tile else None}
    out.update(bounds(w, esize, upd, hbm_bytes, avg_ms * 1e-3, peaks))
    bl, bms = kern["bridge"]
    if bl:
        bupd = bridge_updates(n) * tiles              # both bridges of every tile
        b = bounds(w, esize, bupd, hbm_bytes, bms / bl * 1e-3, peaks)
        out["bridge"] = {"avg_launch_ms": bms / bl, "updates_per_launch": bupd,
                         "bound": b["bound"], "frac": b["frac"]}
    return out


# ----------------------------------------------------------------- ours

def main():
    args, w = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if w.init == "batch":
        run_batch(args, w, world, rank, local)
        return
    if args.impl == "reference":
        run_reference(args, w, rank)
        return

    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_1602_07558_gb300.swept2d import Swept2D, measure_peaks

    N = w.grid
    cells = N * N
    stream = torch.cuda.Stream()
    state_host = initial_state(w, rank)
    esize = state_host.dtype.itemsize
    nvars = state_host.shape[0]
    state_dev = torch.from_numpy(state_host).to("cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()

    mk = lambda tile: Swept2D(N, N, op=w.op, tile=tile, params=w.params, stream=stream,
                              dtype=w.dtype)
    tune_table = None
    if args.autotune:
        from paper_1602_07558_gb300.autotune import autotune
        (w.tile, args.threads, stage), tune_table = autotune(
            N, N, w.op, w.params, dtype=w.dtype, state=state_dev, stream=stream)
        args.stage = int(stage)
    sw = mk(w.tile)
    if args.threads is None and w.threads:
        args.threads = w.threads
    if args.threads is not None or args.stage is not None:
        sw.set_tuning(args.threads or int(sw.query("threads")),
                      bool(args.stage) if args.stage is not None else bool(sw.query("stage")))
    args.threads, args.stage = int(sw.query("threads")), int(sw.query("stage"))
    two_stage = w.op in ("euler_rk2", "euler_kahan")
    nv = None if args.no_naive else mk(0)

    if args.profile_case:
        with torch.cuda.stream(stream):
            for s in filter(None, (sw, nv)):
                s.set_state(state_dev)
                s.advance(4 * w.tile // (2 if two_stage else 1),
                          mode=("persistent" if args.persistent else "swept") if s is sw
                          else "naive")
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": True, "workload": w.describe, "grid": N,
                          "tile": w.tile}), flush=True)
        return

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_steps(s, mode, k, wu):
        times = []
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        launches0 = s.query("launches")
        for i in range(wu + k):
            if i == wu:
                barrier()
                launches0 = s.query("launches")
            with torch.cuda.stream(stream):
                flush.zero_()                       # L2 flush, outside the timed events
                start.record(stream)
                s.set_state(state_dev)
                s.advance(w.nsteps, mode=mode, graph=args.graph)
                stop.record(stream)
            stop.synchronize()
            if i >= wu:
                times.append(start.elapsed_time(stop))
        barrier()
        return times, int(s.query("launches") - launches0)

    with ClockSampler(local) as clocks:
        t_sw, launches = timed_steps(sw, "persistent" if args.persistent else "swept",
                                     args.steps, args.warmup)
        t_nv = timed_steps(nv, "naive", max(1, args.steps - 1), 1)[0] if nv else None

    ms_sw, value = aggregate_over_ranks(statistics.mean(t_sw), cells, w.nsteps, dist, "cuda")
    ms_nv, naive_value = (aggregate_over_ranks(statistics.mean(t_nv), cells, w.nsteps, dist,
                                               "cuda") if t_nv else (None, None))

    out_sw = sw.get_state()
    same = bool(np.array_equal(out_sw, nv.get_state())) if nv is not None else None

    # per-kernel CUDA-event timing on one more pass (not the headline timing)
    peaks = measure_peaks(stream)
    sw.set_timing(True)
    with torch.cuda.stream(stream):
        sw.set_state(state_dev)
        sw.advance(w.nsteps, mode="swept")
    kern = {k: sw.kernel_stats(k) for k in ("up", "bridge", "octahedron", "down", "naive")}
    sw.set_timing(False)
    rf = roofline(w, kern, peaks, esize, nvars)

    result = None
    if rank == 0:
        errors = accuracy_report(w, sw, state_host, state_dev, out_sw, stream, Swept2D,
                                 full=not args.quick_check, oracle_steps=args.oracle_steps)
        h_in = torch.from_numpy(state_host.copy()).pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        e2e_t = []
        for i in range(1 + min(args.steps, 3)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sw.set_state(h_in)
            sw.advance(w.nsteps, mode="persistent" if args.persistent else "swept",
                       graph=args.graph)
            sw.get_state(h_out)
            dt = time.perf_counter() - t0
            if i >= 1:
                e2e_t.append(dt)
        e2e_value = cells * w.nsteps / statistics.mean(e2e_t) / 1e9
        cpu = None
        if not args.no_cpu and world == 1:
            rate, nsteps_cpu, runs, secs, cores = cpu_oracle_rate(w, state_host, args.cpu_seconds)
            cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": sample_text(N, w, nsteps_cpu, runs, secs)}
            if N <= 64:                  # the small grid: the single-core oracle too
                import oracle
                oracle.set_threads(1)
                cpu["value_1core"] = cpu_oracle_rate(w, state_host, args.cpu_seconds / 4)[0]
                oracle.set_threads(cores)
        naive_rf = None
        if nv is not None:
            nk = naive_kernel_ms(nv, state_dev, stream, w)
            naive_rf = {"avg_launch_ms": nk}
            naive_rf.update(bounds(w, esize, cells, 2 * nvars * esize * cells, nk * 1e-3, peaks))
        trace = None
        if args.persistent:
            trace = persistent_trace(sw, w, state_dev, stream, clocks.summary().get("sm_mhz"))
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_sw,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": w.dtype, "data": "synthetic",
            "config": {"workload": f"{w.describe}, swept tile {w.tile}", "grid": N,
                       "nsteps": w.nsteps, "tile": w.tile, "threads": args.threads,
                       "stage": args.stage, "autotune": tune_table,
                       "parallelism": "replicas" if world > 1 else "single",
                       "cuda_graph": bool(args.graph),
                       "persistent": bool(args.persistent),
                       "l2": "flushed (256 MB write) between timed steps"},
            "naive": {"value": naive_value, "unit": UNIT, "ms_per_step": ms_nv,
                      "roofline": naive_rf} if ms_nv else None,
            "speedup_vs_naive": (value / naive_value) if naive_value else None,
            "swept_equals_naive_bitwise": same,
            "error_vs_fp64": errors,
            "roofline": rf,
            "measured_rates": peaks,
            "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in kern.items()},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(state_host.nbytes),
                    "d2h_bytes_per_step": int(state_host.nbytes)},
            "gpu_launches": launches,
            "gpu_launches_per_step": launches // max(1, args.steps),
            "persistent_trace": trace,
            "clocks": clocks.summary(),
        }
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if result is not None:
        if world == 1 and args.workload == DEFAULT_WORKLOAD and not args.no_secondary and \
                not any(f"--{k}" in sys.argv for k in ("grid", "nsteps", "tile", "threads")):
            result["secondary"] = secondary_lines()
        print(json.dumps(result), flush=True)


# The other workloads, measured after the headline by the default run, each by
# this script in a child process with the same timing rules (3 warm-up and 3
# timed steps, L2 flushed between them, clocks sampled) in the workload's
# default form. The long runs take fewer steps than the workload names: the
# time per step does not depend on the step count (one first Up and one final
# Down per advance). The state is compared with the CPU oracle over the first
# steps (--quick-check); the headline line carries the full-length comparison.
DEFAULT_WORKLOAD = "heat4096"
SECONDARY = (
    ("heat64", ()), ("heat64", ("--graph",)),
    ("heat2048_f32", ("--nsteps", "10000")), ("heat2048_bf16", ("--nsteps", "10000")),
    ("wave1024", ()),
    ("euler2048", ("--nsteps", "500")), ("euler2048_f32", ("--nsteps", "500")),
    ("euler2048_bf16", ("--nsteps", "500")),
    ("batch1024", ("--nsteps", "2000")), ("batch1024_euler", ("--nsteps", "200")),
    # the other batch form of each: heat per class (one launch per tile class
    # and phase, graph), Euler in one persistent launch
    ("batch1024", ("--nsteps", "2000", "--launch-per-phase", "--batch-tiles", "16,32,64")),
    ("batch1024_euler", ("--nsteps", "200", "--persistent", "--one-launch", "--batch-tiles",
                         "16,32")),
)


def secondary_lines(timeout_s=300):
    import subprocess
    out = []
    for name, extra in SECONDARY:
        cmd = [sys.executable, os.path.abspath(__file__), "--workload", name, "--no-cpu",
               "--quick-check", "--no-secondary", "--steps", "3", "--warmup", "3", *extra]
        entry = {"workload": name, "args": " ".join(extra)}
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s,
                               cwd=ROOT)
            lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
            if r.returncode != 0 or not lines:
                entry["error"] = f"exit {r.returncode}: {r.stderr.strip()[-300:]}"
                out.append(entry)
                continue
            d = json.loads(lines[-1])
        except (subprocess.TimeoutExpired, ValueError) as e:
            entry["error"] = f"{type(e).__name__}: {e}"[:300]
            out.append(entry)
            continue
        rf = d.get("roofline") or {}
        cfg = d.get("config") or {}
        entry.update({
            "describe": cfg.get("workload"), "nsteps": cfg.get("nsteps"),
            "tile": cfg.get("tile"), "persistent": cfg.get("persistent"),
            "one_launch": cfg.get("one_launch"), "cuda_graph": cfg.get("cuda_graph"), "value": d.get("value"), "unit": d.get("unit"),
            "ms_per_step": d.get("ms_per_step"),
            "naive": (d.get("naive") or d.get("naive_batched") or {}).get("value"),
            "speedup_vs_naive": d.get("speedup_vs_naive"),
            "swept_equals_naive_bitwise": d.get("swept_equals_naive_bitwise"),
            "roofline": {k: rf.get(k) for k in ("bound", "frac", "unit", "traffic")} if rf else None,
            "error_vs_fp64": d.get("error_vs_fp64"),
            "e2e": (d.get("e2e") or {}).get("value"),
            "looped_single_grid": (d.get("looped_single_grid") or {}).get("value"),
            "clocks": d.get("clocks"),
        })
        out.append(entry)
    return out


def rel_errors(got, ref, u0):
    """max |a - b| / max(max|b|, max|u0|) and ||a - b||_2 / ||b||_2 (the first
    stays meaningful where the solution has decayed to rounding noise)."""
    denom = max(float(np.max(np.abs(ref))), float(np.max(np.abs(u0))))
    d = got - ref
    return float(np.max(np.abs(d)) / denom), float(np.linalg.norm(d) / max(np.linalg.norm(ref), 1e-300))


def fp64_oracle_of(w, state_host):
    """Initial state of the FP64 oracle run that a reduced-precision workload
    is compared with (its stored values, exactly, in binary64)."""
    if w.op == "heat_kahan":
        return storage_to_f64(state_host[:1], w.dtype)
    U0 = storage_to_f64(state_host[:4], w.dtype)
    return np.concatenate([U0, U0])


def accuracy_report(w, sw, state_host, state_dev, out_sw, stream, Swept2D, full=True,
                    oracle_steps=None):
    """Error against FP64, on the final state of the timed run (all of the
    workload's steps) against the CPU oracle run over the same steps from the
    same initial values: for the FP64 workloads whether every point is equal
    to the oracle's, and the max-norm and L2 errors; for the reduced-precision
    forms the same errors against the FP64 oracle (the Euler form compares the
    four conserved variables), plus a bitwise check of the precision path
    itself against its own oracle after a few steps, and for those forms the
    same errors over all steps against the GPU FP64 path of the same update
    (bitwise equal to the oracle in the parity tests). With full=False the
    oracle comparison is made after 53 steps (20 for Euler) instead, with
    oracle_steps after that many."""
    import torch
    N = w.grid
    rep = {}
    t0 = time.perf_counter()
    if full and (oracle_steps is None or oracle_steps >= w.nsteps):
        nsteps_ref, got = w.nsteps, out_sw
    else:
        nsteps_ref = oracle_steps or (20 if w.op in ("euler_rk2", "euler_kahan") else 53)
        with torch.cuda.stream(stream):
            sw.set_state(state_dev)
            sw.advance(nsteps_ref)
        got = sw.get_state()
    if w.op in ("heat", "wave", "euler_rk2"):
        ref = oracle_advance(w, state_host, nsteps_ref)
        nv = 4 if w.op == "euler_rk2" else ref.shape[0]
        got64, ref64 = got[:nv].astype(np.float64), ref[:nv].astype(np.float64)
        mx, l2 = rel_errors(got64, ref64, state_host[:nv])
        rep.update({"reference": f"CPU FP64 oracle, {nsteps_ref} steps, every point",
                    "equal_to_oracle_bitwise": bool(np.array_equal(got[:nv], ref[:nv])),
                    "max_abs": float(np.max(np.abs(got64 - ref64))),
                    "max_rel": mx, "l2_rel": l2})
    else:
        # the precision path itself, bitwise against its oracle after a few steps
        nchk = 20
        with torch.cuda.stream(stream):
            sw.set_state(state_dev)
            sw.advance(nchk)
        own = sw.get_state()
        rep[f"equal_to_own_oracle_bitwise_{nchk}_steps"] = bool(
            np.array_equal(own, oracle_advance(w, state_host, nchk)))
        import oracle
        init64 = fp64_oracle_of(w, state_host)
        if w.op == "heat_kahan":
            ref64 = oracle.heat(init64[0], w.params[0], nsteps_ref)[None]
            U = storage_to_f64(got[:1], w.dtype)
            C = storage_to_f64(got[1:2], w.dtype)
        else:
            a, dt = oracle.euler_setup(init64[:4], GAMMA, CFL)
            ref64 = oracle.euler_rk2(init64[:4], GAMMA, dt, KAPPA, a, nsteps_ref)
            U = storage_to_f64(got[:4], w.dtype)
            C = storage_to_f64(got[8:12], w.dtype)
        mx, l2 = rel_errors(U, ref64, init64[:ref64.shape[0]])
        rep.update({"reference": f"CPU FP64 oracle, {nsteps_ref} steps from the same initial "
                                 "values, every point",
                    "max_rel": mx, "l2_rel": l2,
                    "u_minus_c_max_rel": rel_errors(U - C, ref64, init64[:ref64.shape[0]])[0]})
        if w.op == "euler_kahan":
            for v, name in enumerate(("rho", "m", "q", "E")):
                rep[f"{name}_max_rel"], rep[f"{name}_l2_rel"] = rel_errors(
                    U[v], ref64[v], init64[v])
        # all steps against the GPU FP64 path (the final state of the timed run)
        op64 = "heat" if w.op == "heat_kahan" else "euler_rk2"
        with Swept2D(N, N, op=op64, tile=w.tile, params=w.params, stream=stream) as f64:
            f64.set_state(np.ascontiguousarray(init64))
            f64.advance(w.nsteps)
            g64 = f64.get_state()[:ref64.shape[0]]
        Uf = storage_to_f64(out_sw[:g64.shape[0]], w.dtype)
        mx, l2 = rel_errors(Uf, g64, init64[:g64.shape[0]])
        rep["vs_gpu_fp64_all_steps"] = {"steps": w.nsteps, "max_rel": mx, "l2_rel": l2}
    rep["oracle_seconds"] = time.perf_counter() - t0
    return rep


def persistent_trace(sw, w, state_dev, stream, sm_mhz):
    """One persistent advance with the per-item trace on: the mean SM cycles
    (and microseconds at the sampled SM clock) a block waited for an item's
    3 x 3 neighbourhood and spent on the item, per kind of item."""
    import torch
    n, N = w.tile, w.grid
    NT = (N // n) ** 2
    nst = 2 if w.op in ("euler_rk2", "euler_kahan") else 1
    H = w.nsteps * nst // (n // 2)
    items = NT * (1 + 3 * H)
    buf = torch.zeros(2 * items, dtype=torch.int32, device="cuda")
    sw.set_trace(buf)
    with torch.cuda.stream(stream):
        sw.set_state(state_dev)
        sw.advance(w.nsteps, mode="persistent")
    torch.cuda.synchronize()
    sw.set_trace(None)
    t = buf.cpu().numpy().view(np.uint32).astype(np.float64).reshape(items, 2)
    kind = np.empty(items, dtype=object)
    kind[:NT] = "first_up"
    r = np.arange(items - NT) % (3 * NT)
    kind[NT:] = np.where(r < 2 * NT, "bridge", "octahedron")
    last = NT + (H - 1) * 3 * NT + 2 * NT
    kind[last:] = "final_down"
    mhz = sm_mhz or 2070.0
    out = {"sm_mhz_used": mhz, "items": int(items), "half_cycles": int(H)}
    for k in ("first_up", "bridge", "octahedron", "final_down"):
        sel = kind == k
        if sel.any():
            out[k] = {"count": int(sel.sum()),
                      "wait_us_mean": float(t[sel, 0].mean() / mhz),
                      "work_us_mean": float(t[sel, 1].mean() / mhz),
                      "wait_us_max": float(t[sel, 0].max() / mhz)}
    tot_wait, tot_work = t[:, 0].sum(), t[:, 1].sum()
    out["wait_share_of_block_time"] = float(tot_wait / max(tot_wait + tot_work, 1.0))
    return out


def naive_kernel_ms(nv, state_dev, stream, w):
    import torch
    nv.set_timing(True)
    with torch.cuda.stream(stream):
        nv.set_state(state_dev)
        nv.advance(20 if w.op in ("euler_rk2", "euler_kahan") else 200, mode="naive")
    n, ms = nv.kernel_stats("naive")
    nv.set_timing(False)
    return ms / max(1, n)


# ------------------------------------------------------------ batched form

def batch_sizes(seed, count=1024):
    rng = np.random.default_rng(seed)
    vals = np.arange(32, 513, 16)                 # {32, 48, ..., 512}
    return [int(v) for v in rng.choice(vals, size=count)], \
        [int(v) for v in rng.choice(vals, size=count)]


def batch_states(nx, ny, seed, dtype, op="heat_kahan"):
    """Per grid: heat (u, c = 0) from U[0,1) (seed 100000 seed + i), or Euler
    (U, U* = U, C = 0) from the pressure pulse (seed 100000 seed + i)."""
    from paper_1602_07558_gb300 import inputs
    parts = []
    for i, (a, b) in enumerate(zip(nx, ny)):
        if op == "euler_kahan":
            U = to_storage(inputs.euler_pulse(a, b, seed * 100_000 + i, gamma=GAMMA)
                           .astype(np.float32), dtype)
            parts.append(np.concatenate([U, U, np.zeros_like(U)]).reshape(-1))
            continue
        u = to_storage(inputs.uniform(a, b, seed * 100_000 + i).astype(np.float32), dtype)
        parts.append(np.stack([u, np.zeros_like(u)]).reshape(-1))
    return parts


def batch_oracle(w, part, a, b, nsteps):
    """The oracle on one grid of the batch (same layout as the grid's slice)."""
    import oracle
    if w.op == "euler_kahan":
        S = part.reshape(12, b, a)
        av, dt = oracle.euler_setup(storage_to_f64(S[:4], w.dtype), GAMMA, CFL)
        return oracle.euler_kahan(S, GAMMA, dt, KAPPA, av, nsteps, storage=w.dtype)
    st = part.reshape(2, b, a)
    return np.stack(oracle.heat_kahan(st[0], st[1], w.params[0], nsteps, storage=w.dtype))


def run_batch(args, w, world, rank, local):
    nx, ny = batch_sizes(w.seed + rank)
    count = len(nx)
    cells = sum(a * b for a, b in zip(nx, ny))
    parts = batch_states(nx, ny, w.seed + rank, w.dtype, w.op)
    nv = 12 if w.op == "euler_kahan" else 2
    flat = np.concatenate(parts)
    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        oracle.build()
        rng = np.random.default_rng(7)
        sample = sorted(rng.choice(count, size=16, replace=False).tolist())
        nsteps = max(1, args.nsteps or 200) if args.nsteps else 200
        t0 = time.perf_counter()
        done = 0
        for i in sample:
            batch_oracle(w, parts[i], nx[i], ny[i], nsteps)
            done += nx[i] * ny[i] * nsteps
        dt = time.perf_counter() - t0
        value = done / dt / 1e9
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": 1, "warmup": 0, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": w.dtype, "data": "synthetic",
            "config": {"workload": w.describe + " (CPU oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"16 of the {count} grids, {nsteps} steps each"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }), flush=True)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:                       # replicas: one batch per rank, max time over ranks
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1602_07558_gb300.autotune import autotune_batch
    from paper_1602_07558_gb300.swept2d import Swept2D, SweptBatch
    stream = torch.cuda.Stream()
    dev = torch.from_numpy(flat).to("cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    nsteps = w.nsteps
    cand = tuple(int(t) for t in args.batch_tiles.split(","))
    tiles, class_tuning, tune_table = autotune_batch(nx, ny, w.op, w.params, dtype=w.dtype,
                                                     stream=stream, tiles=cand)
    stage = {str(k): v for k, v in class_tuning.items()}
    sw_mode = ("persistent_one" if args.one_launch else "persistent") \
        if args.persistent else "swept"

    def tuned(sb):
        if args.persistent and args.one_launch:
            # one block shape for every class (the batch-wide tuning)
            sb.set_tuning(args.threads or 256, args.stage or 0)
        else:
            for tile_n, (thr, stg) in class_tuning.items():
                sb.set_tuning(thr, stg, tile=tile_n)

    if args.profile_case:             # one short advance in the default form, for ncu
        with SweptBatch(nx, ny, tiles, op=w.op, params=w.params, stream=stream,
                        dtype=w.dtype) as sb:
            tuned(sb)
            with torch.cuda.stream(stream):
                sb.set_state(dev)
                sb.advance(64, mode=sw_mode)
            torch.cuda.synchronize()
        print(json.dumps({"profile_case": True, "workload": w.describe, "mode": sw_mode}),
              flush=True)
        return

    def timed(b, mode, k, wu):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        times, l0 = [], 0
        for i in range(wu + k):
            if i == wu:
                if dist is not None:
                    dist.barrier()
                torch.cuda.synchronize()
                l0 = b.query("launches")
            with torch.cuda.stream(stream):
                flush.zero_()
                ev0.record(stream)
                b.set_state(dev)
                b.advance(nsteps, mode=mode, graph=True)
                ev1.record(stream)
            ev1.synchronize()
            if i >= wu:
                times.append(ev0.elapsed_time(ev1))
        if dist is not None:
            dist.barrier()
        return statistics.mean(times), int(b.query("launches") - l0)

    with ClockSampler(local) as clocks:
        with SweptBatch(nx, ny, tiles, op=w.op, params=w.params, stream=stream,
                        dtype=w.dtype) as sb:
            tuned(sb)
            ms_sw, launches = timed(sb, sw_mode, args.steps, args.warmup)
            out_sw = sb.get_state()
            h_in = torch.from_numpy(flat.copy()).pin_memory()
            h_out = torch.empty_like(h_in).pin_memory()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sb.set_state(h_in)
            sb.advance(nsteps, mode=sw_mode, graph=True)
            sb.get_state(h_out)
            e2e_s = time.perf_counter() - t0
        naive_ms = None
        if not args.no_naive:
            with SweptBatch(nx, ny, [0] * count, op=w.op, params=w.params, stream=stream,
                            dtype=w.dtype) as nb:
                naive_ms, _ = timed(nb, "naive", args.steps, args.warmup)
                same = bool(np.array_equal(out_sw, nb.get_state()))
        # looping single-grid swept runs, one handle per grid, on a random sample
        rng = np.random.default_rng(11)
        sample = sorted(rng.choice(count, size=16, replace=False).tolist())
        loop_ms, loop_cells = 0.0, 0
        for i in sample:
            with Swept2D(nx[i], ny[i], op=w.op, tile=tiles[i], params=w.params, stream=stream,
                         dtype=w.dtype) as h:
                st = torch.from_numpy(parts[i]).to("cuda")
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                for rep in range(2):
                    with torch.cuda.stream(stream):
                        h.set_state(st)
                        ev0.record(stream)
                        h.advance(nsteps, graph=True)
                        ev1.record(stream)
                    ev1.synchronize()
                loop_ms += ev0.elapsed_time(ev1)
                loop_cells += nx[i] * ny[i]
    ms_sw, value = aggregate_over_ranks(ms_sw, cells, nsteps, dist, "cuda")
    naive_value = None
    if naive_ms:
        naive_ms, naive_value = aggregate_over_ranks(naive_ms, cells, nsteps, dist, "cuda")
    loop_value = loop_cells * nsteps / (loop_ms * 1e-3) / 1e9
    # error against FP64 on four sample grids (the GPU FP64 path of the same
    # update from the same values, bitwise the oracle in the parity tests)
    split, off = [], 0
    for a, b in zip(nx, ny):
        split.append(out_sw[off:off + nv * a * b].reshape(nv, b, a))
        off += nv * a * b
    errs = []
    for i in sample[:4]:
        v0 = storage_to_f64(parts[i].reshape(nv, ny[i], nx[i]), w.dtype)
        if w.op == "euler_kahan":
            f64 = Swept2D(nx[i], ny[i], op="euler_rk2", tile=16, params=w.params, stream=stream)
            init = np.concatenate([v0[:4], v0[:4]])
        else:
            f64 = Swept2D(nx[i], ny[i], op="heat", tile=16, params=w.params, stream=stream)
            init = v0[:1]
        with f64:
            f64.set_state(np.ascontiguousarray(init))
            f64.advance(nsteps)
            ref = f64.get_state()[:4 if w.op == "euler_kahan" else 1]
        got = storage_to_f64(split[i][:ref.shape[0]], w.dtype)
        denom = max(np.max(np.abs(ref)), np.max(np.abs(init)))
        errs.append(float(np.max(np.abs(got - ref)) / denom))
    # parity of the two smallest grids against the oracle (every point)
    import oracle
    oracle.build()
    smallest = sorted(range(count), key=lambda i: nx[i] * ny[i])[:2]
    par = [bool(np.array_equal(split[i], batch_oracle(w, parts[i], nx[i], ny[i], nsteps)))
           for i in smallest]
    class_counts = {}
    for t in tiles:
        class_counts[str(t)] = class_counts.get(str(t), 0) + 1
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(1, args.warmup // 3), "ms_per_step": ms_sw, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": w.dtype, "data": "synthetic",
            "config": {"workload": w.describe, "grids": count, "cells": cells,
                       "tiles_chosen": class_counts, "persistent": bool(args.persistent),
                       "one_launch": bool(args.persistent and args.one_launch),
                       "class_tuning (threads, stage)": stage,
                       "autotune": tune_table,
                       "cuda_graph": True, "l2": "flushed (256 MB write) between timed steps"},
            "naive_batched": {"value": naive_value, "unit": UNIT, "ms_per_step": naive_ms,
                              "note": "one naive launch per sub-step covering all grids, graph"},
            "looped_single_grid": {"value": loop_value, "unit": UNIT,
                                   "sample": "16 random grids, one swept handle each, graph",
                                   "estimated_ms_all_grids": loop_ms * cells / loop_cells},
            "speedup_vs_naive": value / naive_value if naive_value else None,
            "speedup_vs_looped": value / loop_value,
            "swept_equals_naive_bitwise": same if not args.no_naive else None,
            "oracle_parity_two_smallest_grids": par,
            "error_vs_fp64": {"max_rel_4_sample_grids": errs,
                              "fp64_reference": "GPU FP64 path of the same update from the same "
                                                "initial values"},
            "e2e": {"value": cells * nsteps / e2e_s / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": int(flat.nbytes), "d2h_bytes_per_step": int(flat.nbytes)},
            "gpu_launches": launches, "clocks": clocks.summary(),
        }), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
