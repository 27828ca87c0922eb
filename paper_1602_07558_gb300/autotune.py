"""Autotuner for the swept path's launch shape.

For one grid and point update it times a short swept advance for every
candidate tile side n (even, dividing nx and ny, fitting shared memory),
threads per block and panel staging, and returns the fastest. All candidates
give bitwise the same result, so the choice is purely about speed. The probe
runs whole half cycles of every candidate tile (4 of the largest), timed with
CUDA events on the given stream after one warm-up pass.

The cost model of the paper (Section 4, eq. (cost): n^2 s + 4 tau / n per
sub-step) predicts an optimum n* = (2 tau / s)^(1/3); here tau is a kernel
boundary and s the time of one point update, and the measured table stands in
for the model.
"""
from __future__ import annotations

from .swept2d import Swept2D, SweptError


def candidates(nx, ny, tiles=(16, 32, 64), threads=(64, 128, 256, 512), stages=(False, True)):
    for n in tiles:
        if nx % n == 0 and ny % n == 0:
            for t in threads:
                for st in stages:
                    yield n, t, st


def autotune(nx, ny, op, params, dtype=None, state=None, stream=None, probe_steps=None,
             tiles=(16, 32, 64), threads=(64, 128, 256, 512), stages=(False, True)):
    """Returns ((tile, threads, stage), table) with table a list of
    {"tile", "threads", "stage", "ms", "gcell_per_s"} for every candidate that ran."""
    import torch
    table = []
    valid = [n for n in tiles if nx % n == 0 and ny % n == 0]
    if not valid:
        raise ValueError("no candidate tile divides the grid")
    nst = {"euler_rk2": 2, "wide2": 2}.get(op, 1)
    if probe_steps is None:
        probe_steps = max(4 * (max(valid) // 2) // nst, 8)
    stream = stream or torch.cuda.current_stream()
    for n in valid:
        try:
            s = Swept2D(nx, ny, op=op, tile=n, params=params, stream=stream, dtype=dtype)
        except SweptError:
            continue
        with s:
            for t in threads:
                for st in stages:
                    try:
                        s.set_tuning(t, st)
                    except SweptError:
                        continue
                    ev0 = torch.cuda.Event(enable_timing=True)
                    ev1 = torch.cuda.Event(enable_timing=True)
                    times = []
                    for rep in range(2):
                        with torch.cuda.stream(stream):
                            if state is not None:
                                s.set_state(state)
                            else:
                                s.set_state(torch.zeros(s.shape, device="cuda",
                                                        dtype=_torch_dtype(s.np_dtype)))
                            ev0.record(stream)
                            s.advance(probe_steps)
                            ev1.record(stream)
                        ev1.synchronize()
                        times.append(ev0.elapsed_time(ev1))
                    ms = times[-1]
                    table.append({"tile": n, "threads": t, "stage": bool(st), "ms": ms,
                                  "gcell_per_s": nx * ny * probe_steps / (ms * 1e-3) / 1e9})
    if not table:
        raise RuntimeError("no candidate could run")
    best = min(table, key=lambda r: r["ms"])
    return (best["tile"], best["threads"], best["stage"]), table


def _torch_dtype(np_dtype):
    import numpy as np
    import torch
    return {np.dtype(np.float64): torch.float64, np.dtype(np.float32): torch.float32,
            np.dtype(np.uint16): torch.int16, np.dtype(np.uint64): torch.int64}[np.dtype(np_dtype)]


def size_class(nx, ny, tiles=(16, 32, 64)):
    """The tile sides that divide both nx and ny (the grid's candidates)."""
    return tuple(n for n in tiles if nx % n == 0 and ny % n == 0)


def _probe_state(b, op):
    """A valid state for timing probes: zeros, or for the Euler updates a gas at
    rest (rho = 1, E = 2.5) in every grid (zeros would divide by zero)."""
    import numpy as np
    import torch
    dt = _torch_dtype(b.np_dtype)
    if op not in ("euler_rk2", "euler_kahan"):
        return torch.zeros(b.total, device="cuda", dtype=dt)
    parts = []
    for a, c in zip(b.nx, b.ny):
        U = np.zeros((b.nvars, c, a), np.float32)
        U[0] = U[4] = 1.0
        U[3] = U[7] = 2.5
        parts.append(U.reshape(-1))
    host = torch.from_numpy(np.concatenate(parts))
    if dt == torch.int16:                      # bfloat16 bits
        host = host.to(torch.bfloat16).view(torch.int16)
    elif dt == torch.float64:
        host = host.double()
    return host.to("cuda")


def autotune_batch(nx, ny, op, params, dtype=None, state=None, stream=None, probe_steps=64,
                   tiles=(16, 32, 64), stages=(False, True), threads=(64, 128, 256)):
    """Per size class (grids sharing the same candidate tiles), time each
    candidate tile, threads per block and staging on that class's own grids (a
    batch of them, so the probe launches have the real width) and keep the
    fastest. Returns (tiles per grid, {tile: (threads, stage)}, table)."""
    import numpy as np
    import torch

    from .swept2d import SweptBatch
    classes = {}
    for i, (a, b) in enumerate(zip(nx, ny)):
        classes.setdefault(size_class(a, b, tiles), []).append(i)
    stream = stream or torch.cuda.current_stream()
    choice = [0] * len(nx)
    table = []
    best_stage = {}
    for cand, members in classes.items():
        if not cand:
            continue
        sub_nx = [nx[i] for i in members]
        sub_ny = [ny[i] for i in members]
        best = None
        for n in cand:
            try:
                b = SweptBatch(sub_nx, sub_ny, [n] * len(members), op=op, params=params,
                               stream=stream, dtype=dtype)
            except SweptError:
                continue
            with b:
                zeros = _probe_state(b, op)
                for t in threads:
                    for st in stages:
                        try:
                            b.set_tuning(t, st)
                        except SweptError:
                            continue
                        ev0 = torch.cuda.Event(enable_timing=True)
                        ev1 = torch.cuda.Event(enable_timing=True)
                        ms = None
                        for rep in range(2):
                            with torch.cuda.stream(stream):
                                b.set_state(zeros)
                                ev0.record(stream)
                                b.advance(probe_steps, graph=True)
                                ev1.record(stream)
                            ev1.synchronize()
                            ms = ev0.elapsed_time(ev1)
                        cells = float(np.sum(np.array(sub_nx) * np.array(sub_ny)))
                        row = {"class": list(cand), "grids": len(members), "tile": n,
                               "threads": t, "stage": st, "ms": ms,
                               "gcell_per_s": cells * probe_steps / (ms * 1e-3) / 1e9}
                        table.append(row)
                        if best is None or ms < best["ms"]:
                            best = row
        for i in members:
            choice[i] = best["tile"]
        best_stage[best["tile"]] = (best["threads"], best["stage"])
    return choice, best_stage, table
