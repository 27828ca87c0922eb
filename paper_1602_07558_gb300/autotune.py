"""Autotuner for the swept path's launch shape, seeded by the paper's cost model.

Section 4, eq. (cost): one sub-step of a swept half cycle costs n^2 s + 4 tau / n
on a node that owns an n x n tile (s the time of one point update, tau the
latency of one exchange). On one GPU all tiles of an N x N grid run at once, so
the time of one sub-step over the grid reads t(n) = N^2 s + 4 tau / n, with tau
now the cost of a kernel boundary (or a phase wait) per half cycle and s the
time per point update of the whole GPU. The tuner
  1. times a short swept advance at the smallest and the largest candidate
     tile (default launch shape) and fits s and tau to those two probes,
  2. predicts t(n) for every candidate tile and ranks them,
  3. times every launch shape (threads per block, panel staging) of the
     best-ranked tiles only,
and returns the fastest, with a table of predicted against measured times.
Within the model the optimum tile is n* = (2 tau / s')^(1/3) per node (s' the
time of one point update on that node); across a whole GPU the 4 tau / n term
alone depends on n, so the model favours large tiles and the measured table
(occupancy, panel and border overheads, which the model leaves out) decides.
Steps per stage are n/2 for tile n (the swept rule advances each tile n/2
sub-steps between exchanges), so choosing the tile chooses them.
All candidates give bitwise the same result, so the choice is purely about speed.
"""
from __future__ import annotations

from .swept2d import Swept2D, SweptError


def fit_cost_model(N2, probes):
    """s and tau of t(n) = N2 s + 4 tau / n from two (n, seconds per sub-step)
    probes. Where the probes fall faster than 1/n (per-level overheads that
    the model leaves out grow as the tile shrinks) the exact fit would give
    s < 0; s is then taken as 0 and tau from the larger tile's probe, so the
    model still ranks the tiles by their 1/n term."""
    (na, ta), (nb, tb) = sorted(probes)
    if na == nb:
        return ta / N2, 0.0
    b = (ta - tb) / (1.0 / na - 1.0 / nb)          # 4 tau
    s = (ta - b / na) / N2
    if s < 0:
        return 0.0, tb * nb / 4.0
    return s, b / 4.0


def predict(N2, s, tau, n):
    return N2 * s + 4.0 * tau / n


def candidates(nx, ny, tiles=(16, 32, 64), threads=(64, 128, 256, 512), stages=(False, True)):
    for n in tiles:
        if nx % n == 0 and ny % n == 0:
            for t in threads:
                for st in stages:
                    yield n, t, st


def _time_advance(s, state, steps, stream):
    """ms of one advance of `steps` steps (second of two runs)."""
    import torch
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ms = None
    for rep in range(2):
        with torch.cuda.stream(stream):
            if state is not None:
                s.set_state(state)
            else:
                s.set_state(torch.zeros(s.shape, device="cuda", dtype=_torch_dtype(s.np_dtype)))
            ev0.record(stream)
            s.advance(steps)
            ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
    return ms


def autotune(nx, ny, op, params, dtype=None, state=None, stream=None, probe_steps=None,
             tiles=(16, 32, 64), threads=(64, 128, 256, 512), stages=(False, True), top=2):
    """Returns ((tile, threads, stage), table): table rows {"tile", "threads",
    "stage", "ms", "gcell_per_s", "predicted_ms"} for every candidate that ran,
    plus one {"model": ...} row with the fitted s and tau and the ranking."""
    import torch
    valid = [n for n in tiles if nx % n == 0 and ny % n == 0]
    if not valid:
        raise ValueError("no candidate tile divides the grid")
    nst = {"euler_rk2": 2, "euler_kahan": 2, "wide2": 2}.get(op, 1)
    if probe_steps is None:
        probe_steps = max(4 * (max(valid) // 2) // nst, 8)
    substeps = probe_steps * nst
    stream = stream or torch.cuda.current_stream()
    N2 = float(nx) * ny
    handles = {}

    def handle(n):
        if n not in handles:
            try:
                handles[n] = Swept2D(nx, ny, op=op, tile=n, params=params, stream=stream,
                                     dtype=dtype)
            except SweptError:
                handles[n] = None
        return handles[n]

    table = []
    try:
        # 1. the two probes of the model (default launch shape)
        probes = []
        for n in sorted({min(valid), max(valid)}):
            h = handle(n)
            if h is None:
                continue
            ms = _time_advance(h, state, probe_steps, stream)
            probes.append((n, ms * 1e-3 / substeps))
        if not probes:
            raise RuntimeError("no candidate could run")
        s_pt, tau = fit_cost_model(N2, probes if len(probes) == 2 else probes * 2)
        # 2. ranking by the model
        pred = {n: predict(N2, s_pt, tau, n) * substeps * 1e3 for n in valid}
        ranked = sorted(valid, key=lambda n: pred[n])
        # 3. every launch shape of the best-ranked tiles
        for n in ranked[:top]:
            h = handle(n)
            if h is None:
                continue
            for t in threads:
                for st in stages:
                    try:
                        h.set_tuning(t, st)
                    except SweptError:
                        continue
                    ms = _time_advance(h, state, probe_steps, stream)
                    table.append({"tile": n, "threads": t, "stage": bool(st), "ms": ms,
                                  "gcell_per_s": N2 * probe_steps / (ms * 1e-3) / 1e9,
                                  "predicted_ms": pred[n]})
    finally:
        for h in handles.values():
            if h is not None:
                h.close()
    if not table:
        raise RuntimeError("no candidate could run")
    best = min(table, key=lambda r: r["ms"])
    table.append({"model": "t(n) = N^2 s + 4 tau / n per sub-step (Section 4, eq. (cost))",
                  "s_ns_per_point_update": s_pt * 1e9, "tau_us": tau * 1e6,
                  "probes": [{"tile": n, "us_per_substep": t * 1e6} for n, t in probes],
                  "ranking": ranked, "timed_tiles": ranked[:top],
                  "predicted_ms": {str(n): pred[n] for n in valid}})
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
                   tiles=(16, 32, 64), stages=(False, True), threads=(32, 64, 128, 256), top=2):
    """Per size class (grids sharing the same candidate tiles), fit the cost
    model of autotune() to probes of the class's smallest and largest tile on
    the class's own grids (a batch of them, so the probe launches have the real
    width), rank the tiles by it, time every threads-per-block and staging
    setting of the best-ranked tiles and keep the fastest. Returns (tiles per
    grid, {tile: (threads, stage)}, table with predicted and measured times)."""
    import numpy as np
    import torch

    from .swept2d import SweptBatch
    classes = {}
    for i, (a, b) in enumerate(zip(nx, ny)):
        classes.setdefault(size_class(a, b, tiles), []).append(i)
    stream = stream or torch.cuda.current_stream()
    nst = {"euler_rk2": 2, "euler_kahan": 2}.get(op, 1)
    substeps = probe_steps * nst
    choice = [0] * len(nx)
    table = []
    best_stage = {}

    def timed(b, state):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ms = None
        for rep in range(2):
            with torch.cuda.stream(stream):
                b.set_state(state)
                ev0.record(stream)
                b.advance(probe_steps, graph=True)
                ev1.record(stream)
            ev1.synchronize()
            ms = ev0.elapsed_time(ev1)
        return ms

    for cand, members in classes.items():
        if not cand:
            continue
        sub_nx = [nx[i] for i in members]
        sub_ny = [ny[i] for i in members]
        cells = float(np.sum(np.array(sub_nx) * np.array(sub_ny)))
        batches = {}

        def batch(n):
            if n not in batches:
                try:
                    batches[n] = SweptBatch(sub_nx, sub_ny, [n] * len(members), op=op,
                                            params=params, stream=stream, dtype=dtype)
                except SweptError:
                    batches[n] = None
            return batches[n]

        best = None
        try:
            probes = []
            for n in sorted({min(cand), max(cand)}):
                b = batch(n)
                if b is not None:
                    probes.append((n, timed(b, _probe_state(b, op)) * 1e-3 / substeps))
            if not probes:
                continue
            s_pt, tau = fit_cost_model(cells, probes if len(probes) == 2 else probes * 2)
            pred = {n: predict(cells, s_pt, tau, n) * substeps * 1e3 for n in cand}
            ranked = sorted(cand, key=lambda n: pred[n])
            for n in ranked[:top]:
                b = batch(n)
                if b is None:
                    continue
                zeros = _probe_state(b, op)
                for t in threads:
                    for st in stages:
                        try:
                            b.set_tuning(t, st)
                        except SweptError:
                            continue
                        ms = timed(b, zeros)
                        row = {"class": list(cand), "grids": len(members), "tile": n,
                               "threads": t, "stage": st, "ms": ms,
                               "gcell_per_s": cells * probe_steps / (ms * 1e-3) / 1e9,
                               "predicted_ms": pred[n]}
                        table.append(row)
                        if best is None or ms < best["ms"]:
                            best = row
            table.append({"class": list(cand), "model": "t(n) = N^2 s + 4 tau / n per sub-step",
                          "s_ns_per_point_update": s_pt * 1e9, "tau_us": tau * 1e6,
                          "ranking": ranked, "predicted_ms": {str(n): pred[n] for n in cand}})
        finally:
            for b in batches.values():
                if b is not None:
                    b.close()
        if best is None:
            continue
        for i in members:
            choice[i] = best["tile"]
        best_stage[best["tile"]] = (best["threads"], best["stage"])
    return choice, best_stage, table
