"""The bench's roofline arithmetic (CPU): update counts of the swept kernels
from the level geometry, the slowest of the four bounds, and the error metric.
The counts are checked against a brute-force walk of the levels; the bound
choice against hand-computed times."""
import importlib.util
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
bench = importlib.util.module_from_spec(spec)
sys.modules["bench"] = bench          # (its dataclasses look their module up there)
spec.loader.exec_module(bench)


@pytest.mark.parametrize("n", [4, 8, 16, 32, 64])
def test_update_counts_partition_a_half_cycle(n):
    """An octahedron (Down of one half cycle, Up of the next) and the two
    bridges of a tile together compute every point of the tile at every level
    of a half cycle: octahedron + bridges = n^2 n/2 updates per tile, with the
    octahedron's share counted over the down squares and the up squares."""
    h = n // 2
    down = sum((2 * k + 2) ** 2 for k in range(h))            # levels 1..h of the Down
    up = sum((n - 2 * k - 2) ** 2 for k in range(h - 1))      # levels 1..h-1 of the Up
    bridges = 2 * sum((n - 2 * k - 2) * (2 * k + 2) for k in range(h - 1))
    assert bench.octahedron_updates(n) == down + up
    assert bench.bridge_updates(n) == bridges
    # every point of the tile at every level of a half cycle, exactly once:
    # at levels 1..h-1 the Up square, the two bridges and the Down square
    # partition the tile (Section 3's four components); level h is the Down's
    # whole tile
    assert down + up + bridges == n * n * h
    per_level = [(n - 2 * t) ** 2 + 4 * t * (n - 2 * t) + (2 * t) ** 2 for t in range(1, h + 1)]
    assert all(v == n * n for v in per_level)


def test_the_slowest_bound_is_reported():
    w = bench.WORKLOADS["heat4096"]
    peaks = {"fp64_ops_per_s": 500e9, "fp32_ops_per_s": 40e12, "smem_wavefronts_per_s": 300e9}
    upd = 1_000_000
    # FP64: 4 ops/update -> 8 us; HBM 1.5 MB at the file's peak -> ~0.2 us
    r = bench.bounds(w, 8, upd, 1.5e6, 10e-6, peaks)
    assert r["bound"] == "fp64"
    assert r["frac"] == pytest.approx(4 * upd / 500e9 / 10e-6)
    assert r["achieved"] == pytest.approx(4 * upd / 10e-6 / 1e9)
    # the same work with a huge byte count is HBM-bound
    r = bench.bounds(w, 8, upd, 1e12, 1.0, peaks)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    # binary32 heat: 9 FP32 ops, 4 shared accesses of 4 bytes = 4/32 wavefronts
    wk = bench.WORKLOADS["heat2048_f32"]
    r = bench.bounds(wk, 4, upd, 0.0, 1.0, peaks)
    assert r["bound"] == "smem"
    assert r["all_bounds_frac"]["smem"] == pytest.approx(4 * upd / 32 / 300e9)
    assert r["all_bounds_frac"]["fp32"] == pytest.approx(9 * upd / 40e12)


def test_relative_error_uses_the_larger_of_the_solution_and_the_start():
    """max |a - b| / max(max|b|, max|u0|): a decayed solution (~1e-15 of its
    start) does not inflate the error."""
    u0 = np.array([1.0, -1.0])
    ref = np.array([1e-15, -1e-15])
    got = ref + np.array([1e-17, 0.0])
    mx, l2 = bench.rel_errors(got, ref, u0)
    assert mx == pytest.approx(1e-17)
    assert l2 == pytest.approx(1e-17 / np.linalg.norm(ref))


def test_secondary_lines_summarise_each_child_run(monkeypatch):
    """The default run's other workloads: one child process per entry of
    SECONDARY, its last JSON line summarised; a failing child is recorded as
    an error and does not stop the others."""
    import json
    import subprocess
    calls = []

    class Done:
        def __init__(self, rc, out, err=""):
            self.returncode, self.stdout, self.stderr = rc, out, err

    def fake_run(cmd, **kw):
        calls.append(cmd)
        name = cmd[cmd.index("--workload") + 1]
        if name == "wave1024":
            return Done(1, "", "boom")
        line = {"value": 10.0, "unit": "Gcell-updates/s", "ms_per_step": 5.0,
                "config": {"workload": name, "nsteps": 7, "tile": 16, "persistent": False,
                           "cuda_graph": False},
                "naive": {"value": 8.0}, "speedup_vs_naive": 1.25,
                "swept_equals_naive_bitwise": True,
                "roofline": {"bound": "fp64", "frac": 0.5, "unit": "Gop/s", "traffic": None,
                             "extra": 1},
                "error_vs_fp64": {"max_rel": 0.0}, "e2e": {"value": 9.0},
                "clocks": {"sm_mhz": 2070.0}}
        return Done(0, "noise\n" + json.dumps(line) + "\n")

    monkeypatch.setattr(subprocess, "run", fake_run)
    out = bench.secondary_lines()
    assert [e["workload"] for e in out] == [n for n, _ in bench.SECONDARY]
    for cmd, (name, extra) in zip(calls, bench.SECONDARY):
        assert cmd[cmd.index("--steps") + 1] == "3" and cmd[cmd.index("--warmup") + 1] == "3"
        assert "--no-secondary" in cmd and "--no-cpu" in cmd
        assert cmd[-len(extra):] == list(extra) if extra else True
    bad = [e for e in out if e["workload"] == "wave1024"]
    assert bad and "boom" in bad[0]["error"]
    good = [e for e in out if "error" not in e]
    assert good and all(e["value"] == 10.0 and e["speedup_vs_naive"] == 1.25 for e in good)
    assert good[0]["roofline"] == {"bound": "fp64", "frac": 0.5, "unit": "Gop/s", "traffic": None}


def test_the_default_run_measures_every_workload():
    """The headline plus the secondary list cover every workload the bench
    defines, each batch in both of its forms."""
    names = {n for n, _ in bench.SECONDARY} | {bench.DEFAULT_WORKLOAD}
    assert names == set(bench.WORKLOADS)
    batch_forms = [(n, a) for n, a in bench.SECONDARY if n.startswith("batch")]
    for n in ("batch1024", "batch1024_euler"):
        assert len([1 for m, _ in batch_forms if m == n]) == 2
