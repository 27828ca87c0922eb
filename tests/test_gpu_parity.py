"""GPU parity: the CUDA paths (through the C ABI) against the CPU oracle.

Bar (stated per test): bitwise for the integer/word updates and for heat (the
GPU and the oracle evaluate the same IEEE operations in the same order);
swept == naive bitwise for every update (the same point-update code); Euler
within 1e-12 of the oracle in the max-norm relative to max(|oracle|, |u0|)
(the test also reports whether it is bitwise).
"""
import numpy as np
import pytest

from paper_1602_07558_gb300 import inputs
from paper_1602_07558_gb300.swept2d import Swept2D

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

GAMMA, CFL, KAPPA = 1.4, 0.3, 0.5


def run(op, u0, nsteps, tile, mode, params=(), chunks=None, dtype=None):
    ny, nx = u0.shape[-2:]
    with Swept2D(nx, ny, op=op, tile=tile, params=params, dtype=dtype) as s:
        s.set_state(np.ascontiguousarray(u0.reshape(s.shape)))
        for c in (chunks or [nsteps]):
            s.advance(c, mode=mode)
        return s.get_state()


# ------------------------------------------------------------------ heat, 64^2

def test_heat_64_uniform_512_steps_matches_oracle_bitwise(oracle_lib):
    """Heat, periodic 64 x 64, r = 0.2, 512 steps, U[0,1) from seed 0, tile 16."""
    u0 = inputs.uniform(64, 64, seed=0)
    ref = oracle_lib.heat(u0, 0.2, 512)
    naive = run("heat", u0, 512, 16, "naive", (0.2,))[0]
    swept = run("heat", u0, 512, 16, "swept", (0.2,))[0]
    assert np.array_equal(naive, ref)
    assert np.array_equal(swept, naive)


def test_heat_64_fourier_mode_matches_oracle_and_decays(oracle_lib):
    u0 = inputs.fourier_mode(64, 64, 3, 5)
    ref = oracle_lib.heat(u0, 0.2, 512)
    swept = run("heat", u0, 512, 16, "swept", (0.2,))[0]
    assert np.array_equal(swept, ref)
    g = 1.0 - 0.8 * (np.sin(np.pi * 3 / 64) ** 2 + np.sin(np.pi * 5 / 64) ** 2)
    assert np.max(np.abs(swept - g ** 512 * u0)) <= 4 * 512 * np.finfo(float).eps


@pytest.mark.parametrize("nx,ny,tile,nsteps", [
    (96, 64, 32, 77),      # several tiles, ragged tail (77 = 4*16 + 13)
    (64, 96, 16, 41),      # nx != ny the other way, odd number of half cycles + tail
    (40, 24, 8, 35),
    (32, 32, 4, 30),       # smallest tile
    (128, 64, 64, 100),    # largest FP64 heat tile that fits two level buffers
    (16, 48, 16, 21),      # one tile across x: a tile borders itself
    (64, 64, 16, 7),       # fewer steps than a half cycle: naive tail only
    (64, 64, 16, 0),
])
def test_heat_swept_equals_naive_and_oracle(oracle_lib, nx, ny, tile, nsteps):
    u0 = inputs.uniform(nx, ny, seed=nx + ny + tile)
    ref = oracle_lib.heat(u0, 0.2, nsteps)
    swept = run("heat", u0, nsteps, tile, "swept", (0.2,))[0]
    naive = run("heat", u0, nsteps, tile, "naive", (0.2,))[0]
    assert np.array_equal(naive, ref)
    assert np.array_equal(swept, ref)


# ---------------------------------------------------- test updates (bitwise)

@pytest.mark.parametrize("nx,ny,tile,nsub", [
    (64, 48, 16, 40), (48, 64, 8, 29), (24, 24, 4, 13), (32, 16, 16, 24), (16, 16, 16, 16),
])
def test_hash_swept_is_bitwise_the_oracle(oracle_lib, nx, ny, tile, nsub):
    """Any wrong, missing or stale neighbour in any swept component changes the
    64-bit mix; every level of every component is exercised."""
    u0 = inputs.random_words(nx, ny, seed=tile * 7 + nsub)[0]
    ref = oracle_lib.hash_op(u0, nsub)
    assert np.array_equal(run("hash", u0, nsub, tile, "swept")[0], ref)
    assert np.array_equal(run("hash", u0, nsub, tile, "naive")[0], ref)


def test_hash_sub_step_counter_runs_across_advance_calls(oracle_lib):
    u0 = inputs.random_words(32, 32, seed=1)[0]
    ref = oracle_lib.hash_op(u0, 3 + 16 + 5)
    got = run("hash", u0, None, 8, "swept", chunks=[3, 16, 5])[0]
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("tile,nsub", [(8, 24), (16, 40), (32, 48)])
def test_leveltag_every_point_sees_nine_neighbours_of_its_level(tile, nsub):
    u0 = np.zeros((64, 64))
    got = run("leveltag", u0, nsub, tile, "swept")[0]
    assert not np.isnan(got).any()
    assert np.all(got == nsub)


def test_increment_worked_example():
    """Section 3.1 example, 8 x 8 tiles on 4 subdomains, one full cycle."""
    got = run("increment", np.ones((16, 16)), 8, 8, "swept")[0]
    assert np.all(got == 9.0)


@pytest.mark.parametrize("tile,nsteps", [(8, 12), (16, 9), (4, 7)])
def test_wide2_two_substep_scheme_matches_direct_radius2(oracle_lib, tile, nsteps):
    """nstages = 2 with a 5-component point state through every component."""
    words = inputs.random_words(48, 32, seed=tile)[0]
    u0 = np.zeros((5, 32, 48), dtype=np.uint64)
    u0[0] = words
    ref = oracle_lib.wide2(words, nsteps)
    swept = run("wide2", u0, nsteps, tile, "swept")
    naive = run("wide2", u0, nsteps, tile, "naive")
    assert np.array_equal(swept, naive)
    assert np.array_equal(swept[0], ref)


# ---------------------------------------------------------------------- Euler

def _euler_u0(nx, ny, seed, literal=False):
    U = inputs.euler_pulse(nx, ny, seed, gamma=GAMMA, literal=literal)
    return np.concatenate([U, U]), U


@pytest.mark.parametrize("nx,ny,tile,nsteps", [(64, 48, 16, 40), (32, 32, 8, 13), (64, 64, 32, 20),
                                               (60, 40, 10, 17)])   # n = 2 mod 4: wider flux pitch
def test_euler_swept_equals_naive_and_oracle(oracle_lib, nx, ny, tile, nsteps):
    u0, U = _euler_u0(nx, ny, seed=2)
    a, dt = oracle_lib.euler_setup(U, GAMMA, CFL)
    ref = oracle_lib.euler_rk2(U, GAMMA, dt, KAPPA, a, nsteps)
    with Swept2D(nx, ny, op="euler_rk2", tile=tile, params=(GAMMA, CFL, KAPPA)) as s:
        s.set_state(u0)
        assert s.query("wavespeed") == a and s.query("dt") == dt
        s.advance(nsteps, mode="swept")
        swept = s.get_state()
    naive = run("euler_rk2", u0, nsteps, tile, "naive", (GAMMA, CFL, KAPPA))
    assert np.array_equal(swept, naive)
    denom = max(np.max(np.abs(ref)), np.max(np.abs(U)))
    assert np.max(np.abs(swept[:4] - ref)) / denom <= 1e-12
    assert np.array_equal(swept[:4], ref)      # same operations in the same order


# ------------------------------------------- reduced-precision forms (bitwise)

def _to_bf16_bits(a):
    """binary32 -> bfloat16 bits with torch's conversion (round to nearest even)."""
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16) \
        .view(torch.int16).numpy().view(np.uint16)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("nx,ny,tile,nsteps", [
    (96, 64, 32, 77), (64, 64, 16, 40), (32, 48, 8, 23), (128, 64, 64, 70),
    (60, 40, 10, 23),      # a tile side built only with the run-time side
])
def test_heat_kahan_swept_equals_naive_and_oracle(oracle_lib, storage, nx, ny, tile, nsteps):
    """Binary32 arithmetic, Kahan-compensated update, binary32 or bfloat16
    storage: u and c bit for bit the oracle's, swept == naive."""
    u32 = inputs.uniform(nx, ny, seed=nx + tile).astype(np.float32)
    u0 = u32 if storage == "f32" else _to_bf16_bits(u32)
    c0 = np.zeros_like(u0)
    ref_u, ref_c = oracle_lib.heat_kahan(u0, c0, 0.2, nsteps, storage=storage)
    state = np.stack([u0, c0])
    swept = run("heat_kahan", state, nsteps, tile, "swept", (0.2,), dtype=storage)
    naive = run("heat_kahan", state, nsteps, tile, "naive", (0.2,), dtype=storage)
    assert np.array_equal(swept, naive)
    assert np.array_equal(swept[0], ref_u)
    assert np.array_equal(swept[1], ref_c)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_heat_kahan_2048_full_grid_matches_oracle(oracle_lib, storage):
    """The precision workload's grid and tile (2048 x 2048, n = 32), 3 half
    cycles and a tail, every point of u and c against the oracle."""
    u32 = inputs.smooth_field(2048, 2048, seed=1).astype(np.float32)
    u0 = u32 if storage == "f32" else _to_bf16_bits(u32)
    c0 = np.zeros_like(u0)
    ref_u, ref_c = oracle_lib.heat_kahan(u0, c0, 0.2, 53, storage=storage)
    got = run("heat_kahan", np.stack([u0, c0]), 53, 32, "swept", (0.2,), dtype=storage)
    assert np.array_equal(got[0], ref_u) and np.array_equal(got[1], ref_c)


# ------------------------------------------------- launch shape never matters

@pytest.mark.parametrize("op,dtype,params", [
    ("heat", "f64", (0.2,)), ("heat_kahan", "f32", (0.2,)), ("heat_kahan", "bf16", (0.2,)),
    ("hash", "u64", ()), ("wide2", "u64", ()), ("euler_kahan", "f32", (GAMMA, CFL, KAPPA)),
])
@pytest.mark.parametrize("threads,stage", [(32, False), (32, True), (64, False), (128, True),
                                           (256, True), (256, False), (512, False), (512, True)])
def test_tuning_gives_identical_bits(op, dtype, params, threads, stage):
    """Threads per block and TMA panel staging change the schedule, never the
    result: every setting equals the naive path bit for bit."""
    nx, ny, tile, nsteps = 64, 48, 16, 37
    rng = np.random.default_rng(threads + stage)
    shape = {"heat": 1, "heat_kahan": 2, "hash": 1, "wide2": 5, "euler_kahan": 12}[op]
    if op == "euler_kahan":
        u0 = _euler_kahan_state(nx, ny, dtype, seed=threads + stage)
    elif dtype == "f64":
        u0 = rng.random((shape, ny, nx))
    elif dtype == "f32":
        u0 = np.stack([rng.random((ny, nx)), np.zeros((ny, nx))]).astype(np.float32)
    elif dtype == "bf16":
        u0 = np.stack([_to_bf16_bits(rng.random((ny, nx))), np.zeros((ny, nx), np.uint16)])
    else:
        u0 = rng.integers(0, 2**64, size=(shape, ny, nx), dtype=np.uint64)
    naive = run(op, u0, nsteps, tile, "naive", params, dtype=dtype)
    with Swept2D(nx, ny, op=op, tile=tile, params=params, dtype=dtype) as s:
        s.set_tuning(threads, stage)
        s.set_state(np.ascontiguousarray(u0))
        s.advance(nsteps)
        got = s.get_state()
    assert np.array_equal(got, naive)


# ----------------------------------------------------------------------- wave

@pytest.mark.parametrize("nx,ny,tile,nsteps", [(64, 64, 16, 100), (96, 64, 32, 45), (48, 32, 8, 19),
                                               (60, 40, 10, 21)])
def test_wave_swept_equals_naive_and_oracle(oracle_lib, nx, ny, tile, nsteps):
    """Leapfrog wave (Section 6's experiment, Courant number 0.3): the 2-value
    point state (u^n, u^{n-1}) through every swept component, bitwise."""
    u0 = inputs.wave_source(nx, ny)
    ref_u, ref_uo = oracle_lib.wave(u0[0], u0[1], 0.3 * 0.3, nsteps)
    swept = run("wave", u0, nsteps, tile, "swept", (0.3,))
    naive = run("wave", u0, nsteps, tile, "naive", (0.3,))
    assert np.array_equal(swept, naive)
    assert np.array_equal(swept[0], ref_u) and np.array_equal(swept[1], ref_uo)


def _euler_kahan_state(nx, ny, storage, seed):
    U = inputs.euler_pulse(nx, ny, seed, gamma=GAMMA).astype(np.float32)
    if storage == "bf16":
        U = _to_bf16_bits(U)
    return np.concatenate([U, U, np.zeros_like(U)])


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("nx,ny,tile,nsteps", [(64, 48, 16, 21), (32, 32, 8, 13), (64, 64, 32, 20),
                                               (60, 40, 10, 17), (36, 24, 6, 11)])
def test_euler_kahan_swept_equals_naive_and_oracle(oracle_lib, storage, nx, ny, tile, nsteps):
    """Euler in binary32 arithmetic with compensated update and binary32 /
    bfloat16 storage: all 12 planes (U, U*, C) bit for bit the oracle's, and
    swept == naive; a and dt (formed in FP64 from the stored values) exactly
    the oracle's."""
    S = _euler_kahan_state(nx, ny, storage, seed=5)
    Uf = (oracle_lib.bf16_bits_to_f32(S[:4]) if storage == "bf16" else S[:4]).astype(np.float64)
    a, dt = oracle_lib.euler_setup(Uf, GAMMA, CFL)
    ref = oracle_lib.euler_kahan(S, GAMMA, dt, KAPPA, a, nsteps, storage)
    params = (GAMMA, CFL, KAPPA)
    with Swept2D(nx, ny, op="euler_kahan", tile=tile, params=params, dtype=storage) as s:
        s.set_state(S)
        assert s.query("wavespeed") == a and s.query("dt") == dt
        s.advance(nsteps, mode="swept")
        swept = s.get_state()
    naive = run("euler_kahan", S, nsteps, tile, "naive", params, dtype=storage)
    assert np.array_equal(swept, naive)
    assert np.array_equal(swept, ref)


# ---------------------------------------------------------- persistent form

@pytest.mark.parametrize("op,dtype,nx,ny,tile,nsteps", [
    ("hash", "u64", 64, 48, 16, 61),      # all 9 neighbours: any missed dependency shows
    ("hash", "u64", 32, 16, 8, 40),       # fewer than 3 tiles across: neighbourhoods wrap
    ("hash", "u64", 16, 16, 16, 33),      # a single tile borders itself
    ("heat", "f64", 128, 96, 32, 77),
    ("heat", "f64", 128, 128, 64, 100),
    ("heat_kahan", "f32", 96, 64, 16, 45),
    ("heat_kahan", "bf16", 64, 64, 32, 50),
    ("wide2", "u64", 48, 32, 8, 19),      # nstages = 2
    ("wave", "f64", 64, 64, 16, 70),
    ("euler_rk2", "f64", 32, 32, 16, 9),
    ("euler_kahan", "f32", 32, 32, 16, 11),
    ("euler_kahan", "bf16", 64, 32, 16, 12),
])
def test_persistent_form_gives_the_same_bits(oracle_lib, op, dtype, nx, ny, tile, nsteps):
    """One persistent launch per advance (work items with neighbourhood waits)
    equals the naive path bit for bit, with panels staged by TMA and copied
    element-wise, also through a captured graph."""
    rng = np.random.default_rng(nx + ny + tile)
    nv = {"hash": 1, "heat": 1, "heat_kahan": 2, "wide2": 5, "wave": 2, "euler_rk2": 8,
          "euler_kahan": 12}[op]
    params = {"hash": (), "wide2": (), "heat": (0.2,), "heat_kahan": (0.2,), "wave": (0.3,),
              "euler_rk2": (GAMMA, CFL, KAPPA), "euler_kahan": (GAMMA, CFL, KAPPA)}[op]
    if op == "euler_kahan":
        u0 = _euler_kahan_state(nx, ny, dtype, seed=6)
    elif dtype == "u64":
        u0 = rng.integers(0, 2**64, size=(nv, ny, nx), dtype=np.uint64)
    elif dtype == "f32":
        u0 = np.stack([rng.random((ny, nx)), np.zeros((ny, nx))]).astype(np.float32)
    elif dtype == "bf16":
        u0 = np.stack([_to_bf16_bits(rng.random((ny, nx))), np.zeros((ny, nx), np.uint16)])
    elif op == "euler_rk2":
        u0 = _euler_u0(nx, ny, seed=4)[0]
    else:
        u0 = rng.random((nv, ny, nx))
    naive = run(op, u0, nsteps, tile, "naive", params, dtype=dtype)
    stream = torch.cuda.Stream()
    from paper_1602_07558_gb300.swept2d import SweptError
    for stage in (False, True):
        with Swept2D(nx, ny, op=op, tile=tile, params=params, dtype=dtype, stream=stream) as s:
            try:
                s.set_tuning(128 if stage else 256, stage)
            except SweptError:
                continue                    # the staged panels do not fit at this tile
            s.set_state(np.ascontiguousarray(u0))
            s.advance(nsteps, mode="persistent")
            assert np.array_equal(s.get_state(), naive), stage
            s.set_state(np.ascontiguousarray(u0))
            s.advance(nsteps, mode="persistent", graph=True)
            assert np.array_equal(s.get_state(), naive), stage


def test_persistent_wait_timeout_is_reported_and_the_context_stays_usable(oracle_lib):
    """A neighbourhood wait that can never be satisfied gives up after its
    bound, the host reads ETIMEOUT, and the same handle then advances
    correctly."""
    from paper_1602_07558_gb300.swept2d import ETIMEOUT
    u0 = inputs.uniform(64, 64, seed=8)
    ref = oracle_lib.heat(u0, 0.2, 40)
    with Swept2D(64, 64, op="heat", tile=16, params=(0.2,)) as s:
        s.set_state(u0.reshape(s.shape))
        assert s.selftest_wait_timeout(4096) == ETIMEOUT
        assert np.array_equal(s.get_state().reshape(64, 64), u0)    # no work item ran
        s.advance(40, mode="persistent")
        assert np.array_equal(s.get_state().reshape(64, 64), ref)


def test_persistent_trace_records_every_item_and_changes_nothing(oracle_lib):
    """With a trace buffer the persistent advance records a (wait, work) cycle
    pair for every work item; the result stays the oracle's, and a buffer too
    small for an advance is refused."""
    import torch
    from paper_1602_07558_gb300.swept2d import EINVAL, SweptError
    u0 = inputs.uniform(64, 64, seed=9)
    ref = oracle_lib.heat(u0, 0.2, 40)
    NT, H = 16, 5                           # 4 x 4 tiles of 16, 40 steps = 5 half cycles
    items = NT * (1 + 3 * H)
    buf = torch.zeros(2 * items, dtype=torch.int32, device="cuda")
    with Swept2D(64, 64, op="heat", tile=16, params=(0.2,)) as s:
        s.set_trace(buf)
        s.set_state(u0.reshape(s.shape))
        s.advance(40, mode="persistent")
        assert np.array_equal(s.get_state().reshape(64, 64), ref)
        t = buf.cpu().numpy().view(np.uint32).reshape(items, 2)
        assert (t[:, 1] > 0).all()                      # every item ran and was timed
        s.set_trace(buf[:2 * (items - 1)])
        s.set_state(u0.reshape(s.shape))
        with pytest.raises(SweptError) as ei:
            s.advance(40, mode="persistent")
        assert ei.value.code == EINVAL
        s.set_trace(None)
        s.advance(40, mode="persistent")
        assert np.array_equal(s.get_state().reshape(64, 64), ref)


# ------------------------------------------------------------- CUDA graphs

@pytest.mark.parametrize("op,mode,nsteps", [
    ("heat", "swept", 40), ("heat", "naive", 13), ("heat", "swept", 37),
    ("hash", "swept", 21), ("heat_kahan", "swept", 45),
])
def test_graph_replay_gives_the_same_bits(op, mode, nsteps):
    """The first graph-mode advance is captured, the next ones replay it; an
    odd naive tail swaps the state buffers between replays, and the hash
    update keys its graphs by the starting sub-step. Three advances in a row
    must equal three plain advances bit for bit."""
    nx, ny, tile = 64, 48, 16
    rng = np.random.default_rng(5)
    dtype = {"heat": "f64", "hash": "u64", "heat_kahan": "f32"}[op]
    params = () if op == "hash" else (0.2,)
    if op == "hash":
        u0 = rng.integers(0, 2**64, size=(1, ny, nx), dtype=np.uint64)
    elif op == "heat":
        u0 = rng.random((1, ny, nx))
    else:
        u0 = np.stack([rng.random((ny, nx)), np.zeros((ny, nx))]).astype(np.float32)
    plain = run(op, u0, None, tile, mode, params, chunks=[nsteps] * 3, dtype=dtype)
    stream = torch.cuda.Stream()
    with Swept2D(nx, ny, op=op, tile=tile, params=params, dtype=dtype, stream=stream) as s:
        s.set_state(np.ascontiguousarray(u0))
        for _ in range(3):
            s.advance(nsteps, mode=mode, graph=True)
        got = s.get_state()
        assert s.query("substeps") == 3 * nsteps
    assert np.array_equal(got, plain)


# ------------------------------------------------------ full-size sampled check

def test_heat_4096_tile_32_full_grid_matches_oracle(oracle_lib):
    """The benchmark's grid and tile (4096 x 4096, n = 32): three half cycles
    plus a tail, compared with the oracle on every point."""
    u0 = inputs.smooth_field(4096, 4096, seed=1)
    ref = oracle_lib.heat(u0, 0.2, 53)
    got = run("heat", u0, 53, 32, "swept", (0.2,))[0]
    assert np.array_equal(got, ref)
    # conservation over a longer swept run of the same grid
    long = run("heat", u0, 640, 32, "swept", (0.2,))[0]
    assert abs(long.sum() - u0.sum()) <= 640 * u0.size * 4 * np.finfo(float).eps * np.abs(u0).max()


def test_euler_2048_tile_32_full_grid_matches_oracle(oracle_lib):
    """The Euler benchmark's grid and tile (2048 x 2048, n = 32), FP64: three
    half cycles (in-place levels) and a tail, every point against the oracle,
    and the persistent form the same bits."""
    nsteps = 27                        # 54 sub-steps = 3 half cycles + 6
    u0, U = _euler_u0(2048, 2048, seed=2)
    a, dt = oracle_lib.euler_setup(U, GAMMA, CFL)
    ref = oracle_lib.euler_rk2(U, GAMMA, dt, KAPPA, a, nsteps)
    got = run("euler_rk2", u0, nsteps, 32, "swept", (GAMMA, CFL, KAPPA))
    assert np.array_equal(got[:4], ref)
    assert np.array_equal(run("euler_rk2", u0, nsteps, 32, "persistent", (GAMMA, CFL, KAPPA)), got)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_euler_kahan_2048_tile_32_full_grid_matches_oracle(oracle_lib, storage):
    """The precision-form Euler benchmark's grid, tile and default launch
    shape (binary32: unstaged; bfloat16: staged), all 12 planes against the
    oracle after three half cycles and a tail."""
    nsteps = 27
    S = _euler_kahan_state(2048, 2048, storage, seed=2)
    Uf = (oracle_lib.bf16_bits_to_f32(S[:4]) if storage == "bf16" else S[:4]).astype(np.float64)
    a, dt = oracle_lib.euler_setup(Uf, GAMMA, CFL)
    ref = oracle_lib.euler_kahan(S, GAMMA, dt, KAPPA, a, nsteps, storage)
    got = run("euler_kahan", S, nsteps, 32, "swept", (GAMMA, CFL, KAPPA), dtype=storage)
    assert np.array_equal(got, ref)


def test_wave_1024_tile_32_full_grid_matches_oracle(oracle_lib):
    """The wave benchmark's grid and tile: 53 steps (three half cycles and a
    tail) against the oracle on every point."""
    u0 = inputs.wave_source(1024, 1024)
    ru, ro = oracle_lib.wave(u0[0], u0[1], 0.3 * 0.3, 53)
    got = run("wave", u0, 53, 32, "swept", (0.3,))
    assert np.array_equal(got[0], ru) and np.array_equal(got[1], ro)


def test_device_tensors_in_and_out():
    u0 = torch.rand(1, 64, 64, dtype=torch.float64, device="cuda")
    with Swept2D(64, 64, op="heat", tile=16, params=(0.2,),
                 stream=torch.cuda.current_stream()) as s:
        s.set_state(u0)
        s.advance(16)
        out = torch.empty_like(u0)
        s.get_state(out)
        host = s.get_state()
    assert np.array_equal(out.cpu().numpy(), host)
