"""GPU parity of the batched form: every grid of an uneven batch, advanced in
shared launches, equals the oracle (and the single-grid path) bit for bit."""
import numpy as np
import pytest

from paper_1602_07558_gb300 import inputs
from paper_1602_07558_gb300.swept2d import Swept2D, SweptBatch

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

# uneven sizes, nx != ny, several tile classes, one naive-only grid, one grid
# that is a single tile
SIZES = [(32, 48, 16), (64, 64, 32), (48, 96, 16), (96, 32, 32), (16, 16, 16), (40, 24, 8),
         (64, 128, 64), (24, 24, 0)]


def _bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16) \
        .view(torch.int16).numpy().view(np.uint16)


def _states(op, dtype, seed):
    rng = np.random.default_rng(seed)
    out = []
    for nx, ny, _ in SIZES:
        if op == "hash":
            out.append(rng.integers(0, 2**64, size=(1, ny, nx), dtype=np.uint64))
        elif op == "heat":
            out.append(rng.random((1, ny, nx)))
        else:
            u = rng.random((ny, nx)).astype(np.float32)
            u = u if dtype == "f32" else _bf16(u)
            out.append(np.stack([u, np.zeros_like(u)]))
    return out


def _oracle(oracle_lib, op, dtype, s, nsteps):
    if op == "heat":
        return oracle_lib.heat(s[0], 0.2, nsteps)[None]
    if op == "hash":
        return oracle_lib.hash_op(s[0], nsteps)[None]
    u, c = oracle_lib.heat_kahan(s[0], s[1], 0.2, nsteps, storage=dtype)
    return np.stack([u, c])


@pytest.mark.parametrize("op,dtype", [("heat", "f64"), ("hash", "u64"),
                                      ("heat_kahan", "f32"), ("heat_kahan", "bf16")])
@pytest.mark.parametrize("mode", ["swept", "naive", "persistent", "persistent_one"])
def test_batch_equals_the_oracle_for_every_grid(oracle_lib, op, dtype, mode):
    nsteps = 37                           # odd tails for every class
    states = _states(op, dtype, seed=len(op) + len(mode))
    params = () if op == "hash" else (0.2,)
    with SweptBatch([s[0] for s in SIZES], [s[1] for s in SIZES], [s[2] for s in SIZES],
                    op=op, params=params, dtype=dtype) as b:
        b.set_state(states)
        b.advance(nsteps, mode=mode)
        got = b.split(b.get_state())
        assert b.query("substeps") == nsteps
    for s, g in zip(states, got):
        assert np.array_equal(g, _oracle(oracle_lib, op, dtype, s, nsteps))


@pytest.mark.parametrize("op,dtype", [("heat", "f64"), ("heat_kahan", "f32")])
def test_batch_graph_and_split_advances_match(op, dtype):
    """Three graph-replayed advances equal one plain advance of the same total,
    and each grid equals a single-grid handle with the same tile."""
    states = _states(op, dtype, seed=9)
    stream = torch.cuda.Stream()
    kw = dict(op=op, params=(0.2,), dtype=dtype)
    with SweptBatch([s[0] for s in SIZES], [s[1] for s in SIZES], [s[2] for s in SIZES],
                    stream=stream, **kw) as b:
        b.set_state(states)
        for _ in range(3):
            b.advance(21, graph=True)
        got = b.split(b.get_state())
        for mode in ("persistent", "persistent_one"):
            b.set_state(states)
            for _ in range(3):
                b.advance(21, mode=mode, graph=True)
            assert all(np.array_equal(x, y) for x, y in zip(got, b.split(b.get_state())))
    with SweptBatch([s[0] for s in SIZES], [s[1] for s in SIZES], [s[2] for s in SIZES],
                    **kw) as b:
        b.set_state(states)
        b.advance(63)
        plain = b.split(b.get_state())
    for (nx, ny, n), s, g, p in zip(SIZES, states, got, plain):
        assert np.array_equal(g, p)
        with Swept2D(nx, ny, tile=n, **kw) as h:
            h.set_state(np.ascontiguousarray(s))
            h.advance(63, mode="swept" if n else "naive")
            assert np.array_equal(g, h.get_state())


GAMMA, CFL, KAPPA = 1.4, 0.3, 0.5


# the Euler point state does not fit a 64-wide tile's level buffers
EULER_SIZES = [(nx, ny, min(n, 32)) for nx, ny, n in SIZES]


def _euler_states(dtype, seed):
    out = []
    for i, (nx, ny, _) in enumerate(EULER_SIZES):
        U = inputs.euler_pulse(nx, ny, seed + i, gamma=GAMMA)
        if dtype == "f64":
            out.append(np.concatenate([U, U]))
        else:
            U = U.astype(np.float32)
            U = U if dtype == "f32" else _bf16(U)
            out.append(np.concatenate([U, U, np.zeros_like(U)]))
    return out


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("mode", ["swept", "naive", "persistent", "persistent_one"])
def test_batch_euler_every_grid_has_its_own_time_step(oracle_lib, dtype, mode):
    """Euler grids of uneven sizes in one batch: each grid's wave speed and
    time step come from its own state and spacing (exactly the oracle's), and
    every grid equals the oracle bit for bit (FP64: U; binary32 / bfloat16:
    all 12 planes)."""
    nsteps = 13
    op = "euler_rk2" if dtype == "f64" else "euler_kahan"
    states = _euler_states(dtype, seed=40)
    S = EULER_SIZES
    with SweptBatch([s[0] for s in S], [s[1] for s in S], [s[2] for s in S],
                    op=op, params=(GAMMA, CFL, KAPPA), dtype=dtype) as b:
        b.set_state(states)
        consts = [(b.query_grid(i, "wavespeed"), b.query_grid(i, "dt")) for i in range(len(S))]
        b.advance(nsteps, mode=mode)
        got = b.split(b.get_state())
    for s, g, (a_gpu, dt_gpu) in zip(states, got, consts):
        if dtype == "f64":
            a, dt = oracle_lib.euler_setup(s[:4], GAMMA, CFL)
            ref = oracle_lib.euler_rk2(s[:4], GAMMA, dt, KAPPA, a, nsteps)
            gv = g[:4]
        else:
            Uf = (oracle_lib.bf16_bits_to_f32(s[:4]) if dtype == "bf16" else s[:4]).astype(np.float64)
            a, dt = oracle_lib.euler_setup(Uf, GAMMA, CFL)
            ref = oracle_lib.euler_kahan(s, GAMMA, dt, KAPPA, a, nsteps, dtype)
            gv = g
        assert (a_gpu, dt_gpu) == (a, dt)
        assert np.array_equal(gv, ref)


def test_batch_tuning_gives_identical_bits():
    states = _states("heat_kahan", "f32", seed=3)
    outs = []
    for threads, stage in [(256, False), (128, True), (64, False), (32, False), (32, True)]:
        for mode in ("swept", "persistent", "persistent_one"):
            with SweptBatch([s[0] for s in SIZES], [s[1] for s in SIZES], [s[2] for s in SIZES],
                            op="heat_kahan", params=(0.2,), dtype="f32") as b:
                b.set_tuning(threads, stage)
                b.set_state(states)
                b.advance(45, mode=mode)
                outs.append(b.get_state())
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


def test_one_launch_needs_the_persistent_form():
    """SWEPT2D_ONE_LAUNCH alone (without SWEPT2D_PERSISTENT) is refused."""
    from paper_1602_07558_gb300.swept2d import SweptError, lib
    states = _states("heat", "f64", seed=1)
    with SweptBatch([s[0] for s in SIZES], [s[1] for s in SIZES], [s[2] for s in SIZES],
                    op="heat", params=(0.2,), dtype="f64") as b:
        b.set_state(states)
        rc = lib().swept2d_batch_advance(b._h, 5, 0x400)
        assert rc == -1 and "PERSISTENT" in lib().swept2d_batch_last_error(b._h).decode()
