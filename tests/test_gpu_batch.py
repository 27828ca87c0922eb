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
@pytest.mark.parametrize("mode", ["swept", "naive", "persistent"])
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
        b.set_state(states)
        for _ in range(3):
            b.advance(21, mode="persistent", graph=True)
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


def test_batch_tuning_gives_identical_bits():
    states = _states("heat_kahan", "f32", seed=3)
    outs = []
    for threads, stage in [(256, False), (128, True), (64, False)]:
        for mode in ("swept", "persistent"):
            with SweptBatch([s[0] for s in SIZES], [s[1] for s in SIZES], [s[2] for s in SIZES],
                            op="heat_kahan", params=(0.2,), dtype="f32") as b:
                b.set_tuning(threads, stage)
                b.set_state(states)
                b.advance(45, mode=mode)
                outs.append(b.get_state())
    assert all(np.array_equal(outs[0], o) for o in outs[1:])
