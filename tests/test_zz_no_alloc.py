"""GPU test of swept2d_heat_advance_static, the allocation-free entry point.

Some callers cannot allocate device memory where they advance a grid (their
host application owns all device memory through a fixed pool, or they cannot
afford cudaMalloc's implicit synchronisation). This entry point serves them
with a static device scratch array; here it is called through the C ABI and
must give exactly what the handle-based swept path gives (the heat tests'
bar: bitwise), on two different calls in a row that share that array.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1602_07558_gb300 import inputs, swept2d

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def call_static(u_in, u_out, nx, ny, tile, r, nsteps, stream):
    fn = swept2d.lib().swept2d_heat_advance_static
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                   ctypes.c_double, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_char_p,
                   ctypes.c_int]
    fn.restype = ctypes.c_int
    err = ctypes.create_string_buffer(256)
    rc = fn(u_in.data_ptr(), u_out.data_ptr(), nx, ny, tile, r, nsteps,
            stream.cuda_stream, err, 256)
    return rc, err.value.decode()


def handle_path(u0, tile, r, nsteps):
    ny, nx = u0.shape
    with swept2d.Swept2D(nx, ny, op="heat", tile=tile, params=(r,)) as s:
        s.set_state(u0[None])
        s.advance(nsteps, mode="swept")
        return s.get_state()[0]


def test_static_entry_point_equals_handle_path_on_two_calls_in_a_row():
    stream = torch.cuda.Stream()
    # second call: other size and tile, a naive tail (37 = 2*16 + 5); the
    # scratch still holds the first call's panels when it starts
    cases = [(64, 64, 16, 40, 0), (96, 64, 32, 37, 1)]
    for nx, ny, tile, nsteps, seed in cases:
        u0 = inputs.uniform(nx, ny, seed=seed)
        d_in = torch.from_numpy(u0).to("cuda")
        d_out = torch.full_like(d_in, float("nan"))
        torch.cuda.synchronize()
        rc, msg = call_static(d_in, d_out, nx, ny, tile, 0.2, nsteps, stream)
        assert rc == swept2d.OK, msg
        stream.synchronize()
        ref = handle_path(u0, tile, 0.2, nsteps)
        assert np.array_equal(d_out.cpu().numpy(), ref)
        assert np.array_equal(d_in.cpu().numpy(), u0)          # input left as it was


@pytest.mark.parametrize("nx,ny,tile,nsteps,seed", [
    (64, 64, 16, 5, 2),     # fewer steps than a half cycle, odd naive count
    (64, 64, 16, 6, 3),     # fewer steps than a half cycle, even naive count
    (64, 64, 16, 0, 4),     # no step: a plain copy
    (48, 32, 16, 8, 5),     # exactly one half cycle, no tail
])
def test_static_entry_point_short_advances_equal_handle_path(nx, ny, tile, nsteps, seed):
    """Step counts below one half cycle run only the naive kernel, ping-ponging
    through the scratch so that the last sub-step lands in u_out; zero steps
    copy u_in. Each must equal the handle path bit for bit."""
    stream = torch.cuda.Stream()
    u0 = inputs.uniform(nx, ny, seed=seed)
    d_in = torch.from_numpy(u0).to("cuda")
    d_out = torch.full_like(d_in, float("nan"))
    torch.cuda.synchronize()
    rc, msg = call_static(d_in, d_out, nx, ny, tile, 0.2, nsteps, stream)
    assert rc == swept2d.OK, msg
    stream.synchronize()
    assert np.array_equal(d_out.cpu().numpy(), handle_path(u0, tile, 0.2, nsteps))
    assert np.array_equal(d_in.cpu().numpy(), u0)


def test_static_entry_point_rejects_grids_beyond_its_scratch():
    """4096 x 4096 with tile 32 needs about 570 MB of panels, far above the
    static scratch: the call must refuse before touching the device."""
    stream = torch.cuda.Stream()
    d_in = torch.zeros(4096 * 4096, dtype=torch.float64, device="cuda")
    d_out = torch.zeros_like(d_in)
    torch.cuda.synchronize()
    rc, msg = call_static(d_in, d_out, 4096, 4096, 32, 0.2, 100, stream)
    assert rc == swept2d.EINVAL
    assert "scratch" in msg
    assert torch.count_nonzero(d_out).item() == 0
