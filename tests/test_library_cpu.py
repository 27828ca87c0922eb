"""Host-side checks of the C-ABI library that need no GPU: it builds for
sm_103a, loads, exports every entry point declared in include/swept2d.h, and
rejects bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1602_07558_gb300 import build, swept2d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(swept2d_\w+)\s*\(", text)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert "swept2d_create" in names and "swept2d_advance" in names
    for name in names:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("kwargs,needle", [
    (dict(nx=64, ny=64, op="heat", tile=6, params=(0.2,)), "tile"),     # 6 does not divide 64
    (dict(nx=64, ny=64, op="heat", tile=5, params=(0.2,)), "tile"),     # odd
    (dict(nx=64, ny=64, op="heat", tile=2, params=(0.2,)), "tile"),     # < 4
    (dict(nx=64, ny=48, op="heat", tile=32, params=(0.2,)), "tile"),    # 32 does not divide 48
    (dict(nx=64, ny=64, op="heat", tile=16, params=()), "params"),      # heat needs r
    (dict(nx=64, ny=64, op="euler_rk2", tile=16, params=(1.4, 0.3)), "euler"),
    (dict(nx=0, ny=64, op="heat", tile=0, params=(0.2,)), "nx"),
])
def test_create_rejects_bad_arguments(kwargs, needle):
    with pytest.raises(swept2d.SweptError) as ei:
        swept2d.Swept2D(**kwargs)
    assert ei.value.code == swept2d.EINVAL
    assert needle in str(ei.value)


def test_create_rejects_op_shape_mismatch():
    L = swept2d.lib()
    h = ctypes.c_void_p()
    r = (ctypes.c_double * 1)(0.2)
    # heat with 2 variables
    assert L.swept2d_create(ctypes.byref(h), 64, 64, 2, 1, 16, 0, r, 1, 0, None) == swept2d.EINVAL
    assert not h.value
    assert b"nvars" in L.swept2d_last_error(None)
    # hash stored as F64
    assert L.swept2d_create(ctypes.byref(h), 64, 64, 1, 1, 16, 3, r, 0, 0, None) == swept2d.EINVAL
    # unknown op
    assert L.swept2d_create(ctypes.byref(h), 64, 64, 1, 1, 16, 99, r, 0, 0, None) == swept2d.EINVAL


def test_null_handles_are_rejected_without_a_device():
    L = swept2d.lib()
    assert L.swept2d_advance(None, 1, 0) == swept2d.EINVAL
    assert L.swept2d_set_state(None, None, 0) == swept2d.EINVAL
    assert L.swept2d_get_state(None, None, 0) == swept2d.EINVAL
    assert L.swept2d_destroy(None) == swept2d.OK
    out = ctypes.c_double()
    assert L.swept2d_query(None, 0, ctypes.byref(out)) == swept2d.EINVAL


@pytest.mark.parametrize("tiles,needle", [
    ([16, 10], "tile 10"),        # 10 does not divide 48
    ([16, 5], "tile 5"),
])
def test_batch_create_rejects_bad_tiles(tiles, needle):
    with pytest.raises(swept2d.SweptError) as ei:
        swept2d.SweptBatch([32, 48], [32, 48], tiles, op="heat", params=(0.2,))
    assert ei.value.code == swept2d.EINVAL and needle in str(ei.value)


def test_batch_create_rejects_unsupported_ops():
    with pytest.raises(swept2d.SweptError) as ei:
        swept2d.SweptBatch([32], [32], [16], op="wave", params=(0.3,))
    assert "not supported" in str(ei.value)
    with pytest.raises(swept2d.SweptError) as ei:
        swept2d.SweptBatch([32], [32], [16], op="euler_kahan", params=(1.4, 0.3), dtype="f32")
    assert "euler needs params" in str(ei.value)
