"""Python binding of libswept2d.so (argument marshalling only).

Every step of the time advance runs in the library's CUDA kernels; this module
only loads the library, converts arguments and raises on error status. If the
library cannot be built or loaded it raises -- there is no CPU fallback.

The names follow the C ABI in ``include/swept2d.h``::

    s = Swept2D(nx, ny, op="heat", tile=32, params=(0.2,), stream=torch_stream)
    s.set_state(u0)               # numpy array or torch tensor, (nvars, ny, nx)
    s.advance(10_000)             # mode="swept" (default), "persistent" or "naive"
    u = s.get_state()             # numpy array (or fills a given tensor/array)
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

OK, EINVAL, ECUDA, ENOMEM, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5
OPS = {"heat": 0, "euler_rk2": 1, "increment": 2, "hash": 3, "leveltag": 4, "wide2": 5,
       "heat_kahan": 6, "wave": 7, "euler_kahan": 8}
DTYPES = {"f64": (0, np.float64), "f32": (1, np.float32), "bf16": (2, np.uint16),
          "u64": (3, np.uint64)}
# (nvars, nstages, default dtype) of each point update; bf16 states are passed
# as uint16 arrays of bfloat16 bits (or torch.bfloat16 tensors)
OP_SHAPE = {
    "heat": (1, 1, "f64"),
    "euler_rk2": (8, 2, "f64"),
    "increment": (1, 1, "f64"),
    "hash": (1, 1, "u64"),
    "leveltag": (1, 1, "f64"),
    "wide2": (5, 2, "u64"),
    "heat_kahan": (2, 1, "f32"),
    "wave": (2, 1, "f64"),
    "euler_kahan": (12, 2, "f32"),
}
MODES = {"swept": 0, "naive": 1, "persistent": 0x200,
         "persistent_one": 0x600}   # batches: one persistent launch for every tile class
GRAPH = 0x100
Q = {"dt": 0, "wavespeed": 1, "substeps": 2, "launches": 3, "state_bytes": 4,
     "panel_bytes": 5, "smem_bytes": 6, "cells": 7, "threads": 8, "stage": 9}
KERNELS = {"naive": 0, "up": 1, "bridge": 2, "octahedron": 3, "down": 4, "reduce": 5}

_lock = threading.Lock()
_lib = None


class SweptError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"swept2d error {code}: {msg}")
        self.code = code


def lib():
    """Load (building first if sources changed) libswept2d.so."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        L = ctypes.CDLL(path)
        vp, i, ll, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
        L.swept2d_create.argtypes = [ctypes.POINTER(vp), i, i, i, i, i, i,
                                     ctypes.POINTER(d), i, i, vp]
        L.swept2d_set_state.argtypes = [vp, vp, i]
        L.swept2d_advance.argtypes = [vp, ll, i]
        L.swept2d_get_state.argtypes = [vp, vp, i]
        L.swept2d_destroy.argtypes = [vp]
        L.swept2d_last_error.argtypes = [vp]
        L.swept2d_last_error.restype = ctypes.c_char_p
        L.swept2d_query.argtypes = [vp, i, ctypes.POINTER(d)]
        L.swept2d_set_timing.argtypes = [vp, i]
        L.swept2d_set_tuning.argtypes = [vp, i, i]
        L.swept2d_kernel_stats.argtypes = [vp, i, ctypes.POINTER(ll), ctypes.POINTER(d)]
        L.swept2d_measure_fp64_rate.argtypes = [vp, ctypes.POINTER(d)]
        L.swept2d_measure_peaks.argtypes = [vp, ctypes.POINTER(d), i]
        L.swept2d_selftest_wait_timeout.argtypes = [vp, ll]
        L.swept2d_set_trace.argtypes = [vp, vp, ll]
        for name in ("swept2d_create", "swept2d_set_state", "swept2d_advance",
                     "swept2d_get_state", "swept2d_destroy", "swept2d_query",
                     "swept2d_set_timing", "swept2d_kernel_stats", "swept2d_measure_fp64_rate",
                     "swept2d_measure_peaks", "swept2d_set_tuning", "swept2d_set_trace", "swept2d_selftest_wait_timeout"):
            getattr(L, name).restype = i
        _lib = L
        return L


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)          # torch.cuda.Stream / ExternalStream


def _buffer(x, dtype, nbytes):
    """(pointer, is_device, keepalive) of a numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous or x.dtype.itemsize != np.dtype(dtype).itemsize:
            raise ValueError("array must be C-contiguous with the op's element size")
        if x.nbytes != nbytes:
            raise ValueError(f"array has {x.nbytes} bytes, the state has {nbytes}")
        return x.ctypes.data, 0, x
    try:
        import torch
    except ImportError as e:  # pragma: no cover
        raise TypeError("expected a numpy array") from e
    if not isinstance(x, torch.Tensor):
        raise TypeError("expected a numpy array or a torch tensor")
    if not x.is_contiguous() or x.element_size() != np.dtype(dtype).itemsize:
        raise ValueError("tensor must be contiguous with the op's element size")
    if x.numel() * x.element_size() != nbytes:
        raise ValueError("tensor size does not match the state")
    return x.data_ptr(), 1 if x.is_cuda else 0, x


def measure_fp64_rate(stream=None) -> float:
    """FP64 fused multiply-adds per second measured on the current device."""
    out = ctypes.c_double()
    rc = lib().swept2d_measure_fp64_rate(_stream_handle(stream), ctypes.byref(out))
    if rc != OK:
        raise SweptError(rc, "measure_fp64_rate failed")
    return out.value


def measure_peaks(stream=None) -> dict:
    """Measured rates of the current device: FP64 and FP32 lane-operations per
    second, shared-memory wavefronts per second, and FP64 warp instructions per
    second with 32 and with 1 active lane (swept2d_measure_peaks)."""
    out = (ctypes.c_double * 5)()
    rc = lib().swept2d_measure_peaks(_stream_handle(stream), out, 5)
    if rc != OK:
        raise SweptError(rc, "measure_peaks failed")
    return {"fp64_ops_per_s": out[0], "fp32_ops_per_s": out[1],
            "smem_wavefronts_per_s": out[2], "fp64_warp_instr_per_s_32_lanes": out[3],
            "fp64_warp_instr_per_s_1_lane": out[4]}


class Swept2D:
    """One periodic nx x ny grid advanced by the swept rule (or the naive path)."""

    def __init__(self, nx, ny, op="heat", tile=0, params=(), stream=None, dtype=None):
        if op not in OPS:
            raise ValueError(f"unknown op {op!r}; one of {sorted(OPS)}")
        self.nx, self.ny, self.op, self.tile = int(nx), int(ny), op, int(tile)
        self.nvars, self.nstages, default = OP_SHAPE[op]
        self.dtype = dtype or default
        if self.dtype not in DTYPES:
            raise ValueError(f"unknown dtype {dtype!r}; one of {sorted(DTYPES)}")
        self._dtype_code, self.np_dtype = DTYPES[self.dtype]
        self.params = tuple(float(p) for p in params)
        self._stream = _stream_handle(stream)
        self._h = ctypes.c_void_p()
        arr = (ctypes.c_double * max(1, len(self.params)))(*self.params)
        L = lib()
        rc = L.swept2d_create(ctypes.byref(self._h), self.nx, self.ny, self.nvars, self.nstages,
                              self.tile, OPS[op], arr, len(self.params), self._dtype_code,
                              self._stream)
        if rc != OK:
            raise SweptError(rc, L.swept2d_last_error(None).decode())
        self.state_bytes = int(self.query("state_bytes"))

    # -- helpers
    def _check(self, rc):
        if rc != OK:
            raise SweptError(rc, lib().swept2d_last_error(self._h).decode())

    @property
    def shape(self):
        return (self.nvars, self.ny, self.nx)

    # -- the C ABI, one method per entry point
    def set_state(self, state):
        ptr, dev, keep = _buffer(state, self.np_dtype, self.state_bytes)
        self._check(lib().swept2d_set_state(self._h, ptr, dev))
        del keep

    def advance(self, nsteps, mode="swept", graph=False):
        """``graph=True`` replays a captured CUDA graph of the launch sequence
        (needs a handle created with a non-default stream)."""
        m = MODES[mode] | (GRAPH if graph else 0)
        self._check(lib().swept2d_advance(self._h, int(nsteps), m))

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=self.np_dtype)
        ptr, dev, keep = _buffer(out, self.np_dtype, self.state_bytes)
        self._check(lib().swept2d_get_state(self._h, ptr, dev))
        return out

    def query(self, what):
        v = ctypes.c_double()
        self._check(lib().swept2d_query(self._h, Q[what], ctypes.byref(v)))
        return v.value

    def set_tuning(self, threads=256, stage=False):
        """Launch shape of the swept kernels (same results for every setting)."""
        self._check(lib().swept2d_set_tuning(self._h, int(threads), 1 if stage else 0))

    def set_trace(self, buf=None):
        """Record the persistent form's per-item (wait, work) SM cycles into a
        contiguous device tensor of 2 x items 32-bit words (None: stop)."""
        if buf is None:
            self._check(lib().swept2d_set_trace(self._h, None, 0))
            self._trace = None
            return
        if not buf.is_cuda or not buf.is_contiguous() or buf.element_size() != 4:
            raise ValueError("trace buffer: a contiguous CUDA tensor of 32-bit words")
        self._trace = buf                       # keep the memory alive while recording
        self._check(lib().swept2d_set_trace(self._h, buf.data_ptr(), buf.numel() // 2))

    def set_timing(self, on=True):
        self._check(lib().swept2d_set_timing(self._h, 1 if on else 0))

    def kernel_stats(self, kind):
        n, ms = ctypes.c_longlong(), ctypes.c_double()
        self._check(lib().swept2d_kernel_stats(self._h, KERNELS[kind], ctypes.byref(n),
                                               ctypes.byref(ms)))
        return n.value, ms.value

    def selftest_wait_timeout(self, spin_limit=4096):
        """Run the persistent kernel with waits that can never be satisfied;
        returns the status code (ETIMEOUT when the bounded wait gave up)."""
        return lib().swept2d_selftest_wait_timeout(self._h, int(spin_limit))

    def close(self):
        if self._h:
            lib().swept2d_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def heat_advance_static(u_in, u_out, nx, ny, tile, r, nsteps, stream=None):
    """swept2d_heat_advance_static: the allocation-free swept heat advance.

    For callers that may not allocate device memory while they advance (their
    host application owns all device memory through a fixed pool, or they
    cannot afford cudaMalloc's implicit synchronisation). ``u_in`` and
    ``u_out`` are device buffers (torch CUDA tensors or raw pointers) of
    nx*ny FP64 values; the only scratch is the library's static device array
    (``SWEPT2D_STATIC_SCRATCH_BYTES``), shared by every call on a device, so
    calls must not overlap on the GPU. Returns nothing; raises SweptError.
    """
    L = lib()
    fn = L.swept2d_heat_advance_static
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                   ctypes.c_double, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_char_p,
                   ctypes.c_int]
    fn.restype = ctypes.c_int
    ptr = lambda x: x if isinstance(x, int) else x.data_ptr()
    err = ctypes.create_string_buffer(256)
    rc = fn(ptr(u_in), ptr(u_out), int(nx), int(ny), int(tile), float(r), int(nsteps),
            _stream_handle(stream), err, 256)
    if rc != OK:
        raise SweptError(rc, err.value.decode())


class SweptBatch:
    """Many independent periodic grids of uneven sizes advanced together
    (swept2d_batch_*). ``tiles[i]`` is grid i's tile side (0: naive only).
    States are numpy arrays or torch tensors holding the grids' states
    concatenated in grid order; ``split`` cuts such a buffer into per-grid
    (nvars, ny, nx) views."""

    def __init__(self, nx, ny, tiles, op="heat", params=(), stream=None, dtype=None):
        if op not in OPS:
            raise ValueError(f"unknown op {op!r}")
        self.nx = [int(v) for v in nx]
        self.ny = [int(v) for v in ny]
        self.tiles = [int(v) for v in tiles]
        if not (len(self.nx) == len(self.ny) == len(self.tiles)):
            raise ValueError("nx, ny and tiles differ in length")
        self.op = op
        self.nvars, self.nstages, default = OP_SHAPE[op]
        self.dtype = dtype or default
        self._dtype_code, self.np_dtype = DTYPES[self.dtype]
        self.params = tuple(float(p) for p in params)
        self._stream = _stream_handle(stream)
        L = lib()
        self._fns(L)
        n = len(self.nx)
        arr = lambda v: (ctypes.c_int * n)(*v)
        prm = (ctypes.c_double * max(1, len(self.params)))(*self.params)
        self._h = ctypes.c_void_p()
        rc = L.swept2d_batch_create(ctypes.byref(self._h), n, arr(self.nx), arr(self.ny),
                                    arr(self.tiles), OPS[op], prm, len(self.params),
                                    self._dtype_code, self._stream)
        if rc != OK:
            raise SweptError(rc, L.swept2d_batch_last_error(None).decode())
        self.sizes = [self.nvars * a * b for a, b in zip(self.nx, self.ny)]
        self.total = sum(self.sizes)

    @staticmethod
    def _fns(L):
        if getattr(L, "_batch_ready", False):
            return
        vp, i, ll, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
        ip = ctypes.POINTER(ctypes.c_int)
        L.swept2d_batch_create.argtypes = [ctypes.POINTER(vp), i, ip, ip, ip, i,
                                           ctypes.POINTER(d), i, i, vp]
        L.swept2d_batch_set_state.argtypes = [vp, vp, i]
        L.swept2d_batch_advance.argtypes = [vp, ll, i]
        L.swept2d_batch_get_state.argtypes = [vp, vp, i]
        L.swept2d_batch_set_tuning.argtypes = [vp, i, i]
        L.swept2d_batch_set_class_tuning.argtypes = [vp, i, i, i]
        L.swept2d_batch_destroy.argtypes = [vp]
        L.swept2d_batch_last_error.argtypes = [vp]
        L.swept2d_batch_last_error.restype = ctypes.c_char_p
        L.swept2d_batch_query.argtypes = [vp, i, ctypes.POINTER(d)]
        L.swept2d_batch_query_grid.argtypes = [vp, i, i, ctypes.POINTER(d)]
        for name in ("swept2d_batch_create", "swept2d_batch_set_state", "swept2d_batch_advance",
                     "swept2d_batch_get_state", "swept2d_batch_set_tuning",
                     "swept2d_batch_set_class_tuning",
                     "swept2d_batch_destroy", "swept2d_batch_query", "swept2d_batch_query_grid"):
            getattr(L, name).restype = i
        L._batch_ready = True

    def _check(self, rc):
        if rc != OK:
            raise SweptError(rc, lib().swept2d_batch_last_error(self._h).decode())

    def split(self, flat):
        out, off = [], 0
        for a, b, n in zip(self.nx, self.ny, self.sizes):
            out.append(flat[off:off + n].reshape(self.nvars, b, a))
            off += n
        return out

    def pack(self, states):
        return np.concatenate([np.ascontiguousarray(s, dtype=self.np_dtype).reshape(-1)
                               for s in states])

    def set_state(self, state):
        if isinstance(state, (list, tuple)):
            state = self.pack(state)
        nbytes = self.total * np.dtype(self.np_dtype).itemsize
        ptr, dev, keep = _buffer(state, self.np_dtype, nbytes)
        self._check(lib().swept2d_batch_set_state(self._h, ptr, dev))
        del keep

    def advance(self, nsteps, mode="swept", graph=False):
        m = MODES[mode] | (GRAPH if graph else 0)
        self._check(lib().swept2d_batch_advance(self._h, int(nsteps), m))

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.total, dtype=self.np_dtype)
        nbytes = self.total * np.dtype(self.np_dtype).itemsize
        ptr, dev, keep = _buffer(out, self.np_dtype, nbytes)
        self._check(lib().swept2d_batch_get_state(self._h, ptr, dev))
        return out

    def set_tuning(self, threads=256, stage=False, tile=None):
        """Launch shape of every class, or of the class with tile side ``tile``."""
        if tile is None:
            self._check(lib().swept2d_batch_set_tuning(self._h, int(threads), 1 if stage else 0))
        else:
            self._check(lib().swept2d_batch_set_class_tuning(self._h, int(tile), int(threads),
                                                             1 if stage else 0))

    def query(self, what):
        v = ctypes.c_double()
        self._check(lib().swept2d_batch_query(self._h, Q[what], ctypes.byref(v)))
        return v.value

    def query_grid(self, grid, what):
        """Per-grid "dt", "wavespeed" (Euler updates) or "cells"."""
        v = ctypes.c_double()
        self._check(lib().swept2d_batch_query_grid(self._h, int(grid), Q[what], ctypes.byref(v)))
        return v.value

    def close(self):
        if self._h:
            lib().swept2d_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
