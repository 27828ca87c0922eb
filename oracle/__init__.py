"""Plain CPU oracle for the swept-rule hot path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. The product
path (``paper_1602_07558_gb300``) never imports it, and this package imports
nothing from the product path.

Two parts:

* ``swept2d_oracle.c`` -- the plain step-by-step definition (FP64, OpenMP over
  rows), compiled here with gcc into ``_build/liboracle.so`` and called through
  ctypes. This is what every GPU parity test compares against: the swept rule
  reaches exactly the values of plain explicit time marching (Section 4, first
  paragraph; abstract).
* ``swept_sim.py`` -- a slow pure-Python walk through the paper's components
  (Algorithms 1, 2, 3, 5 glued by Algorithm 4), used only to pin the geometric
  claims of Section 3 (panel sizes, exchange counts, exact partition) on tiny
  grids. It is never compared with the GPU directly.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "swept2d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, -fopenmp, -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d, i, ll, p = ctypes.c_double, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p
        lib.oracle_num_threads.restype = i
        lib.oracle_mix64.argtypes = [ctypes.c_uint64]
        lib.oracle_mix64.restype = ctypes.c_uint64
        lib.oracle_heat.argtypes = [i, i, d, ll, p]
        lib.oracle_increment.argtypes = [i, i, ll, p]
        lib.oracle_hash.argtypes = [i, i, ll, ll, p]
        lib.oracle_leveltag.argtypes = [i, i, ll, p]
        lib.oracle_wide2.argtypes = [i, i, ll, p]
        lib.oracle_euler_wavespeed.argtypes = [i, i, d, p]
        lib.oracle_euler_wavespeed.restype = d
        lib.oracle_euler_setup.argtypes = [i, i, d, d, d, d, p,
                                           ctypes.POINTER(d), ctypes.POINTER(d)]
        lib.oracle_euler_rk2.argtypes = [i, i, d, d, d, d, d, d, ll, p]
        lib.oracle_heat_kahan_f32.argtypes = [i, i, d, ll, p, p]
        lib.oracle_wave.argtypes = [i, i, d, ll, p, p]
        lib.oracle_heat_kahan_bf16.argtypes = [i, i, d, ll, p, p]
        lib.oracle_euler_kahan.argtypes = [i, i, i, d, d, d, d, d, d, ll, p]
        lib.oracle_f32_to_bf16.argtypes = [ctypes.c_float]
        lib.oracle_f32_to_bf16.restype = ctypes.c_uint16
        lib.oracle_bf16_to_f32.argtypes = [ctypes.c_uint16]
        lib.oracle_bf16_to_f32.restype = ctypes.c_float
        for name in ("oracle_heat", "oracle_increment", "oracle_hash", "oracle_leveltag",
                     "oracle_wide2", "oracle_euler_setup", "oracle_euler_rk2",
                     "oracle_heat_kahan_f32", "oracle_heat_kahan_bf16", "oracle_wave"):
            getattr(lib, name).restype = i
        _lib = lib
        return lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(n: int) -> None:
    """OpenMP threads of the following oracle calls (results do not change)."""
    L = _load()
    L.oracle_set_threads.argtypes = [ctypes.c_int]
    L.oracle_set_threads(int(n))


def _grid(u, dtype):
    a = np.ascontiguousarray(np.array(u, dtype=dtype, copy=True))
    if a.ndim != 2:
        raise ValueError("expected a (ny, nx) array")
    return a


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def heat(u0, r: float, nsteps: int) -> np.ndarray:
    """Forward-Euler 5-point heat equation, ``nsteps`` steps; returns a new array."""
    u = _grid(u0, np.float64)
    ny, nx = u.shape
    _check(_load().oracle_heat(nx, ny, float(r), int(nsteps), u.ctypes.data), "heat")
    return u


def increment(u0, nsteps: int) -> np.ndarray:
    u = _grid(u0, np.float64)
    ny, nx = u.shape
    _check(_load().oracle_increment(nx, ny, int(nsteps), u.ctypes.data), "increment")
    return u


def mix64(z: int) -> int:
    """The SplitMix64 output function used by the hash update."""
    return int(_load().oracle_mix64(ctypes.c_uint64(int(z) & 0xFFFFFFFFFFFFFFFF)))


def hash_op(u0, nsub: int, substep0: int = 0) -> np.ndarray:
    """``nsub`` sub-steps of the 9-neighbour hash update on uint64 words."""
    a = np.ascontiguousarray(np.asarray(u0))
    if a.dtype.itemsize != 8:
        raise ValueError("hash words are 64-bit")
    u = _grid(a.view(np.uint64), np.uint64)
    ny, nx = u.shape
    _check(_load().oracle_hash(nx, ny, int(substep0), int(nsub), u.ctypes.data), "hash")
    return u


def leveltag(u0, nsub: int) -> np.ndarray:
    u = _grid(u0, np.float64)
    ny, nx = u.shape
    _check(_load().oracle_leveltag(nx, ny, int(nsub), u.ctypes.data), "leveltag")
    return u


def wide2(u0, nsteps: int) -> np.ndarray:
    """Eq. (complex_step) evaluated directly (radius 2) modulo 2^64."""
    u = _grid(u0, np.uint64)
    ny, nx = u.shape
    _check(_load().oracle_wide2(nx, ny, int(nsteps), u.ctypes.data), "wide2")
    return u


def euler_setup(U0, gamma: float, cfl: float, lx: float = 1.0, ly: float = 1.0):
    """Returns (a, dt): max wave speed of ``U0`` (4, ny, nx) and the fixed CFL step."""
    U = np.ascontiguousarray(np.asarray(U0, dtype=np.float64))
    _, ny, nx = U.shape
    a, dt = ctypes.c_double(), ctypes.c_double()
    _check(_load().oracle_euler_setup(nx, ny, float(gamma), float(cfl), float(lx), float(ly),
                                      U.ctypes.data, ctypes.byref(a), ctypes.byref(dt)),
           "euler_setup")
    return a.value, dt.value


def euler_rk2(U0, gamma: float, dt: float, kappa: float, a: float, nsteps: int,
              lx: float = 1.0, ly: float = 1.0) -> np.ndarray:
    """``nsteps`` midpoint-RK2 steps of the Euler system; ``U0`` is (4, ny, nx)."""
    U = np.ascontiguousarray(np.array(U0, dtype=np.float64, copy=True))
    if U.ndim != 3 or U.shape[0] != 4:
        raise ValueError("expected a (4, ny, nx) array")
    _, ny, nx = U.shape
    _check(_load().oracle_euler_rk2(nx, ny, float(gamma), float(dt), float(lx), float(ly),
                                    float(kappa), float(a), int(nsteps), U.ctypes.data),
           "euler_rk2")
    return U


def f32_to_bf16(x: float) -> int:
    """binary32 -> bfloat16 bits, round to nearest even."""
    return int(_load().oracle_f32_to_bf16(ctypes.c_float(x)))


def bf16_to_f32(h: int) -> float:
    return float(_load().oracle_bf16_to_f32(ctypes.c_uint16(h)))


def heat_kahan(u0, c0, r: float, nsteps: int, storage: str = "f32"):
    """Heat in binary32 arithmetic with Kahan-compensated time accumulation.
    ``storage`` "f32": u0, c0 float32 arrays; "bf16": uint16 arrays of bfloat16
    bits. Returns new (u, c) arrays of the same type."""
    dt = np.float32 if storage == "f32" else np.uint16
    u = _grid(u0, dt)
    c = _grid(c0, dt)
    if u.shape != c.shape:
        raise ValueError("u and c differ in shape")
    ny, nx = u.shape
    fn = _load().oracle_heat_kahan_f32 if storage == "f32" else _load().oracle_heat_kahan_bf16
    _check(fn(nx, ny, float(r), int(nsteps), u.ctypes.data, c.ctypes.data), "heat_kahan")
    return u, c


def bf16_bits_to_f32(bits) -> np.ndarray:
    """bfloat16 bits (uint16) -> float32 values (exact)."""
    return (np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def f32_to_bf16_bits(x) -> np.ndarray:
    """float32 values that bfloat16 represents exactly -> their bits."""
    w = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    if np.any(w & 0xFFFF):
        raise ValueError("value not representable in bfloat16")
    return (w >> 16).astype(np.uint16)


def euler_kahan(S0, gamma: float, dt: float, kappa: float, a: float, nsteps: int,
                storage: str = "f32", lx: float = 1.0, ly: float = 1.0) -> np.ndarray:
    """``nsteps`` compensated binary32 midpoint-RK2 steps of the Euler system on
    the 12-plane state (U, U*, C), shape (12, ny, nx): float32 values for
    ``storage`` "f32", uint16 bfloat16 bits for "bf16". Returns the same type."""
    if storage not in ("f32", "bf16"):
        raise ValueError("storage is 'f32' or 'bf16'")
    S0 = np.asarray(S0)
    if S0.ndim != 3 or S0.shape[0] != 12:
        raise ValueError("expected a (12, ny, nx) array")
    S = np.ascontiguousarray(bf16_bits_to_f32(S0) if storage == "bf16"
                             else np.array(S0, dtype=np.float32, copy=True))
    _, ny, nx = S.shape
    _check(_load().oracle_euler_kahan(nx, ny, 1 if storage == "bf16" else 0, float(gamma),
                                      float(dt), float(lx), float(ly), float(kappa), float(a),
                                      int(nsteps), S.ctypes.data), "euler_kahan")
    return f32_to_bf16_bits(S) if storage == "bf16" else S


def wave(u0, uold0, C2: float, nsteps: int):
    """Leapfrog wave equation with squared Courant number C2; returns (u^n, u^{n-1})."""
    u = _grid(u0, np.float64)
    uo = _grid(uold0, np.float64)
    ny, nx = u.shape
    _check(_load().oracle_wave(nx, ny, float(C2), int(nsteps), u.ctypes.data, uo.ctypes.data),
           "wave")
    return u, uo
