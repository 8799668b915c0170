"""CPU oracle for bitslice custom-precision floating point.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never imports, links or calls it, and it shares no
code with the CUDA library.

Two independent oracles live here:

* ``bsfp_oracle.c`` (plain C, built with gcc into ``liboracle.so``): decode ->
  exact integer arithmetic (320-bit integers) -> one rounding (RN-even or RZ) ->
  encode, plus a bit-by-bit pack/unpack.  Used for parity of the CUDA path.
* ``bruteforce.py`` (pure Python, ``fractions.Fraction``): rounds the exact
  rational result by searching the sorted list of every representable value of
  a small format.  Used only to pin the C oracle.

Rounding modes follow the paper's Sec. 4 (round toward zero, round to nearest
ties to even).  Formats are ``1/E/M``: one sign bit, ``E`` exponent bits,
``M`` fraction bits (Sec. 5.2 uses 1/4/3, 1/5/10 and 1/8/23).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bsfp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OPS = {"add": 0, "sub": 1, "mul": 2, "fma2": 3, "div": 4}
RN, RZ, RN_FTZ, RZ_FTZ = 0, 1, 2, 3   # rounding modes; bit 1 = flush to zero


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP over elements)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u32, i32, i64 = ctypes.c_uint32, ctypes.c_int, ctypes.c_int64
            p = ctypes.c_void_p
            for name in ("oracle_add1", "oracle_sub1", "oracle_mul1", "oracle_div1"):
                fn = getattr(L, name)
                fn.argtypes = [i32, i32, i32, u32, u32]
                fn.restype = u32
            L.oracle_fma2_1.argtypes = [i32, i32, i32, u32, u32, u32]
            L.oracle_fma2_1.restype = u32
            L.oracle_binop.argtypes = [i32, i32, i32, i32, p, p, p, p, i64]
            L.oracle_binop.restype = None
            for name in ("oracle_from_f32", "oracle_to_f32"):
                fn = getattr(L, name)
                fn.argtypes = [i32, i32, i32, p, p, i64]
                fn.restype = None
            L.oracle_int_binop.argtypes = [i32, i32, p, p, p, i64]
            L.oracle_int_binop.restype = None
            L.oracle_plane_stride.argtypes = [i64]
            L.oracle_plane_stride.restype = i64
            L.oracle_pack.argtypes = [i32, p, i64, p, i64]
            L.oracle_pack.restype = None
            L.oracle_unpack.argtypes = [i32, p, i64, i64, p]
            L.oracle_unpack.restype = None
            L.oracle_num_threads.argtypes = []
            L.oracle_num_threads.restype = i32
            L.oracle_set_threads.argtypes = [i32]
            L.oracle_set_threads.restype = None
            _lib = L
    return _lib


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def binop(op: str, E: int, M: int, rnd: int, a, b, c=None) -> np.ndarray:
    """Element-wise ``op`` in {add, sub, mul, fma2, div} on B-bit patterns (uint32)."""
    a, b = _u32(a), _u32(b)
    assert a.shape == b.shape
    c = _u32(c) if c is not None else np.zeros_like(a)
    out = np.empty_like(a)
    lib().oracle_binop(OPS[op], E, M, rnd, _ptr(a), _ptr(b), _ptr(c), _ptr(out), a.size)
    return out


def add(E, M, rnd, a, b):
    return binop("add", E, M, rnd, a, b)


def sub(E, M, rnd, a, b):
    return binop("sub", E, M, rnd, a, b)


def mul(E, M, rnd, a, b):
    return binop("mul", E, M, rnd, a, b)


def div(E, M, rnd, a, b):
    return binop("div", E, M, rnd, a, b)


def fma2(E, M, rnd, a, b, c):
    return binop("fma2", E, M, rnd, a, b, c)


def from_f32(E: int, M: int, rnd: int, x) -> np.ndarray:
    """binary32 bit patterns -> 1/E/M encodings, one rounding in mode rnd."""
    x = _u32(x)
    out = np.empty_like(x)
    lib().oracle_from_f32(E, M, rnd, _ptr(x), _ptr(out), x.size)
    return out


def to_f32(E: int, M: int, rnd: int, x) -> np.ndarray:
    """1/E/M encodings -> binary32 bit patterns (exact; NaN canonical)."""
    x = _u32(x)
    out = np.empty_like(x)
    lib().oracle_to_f32(E, M, rnd, _ptr(x), _ptr(out), x.size)
    return out


INT_OPS = {"add": 0, "sub": 1, "mul": 2}


def int_binop(op: str, w: int, a, b) -> np.ndarray:
    """w-bit unsigned integer vectors (Sec. 3): op in {add, sub, mul}, the low
    w bits of the exact result."""
    a, b = _u32(a), _u32(b)
    out = np.empty_like(a)
    lib().oracle_int_binop(INT_OPS[op], w, _ptr(a), _ptr(b), _ptr(out), a.size)
    return out


def plane_stride(n: int) -> int:
    return int(lib().oracle_plane_stride(n))


def pack(B: int, x) -> np.ndarray:
    """Standard array of B-bit patterns -> (B, S) uint32 bitslice planes."""
    x = _u32(x)
    n = x.size
    S = plane_stride(n)
    planes = np.empty((B, S), dtype=np.uint32)
    lib().oracle_pack(B, _ptr(x), n, _ptr(planes), S)
    return planes


def unpack(B: int, planes, n: int) -> np.ndarray:
    planes = _u32(planes)
    S = planes.shape[-1]
    out = np.empty(n, dtype=np.uint32)
    lib().oracle_unpack(B, _ptr(planes), S, n, _ptr(out))
    return out


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_threads(k: int) -> None:
    """Threads of the following oracle calls (k > 0)."""
    lib().oracle_set_threads(int(k))
