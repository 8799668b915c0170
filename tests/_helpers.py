"""Shared helpers for the tests (no method arithmetic lives here)."""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def build_c(src: str, name: str, extra=()) -> str:
    out = os.path.join(tempfile.gettempdir(), "bsfp_test_%s_%d.so" % (name, os.getpid()))
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-o", out, src, *extra])
    return out


_fenv = None


def host_f32(op: str, rz: int, a, b) -> np.ndarray:
    """Host FPU binary32 add/mul/div in RN or RZ (pin for 1/8/23)."""
    global _fenv
    if _fenv is None:
        path = build_c(os.path.join(HERE, "host_fenv.c"), "fenv",
                       ["-frounding-math", "-ffp-contract=off", "-lm"])
        L = ctypes.CDLL(path)
        L.host_f32.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_long]
        _fenv = L
    a = np.ascontiguousarray(a, dtype=np.uint32)
    b = np.ascontiguousarray(b, dtype=np.uint32)
    out = np.empty_like(a)
    _fenv.host_f32({"add": 0, "mul": 1, "div": 2}[op], rz, a.ctypes.data, b.ctypes.data, out.ctypes.data, a.size)
    return out


def fields(E, M, code):
    code = int(code)
    return (code >> (E + M)) & 1, (code >> M) & ((1 << E) - 1), code & ((1 << M) - 1)


def is_nan(E, M, code):
    s, e, f = fields(E, M, code)
    return e == (1 << E) - 1 and f != 0


def is_inf(E, M, code):
    s, e, f = fields(E, M, code)
    return e == (1 << E) - 1 and f == 0


def value(E, M, code) -> Fraction:
    """Exact value of a finite encoding of 1/E/M (IEEE-style reading)."""
    s, e, f = fields(E, M, code)
    bias = (1 << (E - 1)) - 1
    if e == 0:
        v = Fraction(f, 1 << M) * Fraction(2) ** (1 - bias)
    else:
        v = (1 + Fraction(f, 1 << M)) * Fraction(2) ** (e - bias)
    return -v if s else v


def nan_class_equal(E, M, got, want):
    """Bit equality, except that any NaN matches any NaN (for host-FPU pins)."""
    got = np.asarray(got, dtype=np.uint32)
    want = np.asarray(want, dtype=np.uint32)
    emask = ((1 << E) - 1) << M
    fmask = (1 << M) - 1
    gn = ((got & emask) == emask) & ((got & fmask) != 0)
    wn = ((want & emask) == emask) & ((want & fmask) != 0)
    return (got == want) | (gn & wn)
