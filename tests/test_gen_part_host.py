"""The netlists printed for the formats outside the tuned set -- add and mul
(RN, RZ) into each part's header, and division into each part's division
header -- evaluated on the host and compared bit for bit with the oracle on
seeded operands (the value recipe of the benchmarks plus uniformly random
encodings), for two parts of different exponent widths and every format in
them."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1602_04716_gb300", "csrc")
OPS = {"add": 0, "sub": 1, "mul": 2, "div": 4}
_libs = {}


def _lib(e, lo, hi, div):
    key = (e, lo, div)
    if key not in _libs:
        from paper_1602_04716_gb300 import build
        build.generate()
        header = build.div_header(e, lo) if div else build.part_header(e, lo)
        out = os.path.join(tempfile.gettempdir(), "bsfp_gen_part_%d_%d_%d_%d.so" % (e, lo, div, os.getpid()))
        subprocess.check_call(["g++", "-O0", "-w", "-std=c++17", "-fPIC", "-shared", "-DBSFP_HAVE_GEN",
                               "-DBSFP_E=%d" % e, "-DBSFP_M_LO=%d" % lo, "-DBSFP_M_HI=%d" % hi,
                               '-DBSFP_GEN_PART="%s"' % header, "-I", CSRC, "-I", build.GEN_DIR, "-o", out,
                               os.path.join(HERE, "gen_part_host.cpp")])
        L = ctypes.CDLL(out)
        L.host_gen_part.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p] * 3 + [ctypes.c_long] * 2
        L.host_gen_part.restype = ctypes.c_int
        _libs[key] = L
    return _libs[key]


def _check(e, lo, hi, ops):
    tuned = {(4, 3), (4, 4), (5, 7), (5, 10), (8, 7), (8, 23)}
    n = 3000 + 17
    for m in range(lo, hi + 1):
        if (e, m) in tuned or 1 + e + m > 32:
            continue
        B = 1 + e + m
        a = np.concatenate([synth.fp_values(e, m, n, 10 * m + 1), synth.uniform_bits(B, n, 10 * m + 2)]).astype(np.uint32)
        b = np.concatenate([synth.fp_values(e, m, n, 10 * m + 3), synth.uniform_bits(B, n, 10 * m + 4)]).astype(np.uint32)
        pa, pb = oracle.pack(B, a), oracle.pack(B, b)
        S = pa.shape[1]
        for op in ops:
            L = _lib(e, lo, hi, op == "div")
            for rnd in (0, 1):
                out = np.zeros_like(pa)
                assert L.host_gen_part(m, rnd, OPS[op], pa.ctypes.data, pb.ctypes.data, out.ctypes.data, S, S) == 0, \
                    "1/%d/%d %s not printed" % (e, m, op)
                got = oracle.unpack(B, out, a.size)
                want = oracle.binop(op, e, m, rnd, a, b)
                bad = np.nonzero(got != want)[0]
                assert not len(bad), "%s 1/%d/%d rnd=%d: %d bad, first a=%#x b=%#x got %#x want %#x" % (
                    op, e, m, rnd, len(bad), a[bad[0]], b[bad[0]], got[bad[0]], want[bad[0]])


@pytest.mark.parametrize("ops", [("add", "sub", "mul"), ("div",)])
def test_printed_part_netlists_of_exponent_width_2(ops):
    _check(2, 1, 11, ops)


@pytest.mark.parametrize("ops", [("add", "sub", "mul"), ("div",)])
def test_printed_part_netlists_of_exponent_width_6(ops):
    _check(6, 12, 23, ops)
