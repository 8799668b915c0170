"""The library's circuit templates (circuit.cuh), and the gate-by-gate
netlists printed from them for the generated formats (gen_circuits.cuh),
evaluated on the host with 32-bit words and compared bit for bit with the
oracle.  This exercises the same gate-level code the CUDA kernels run,
without a GPU: exhaustively over every operand pair for formats of at most 8
bits and on seeded samples for wider formats, for add, sub, mul and fma2
under RN and RZ."""
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
OPS = ["add", "sub", "mul", "fma2", "div"]

_L = None


def _lib():
    global _L
    if _L is None:
        out = os.path.join(tempfile.gettempdir(), "bsfp_circuit_host_%d.so" % os.getpid())
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-I", CSRC, "-o", out,
                               os.path.join(HERE, "circuit_host.cpp")])
        L = ctypes.CDLL(out)
        L.host_circuit.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p] * 4 + [ctypes.c_long] * 2
        L.host_circuit.restype = ctypes.c_int
        L.host_convert.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p] * 2 + [ctypes.c_long] * 2
        L.host_convert.restype = ctypes.c_int
        L.host_int.argtypes = [ctypes.c_int] * 2 + [ctypes.c_void_p] * 3 + [ctypes.c_long] * 2
        L.host_int.restype = ctypes.c_int
        _L = L
    return _L


_G = None


def _gen_lib():
    """The generated netlists compiled for the host (the build prints them)."""
    global _G
    if _G is None:
        from paper_1602_04716_gb300 import build
        build.generate()
        out = os.path.join(tempfile.gettempdir(), "bsfp_gen_circuit_host_%d.so" % os.getpid())
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-DBSFP_HAVE_GEN", "-I", CSRC,
                               "-I", build.GEN_DIR, "-o", out, os.path.join(HERE, "gen_circuit_host.cpp")])
        L = ctypes.CDLL(out)
        L.host_gen_circuit.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p] * 4 + [ctypes.c_long] * 2
        L.host_gen_circuit.restype = ctypes.c_int
        _G = L
    return _G


def circuit(E, M, rnd, op, a, b, c=None, generated=False):
    """Pack with the oracle's bit loop, run the circuit (the template, or the
    generated netlist), unpack."""
    B = 1 + E + M
    a = np.asarray(a, np.uint32)
    b = np.asarray(b, np.uint32)
    c = np.zeros_like(a) if c is None else np.asarray(c, np.uint32)
    pa, pb, pc = oracle.pack(B, a), oracle.pack(B, b), oracle.pack(B, c)
    S = pa.shape[1]
    out = np.zeros_like(pa)
    fn = _gen_lib().host_gen_circuit if generated else _lib().host_circuit
    rc = fn(E, M, rnd, OPS.index(op), pa.ctypes.data, pb.ctypes.data, pc.ctypes.data, out.ctypes.data, S, S)
    assert rc == 0, "format not in the host harness"
    return oracle.unpack(B, out, a.size)


def _first_bad(got, want, *ins):
    bad = np.nonzero(got != want)[0]
    if not len(bad):
        return ""
    i = bad[0]
    return "%d mismatches; first at %d: in=%s got=%#x want=%#x" % (
        len(bad), i, [hex(int(x[i])) for x in ins], got[i], want[i])


SMALL = [(2, 1), (2, 3), (3, 2), (3, 3), (2, 5), (3, 4), (4, 3), (5, 2)]


MODES = [oracle.RN, oracle.RZ, oracle.RN_FTZ, oracle.RZ_FTZ]


@pytest.mark.parametrize("E,M", SMALL)
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
@pytest.mark.parametrize("rnd", MODES)
def test_circuit_exhaustive_small(E, M, op, rnd):
    a, b = synth.all_pairs(1 + E + M)
    a, b = a.astype(np.uint32), b.astype(np.uint32)
    got = circuit(E, M, rnd, op, a, b)
    want = oracle.binop(op, E, M, rnd, a, b)
    assert (got == want).all(), _first_bad(got, want, a, b)


@pytest.mark.parametrize("rnd", MODES)
def test_circuit_fma2_1_4_3_sampled(rnd):
    n = 1 << 18
    a = synth.uniform_bits(8, n, 11).astype(np.uint32)
    b = synth.uniform_bits(8, n, 12).astype(np.uint32)
    c = synth.uniform_bits(8, n, 13).astype(np.uint32)
    got = circuit(4, 3, rnd, "fma2", a, b, c)
    want = oracle.fma2(4, 3, rnd, a, b, c)
    assert (got == want).all(), _first_bad(got, want, a, b, c)


WIDE = [(4, 4), (5, 4), (4, 5), (5, 7), (5, 10), (8, 7), (8, 23), (3, 23), (8, 2), (6, 9), (7, 13),
        (2, 23), (8, 1), (3, 12)]


@pytest.mark.parametrize("E,M", WIDE)
@pytest.mark.parametrize("rnd", MODES)
def test_circuit_wide_sampled(E, M, rnd):
    n = 1 << 15
    B = 1 + E + M
    for gen in ("fp", "bits"):
        if gen == "fp":
            a, b, c = (synth.fp_values(E, M, n, s).astype(np.uint32) for s in (21, 22, 23))
        else:
            a, b, c = (synth.uniform_bits(B, n, s).astype(np.uint32) for s in (31, 32, 33))
        for op in OPS:
            got = circuit(E, M, rnd, op, a, b, c)
            want = oracle.binop(op, E, M, rnd, a, b, c)
            assert (got == want).all(), "%s %s: %s" % (gen, op, _first_bad(got, want, a, b, c))


GEN = [(4, 3), (4, 4), (5, 7), (5, 10), (8, 7), (8, 23)]


def test_generated_formats_match_the_build_list():
    from paper_1602_04716_gb300 import build
    assert sorted(build.GEN_FORMATS) == sorted(GEN)


@pytest.mark.parametrize("op", ["add", "sub", "mul"])
@pytest.mark.parametrize("rnd", MODES)
def test_generated_netlist_exhaustive_1_4_3(op, rnd):
    a, b = synth.all_pairs(8)
    a, b = a.astype(np.uint32), b.astype(np.uint32)
    got = circuit(4, 3, rnd, op, a, b, generated=True)
    want = oracle.binop(op, 4, 3, rnd, a, b)
    assert (got == want).all(), _first_bad(got, want, a, b)


@pytest.mark.parametrize("E,M", GEN)
@pytest.mark.parametrize("rnd", MODES)
def test_generated_netlist_sampled(E, M, rnd):
    n = 1 << 14
    B = 1 + E + M
    for gen in ("fp", "bits"):
        if gen == "fp":
            a, b, c = (synth.fp_values(E, M, n, s).astype(np.uint32) for s in (41, 42, 43))
        else:
            a, b, c = (synth.uniform_bits(B, n, s).astype(np.uint32) for s in (51, 52, 53))
        for op in OPS:
            got = circuit(E, M, rnd, op, a, b, c, generated=True)
            want = oracle.binop(op, E, M, rnd, a, b, c)
            assert (got == want).all(), "%s %s: %s" % (gen, op, _first_bad(got, want, a, b, c))


CONV = [(2, 1), (3, 2), (4, 3), (5, 2), (3, 4), (4, 4), (5, 7), (5, 10), (8, 7), (8, 23), (6, 9), (7, 13), (3, 23),
        (2, 23), (8, 1)]


def convert(E, M, rnd, direction, x):
    """direction 0: binary32 patterns -> 1/E/M; 1: 1/E/M -> binary32."""
    B = 1 + E + M
    x = np.asarray(x, np.uint32)
    pin = oracle.pack(32 if direction == 0 else B, x)
    S = pin.shape[1]
    out = np.zeros((B if direction == 0 else 32, S), np.uint32)
    rc = _lib().host_convert(E, M, rnd, direction, pin.ctypes.data, out.ctypes.data, S, S)
    assert rc == 0
    return oracle.unpack(B if direction == 0 else 32, out, x.size)


def _f32_samples(n, seed):
    r = synth.splitmix64(seed, 3 * n)
    near = ((r[n:2 * n] & np.uint64(0x807FFFFF)) | ((np.uint64(96) + r[2 * n:] % np.uint64(48)) << np.uint64(23)))
    spec = np.array([0, 0x80000000, 0x7F800000, 0xFF800000, 0x7FC00000, 0x7F800001, 0x00000001, 0x007FFFFF,
                     0x00800000, 0x7F7FFFFF, 0x3F800000], np.uint32)
    return np.concatenate([r[:n].astype(np.uint32), near.astype(np.uint32), (r[2 * n:] & np.uint64(0x807FFFFF))
                           .astype(np.uint32), spec])


@pytest.mark.parametrize("E,M", CONV)
@pytest.mark.parametrize("rnd", MODES)
def test_conversion_circuits(E, M, rnd):
    x = _f32_samples(1 << 13, 300 + 32 * E + M)
    got = convert(E, M, rnd, 0, x)
    want = oracle.from_f32(E, M, rnd, x)
    assert (got == want).all(), "from: " + _first_bad(got, want, x)
    B = 1 + E + M
    y = np.arange(1 << B, dtype=np.uint32) if B <= 14 else synth.uniform_bits(B, 1 << 14, 7).astype(np.uint32)
    got = convert(E, M, rnd, 1, y)
    want = oracle.to_f32(E, M, rnd, y)
    assert (got == want).all(), "to: " + _first_bad(got, want, y)


@pytest.mark.parametrize("w", [1, 2, 3, 5, 8, 9, 13, 16, 17, 24, 31, 32])
def test_integer_circuits(w):
    """The Sec. 3 integer circuits (ripple adder, truncated array multiplier)
    against the oracle: every operand pair for w <= 7, samples beyond."""
    if w <= 7:
        a, b = synth.all_pairs(w)
        a, b = a.astype(np.uint32), b.astype(np.uint32)
    else:
        a, b = (synth.uniform_bits(w, 1 << 15, 700 + w, k).astype(np.uint32) for k in range(2))
    pa, pb = oracle.pack(w, a), oracle.pack(w, b)
    S = pa.shape[1]
    for op, code in (("add", 0), ("sub", 1), ("mul", 2)):
        out = np.zeros_like(pa)
        assert _lib().host_int(w, code, pa.ctypes.data, pb.ctypes.data, out.ctypes.data, S, S) == 0
        got = oracle.unpack(w, out, a.size)
        want = oracle.int_binop(op, w, a, b)
        assert (got == want).all(), "%s w=%d: %s" % (op, w, _first_bad(got, want, a, b))
