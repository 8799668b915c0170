"""The transposes of pack and unpack on the CPU: bit_transpose.cuh compiled
for the host and driven lane by lane and tile by tile as the kernels drive
it, compared bit for bit with the oracle's pack and unpack (the definition
of the layout, Sec. 2, Fig. 1), for every container width, every plane
count, ragged tails and junk above bit B.  Also checks that the staged
16-byte accesses of each quarter-warp hit eight different bank groups."""
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

_lib = None


def lib():
    global _lib
    if _lib is None:
        out = os.path.join(tempfile.gettempdir(), "bsfp_transpose_host_%d.so" % os.getpid())
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-I", CSRC, "-o", out,
                               os.path.join(HERE, "transpose_host.cpp")])
        L = ctypes.CDLL(out)
        L.tp_pack.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_long, ctypes.c_int, ctypes.c_void_p,
                              ctypes.c_long]
        L.tp_unpack.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_long, ctypes.c_int, ctypes.c_void_p,
                                ctypes.c_long]
        L.tp_stage_offset.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.tp_stage_offset.restype = ctypes.c_long
        _lib = L
    return _lib


def stride(n):
    return ((n + 31) // 32 + 31) // 32 * 32


def container(B):
    return (1, np.uint8) if B <= 8 else ((2, np.uint16) if B <= 16 else (4, np.uint32))


@pytest.mark.parametrize("B", [1, 3, 5, 8, 9, 12, 13, 16, 17, 24, 31, 32])
@pytest.mark.parametrize("n", [1, 31, 1023, 1024, 1025, 3000, 4096 + 77])
def test_pack_unpack_match_the_layout(B, n):
    cb, dt = container(B)
    raw = synth.uniform_bits(8 * cb, n, 1000 + B).astype(dt)   # junk above bit B too
    S = stride(n)
    planes = np.full(B * S, 0xDEADBEEF, dtype=np.uint32)
    assert lib().tp_pack(cb, raw.ctypes.data, n, B, planes.ctypes.data, S) == 0
    want = oracle.pack(B, raw.astype(np.uint32) & np.uint32((1 << B) - 1 if B < 32 else 0xFFFFFFFF))
    assert (planes.reshape(B, S) == want.reshape(B, S)).all()
    back = np.full(n, 0xA5A5A5A5 & ((1 << (8 * cb)) - 1), dtype=dt)
    assert lib().tp_unpack(cb, planes.ctypes.data, S, B, back.ctypes.data, n) == 0
    mask = (1 << B) - 1
    assert (back.astype(np.uint64) == (raw.astype(np.uint64) & mask)).all()


@pytest.mark.parametrize("cb", [1, 2, 4])
def test_staged_chunks_of_a_quarter_warp_use_eight_bank_groups(cb):
    L = lib()
    for q in range(2 * cb):
        for quarter in range(4):
            groups = {(L.tp_stage_offset(cb, lane, q) // 16) % 8 for lane in range(8 * quarter, 8 * quarter + 8)}
            assert len(groups) == 8
    # every lane reads each of its 2*cb chunks exactly once, inside its column
    for lane in range(32):
        offs = sorted(L.tp_stage_offset(cb, lane, q) for q in range(2 * cb))
        assert offs == [32 * cb * lane + 16 * k for k in range(2 * cb)]
