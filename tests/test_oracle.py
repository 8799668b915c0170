"""Pins for the CPU oracle (no GPU).

The oracle (``oracle/bsfp_oracle.c``) is checked against things that do not
depend on it:

* the brute-force Fraction checker (``oracle/bruteforce.py``), exhaustively
  over every operand pair of small formats (add, sub, mul; RN and RZ, and both
  with flush to zero, where it searches the normal values only);
* hand-derived values in ``tests/golden/`` (Sec. 5.2's 1/4/3 format, Sec. 2's
  Fig. 1 layout);
* the host FPU: IEEE binary16 through numpy (1/5/10, the paper's FP16),
  binary32 through C ``fesetround`` (1/8/23, the paper's FP32), bfloat16 through
  torch (1/8/7), and binary32 with the CPU's flush-to-zero and
  denormals-are-zero modes through torch (1/8/23 with flush to zero);
* a neighbour check of correct rounding for every sweep format
  (E 3..8 x M 2..23): the result's encoding neighbours bracket the exact value
  as RN-even / RZ require;
* algebraic invariants.
"""
from __future__ import annotations

import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import bruteforce as bf
from tests import _helpers as H

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RND = {"rn": oracle.RN, "rz": oracle.RZ}

SMALL_FORMATS = [(2, 1), (2, 3), (3, 2), (3, 3), (2, 5), (3, 4), (4, 3), (5, 2)]


# ---------------------------------------------------------------------------
# brute force, exhaustive
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("E,M", SMALL_FORMATS)
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
@pytest.mark.parametrize("rnd", [oracle.RN, oracle.RZ, oracle.RN_FTZ, oracle.RZ_FTZ])
def test_exhaustive_vs_bruteforce(E, M, op, rnd):
    F = bf.fmt(E, M)
    a, b = synth.all_pairs(F.B)
    got = oracle.binop(op, E, M, rnd, a, b)
    fn = getattr(F, op)
    want = np.fromiter((fn(int(x), int(y), rnd) for x, y in zip(a, b)), dtype=np.uint32,
                       count=a.size)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, "first mismatch a=%#x b=%#x oracle=%#x brute=%#x" % (
        a[bad[0]], b[bad[0]], got[bad[0]], want[bad[0]])


@pytest.mark.parametrize("E,M", [(4, 3), (3, 3), (4, 4)])
@pytest.mark.parametrize("rnd", [oracle.RN, oracle.RZ, oracle.RN_FTZ, oracle.RZ_FTZ])
def test_fma2_vs_bruteforce_sampled(E, M, rnd):
    F = bf.fmt(E, M)
    n = 6000
    a = synth.uniform_bits(F.B, n, 11, 0)
    b = synth.uniform_bits(F.B, n, 11, 1)
    c = synth.uniform_bits(F.B, n, 11, 2)
    got = oracle.fma2(E, M, rnd, a, b, c)
    want = np.array([F.fma2(int(x), int(y), int(z), rnd) for x, y, z in zip(a, b, c)],
                    dtype=np.uint32)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("E,M", [(4, 4), (5, 4), (4, 5)])
def test_nine_and_ten_bit_vs_bruteforce_sampled(E, M):
    F = bf.fmt(E, M)
    n = 20000
    a = synth.fp_values(E, M, n, 5, 0)
    b = synth.fp_values(E, M, n, 5, 1)
    for rnd in (oracle.RN, oracle.RZ):
        for op in ("add", "mul"):
            got = oracle.binop(op, E, M, rnd, a, b)
            fn = getattr(F, op)
            want = np.array([fn(int(x), int(y), rnd) for x, y in zip(a, b)], dtype=np.uint32)
            assert np.array_equal(got, want), (op, rnd)


# ---------------------------------------------------------------------------
# hand-derived golden values
# ---------------------------------------------------------------------------
def _golden_arith():
    rows = []
    with open(os.path.join(GOLDEN, "arith_1_4_3.txt")) as fh:
        for line in fh:
            body = line.split("#")[0].strip()
            if not body:
                continue
            lhs, exp = body.split("->")
            toks = lhs.split()
            rows.append((toks[0], RND[toks[1]], [int(t, 16) for t in toks[2:]], int(exp, 16),
                         line.strip()))
    return rows


@pytest.mark.parametrize("row", _golden_arith(), ids=lambda r: r[4].split("#")[0].strip())
def test_golden_arith_1_4_3(row):
    op, rnd, args, want, _ = row
    vals = [np.array([v], dtype=np.uint32) for v in args]
    got = int(oracle.binop(op, 4, 3, rnd, *vals)[0])
    assert got == want, "%s: got %#x" % (row[4], got)


def _golden_layout():
    cases, cur = [], None
    with open(os.path.join(GOLDEN, "fig1_layout_1_4_3.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, rest = line.split(None, 1)
            if key == "case":
                cur = {"name": rest}
                cases.append(cur)
            elif key == "elems":
                cur["elems"] = [int(t, 16) for t in rest.split()]
            elif key == "words":
                cur["words"] = [int(t, 16) for t in rest.split()]
    return cases


@pytest.mark.parametrize("case", _golden_layout(), ids=lambda c: c["name"])
def test_golden_fig1_layout(case):
    x = np.array(case["elems"], dtype=np.uint32)
    planes = oracle.pack(8, x)
    assert planes.shape == (8, oracle.plane_stride(16))
    assert [int(w) for w in planes[:, 0]] == case["words"]
    assert not planes[:, 1:].any()          # padding words are zero
    assert np.array_equal(oracle.unpack(8, planes, 16), x)


# ---------------------------------------------------------------------------
# pack / unpack properties
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("B,n", [(8, 1), (9, 31), (13, 32), (13, 33), (16, 1023), (32, 1025), (6, 4097)])
def test_pack_roundtrip_and_counts(B, n):
    x = synth.uniform_bits(B, n, 3).astype(np.uint32)
    planes = oracle.pack(B, x)
    S = oracle.plane_stride(n)
    assert S % 32 == 0 and S * 32 >= n
    assert np.array_equal(oracle.unpack(B, planes, n), x)
    # plane b holds exactly the elements whose bit b is set (popcount check)
    for b in range(B):
        ones = sum(bin(int(w)).count("1") for w in planes[b])
        assert ones == int(((x >> b) & 1).sum())
    # lanes past n are zero
    last = n // 32
    if n % 32:
        assert not (planes[:, last] >> (n % 32)).any()
    assert not planes[:, (n + 31) // 32:].any()


# ---------------------------------------------------------------------------
# host IEEE pins
# ---------------------------------------------------------------------------
def _f16_specials():
    v = [0x0000, 0x8000, 0x0001, 0x8001, 0x03FF, 0x0400, 0x83FF, 0x3C00, 0xBC00, 0x7BFF, 0xFBFF,
         0x7C00, 0xFC00, 0x7E00, 0x7C01, 0x3BFF, 0x3C01, 0x4000, 0x0200, 0x1400, 0x5BFF]
    a = np.repeat(np.array(v, np.uint32), len(v))
    b = np.tile(np.array(v, np.uint32), len(v))
    return a, b


def _f16_operands():
    n = 1 << 17
    a1 = synth.uniform_bits(16, n, 21, 0).astype(np.uint32)
    b1 = synth.uniform_bits(16, n, 21, 1).astype(np.uint32)
    a2 = synth.fp_values(5, 10, n, 22, 0).astype(np.uint32)
    b2 = synth.fp_values(5, 10, n, 22, 1).astype(np.uint32)
    # nearby exponents, so that cancellation and ties happen often
    a3 = a2.copy()
    b3 = (a2 ^ synth.uniform_bits(6, n, 23).astype(np.uint32)) ^ 0x8000
    sa, sb = _f16_specials()
    return np.concatenate([a1, a2, a3, sa]), np.concatenate([b1, b2, b3, sb])


@pytest.mark.parametrize("op", ["add", "mul", "div"])
def test_binary16_rn_vs_numpy(op):
    """numpy computes a binary16 result in binary32 and rounds it to binary16;
    that double rounding is innocuous for +, * and / since 24 >= 2 * 11 + 2
    (Figueroa's theorem)."""
    a, b = _f16_operands()
    fa = a.astype(np.uint16).view(np.float16)
    fb = b.astype(np.uint16).view(np.float16)
    with np.errstate(all="ignore"):
        ref = {"add": fa + fb, "mul": fa * fb, "div": fa / fb}[op]
    want = ref.view(np.uint16).astype(np.uint32)
    got = oracle.binop(op, 5, 10, oracle.RN, a, b)
    ok = H.nan_class_equal(5, 10, got, want)
    assert ok.all(), "first mismatch %#x %#x" % (a[~ok][0], b[~ok][0])


@pytest.mark.parametrize("op", ["add", "mul", "div"])
def test_binary16_rz_vs_exact_double(op):
    """binary16 sums and products are exact in binary64; truncating that exact
    value toward zero is the RZ result.  Quotients are not exact, but a
    quotient of two binary16 values that is not itself a binary16 value lies
    at least 2^-22 (relative) from every binary16 value, far more than the
    2^-53 of the binary64 rounding, so truncating the binary64 quotient gives
    the same binary16 value."""
    a, b = _f16_operands()
    fa = a.astype(np.uint16).view(np.float16).astype(np.float64)
    fb = b.astype(np.uint16).view(np.float16).astype(np.float64)
    with np.errstate(all="ignore"):
        ex = {"add": fa + fb, "mul": fa * fb, "div": fa / fb}[op]
        r = ex.astype(np.float16)                          # correctly rounded (RN)
        over = np.abs(r.astype(np.float64)) > np.abs(ex)   # RN went away from zero
        r = np.where(over, np.nextafter(r, np.float16(0)), r)
    want = r.view(np.uint16).astype(np.uint32)
    # exact zero results: +0 except (-0)+(-0); numpy already follows IEEE here
    got = oracle.binop(op, 5, 10, oracle.RZ, a, b)
    ok = H.nan_class_equal(5, 10, got, want)
    assert ok.all(), "first mismatch %#x %#x got %#x want %#x" % (
        a[~ok][0], b[~ok][0], got[~ok][0], want[~ok][0])


@pytest.mark.parametrize("op", ["add", "mul", "div"])
@pytest.mark.parametrize("rnd", [oracle.RN, oracle.RZ])
def test_binary32_vs_host_fenv(op, rnd):
    n = 1 << 17
    a = np.concatenate([synth.splitmix64(31, n, 0).astype(np.uint32),
                        synth.fp_values(8, 23, n, 32, 0).astype(np.uint32)])
    b = np.concatenate([synth.splitmix64(31, n, 1).astype(np.uint32),
                        synth.fp_values(8, 23, n, 32, 1).astype(np.uint32)])
    # near-cancellation pairs
    b2 = (a[n:] ^ 0x80000000) ^ (synth.splitmix64(33, n).astype(np.uint32) & 0x3FF)
    a = np.concatenate([a, a[n:]])
    b = np.concatenate([b, b2])
    want = H.host_f32(op, rnd, a, b)
    got = oracle.binop(op, 8, 23, rnd, a, b)
    ok = H.nan_class_equal(8, 23, got, want)
    assert ok.all(), "first mismatch %#x %#x got %#x want %#x" % (
        a[~ok][0], b[~ok][0], got[~ok][0], want[~ok][0])


@pytest.mark.parametrize("op", ["add", "sub", "mul"])
def test_binary32_flush_to_zero_vs_host(op):
    """1/8/23 RN with flush to zero against the host FPU's binary32 with
    flush-to-zero and denormals-are-zero set (torch.set_flush_denormal).  A
    product whose exact magnitude lies in [2^-126 (1 - 2^-24), 2^-126) is
    tiny before rounding but rounds to the smallest normal, so FPUs that judge
    tininess after rounding keep it: those few pairs are left out (sums of
    flushed operands are exact, so add and sub have no such band)."""
    torch = pytest.importorskip("torch")
    n = 1 << 16
    # exponent fields near the bottom of the range, so that subnormal operands
    # and tiny results are common, plus uniform bit patterns
    r = synth.splitmix64(61, 8 * n)
    low = lambda k: ((r[k::8] & np.uint64(0x807FFFFF)) |
                     ((r[k + 4::8] % np.uint64(70)) << np.uint64(23))).astype(np.uint32)
    a = np.concatenate([low(0), synth.splitmix64(62, n, 0).astype(np.uint32)])
    b = np.concatenate([low(1), synth.splitmix64(62, n, 1).astype(np.uint32)])
    if op == "add":   # cancellation towards the bottom of the range
        b[:n // 4] = (a[:n // 4] ^ 0x80000000) ^ (low(3)[:n // 4] & 0x3F)
    old_threads = torch.get_num_threads()
    torch.set_num_threads(1)
    try:
        if not torch.set_flush_denormal(True):
            pytest.skip("the host cannot flush denormals")
        ta = torch.from_numpy(a.view(np.float32).copy())
        tb = torch.from_numpy(b.view(np.float32).copy())
        tr = {"add": ta + tb, "sub": ta - tb, "mul": ta * tb}[op]
        want = tr.numpy().view(np.uint32).astype(np.uint32)
    finally:
        torch.set_flush_denormal(False)
        torch.set_num_threads(old_threads)
    got = oracle.binop(op, 8, 23, oracle.RN_FTZ, a, b)
    keep = np.ones(a.size, bool)
    if op == "mul":
        fa = np.where((a >> 23) & 0xFF, a.view(np.float32), 0).astype(np.float64)
        fb = np.where((b >> 23) & 0xFF, b.view(np.float32), 0).astype(np.float64)
        ex = np.abs(fa * fb)                                 # exact: 48-bit products fit in a double
        keep = ~((ex < 2.0 ** -126) & (ex >= 2.0 ** -126 * (1 - 2.0 ** -24)))
    ok = H.nan_class_equal(8, 23, got, want) | ~keep
    assert keep.sum() > a.size - 16
    assert ok.all(), "first mismatch %#x %#x got %#x want %#x" % (
        a[~ok][0], b[~ok][0], got[~ok][0], want[~ok][0])
    # flushing changed something: the sample does reach the subnormal range
    plain = oracle.binop(op, 8, 23, oracle.RN, a, b)
    assert (plain != got).sum() > 100


def test_bfloat16_rn_vs_torch():
    torch = pytest.importorskip("torch")
    # subnormal behaviour of torch's CPU bfloat16 first (2^-133 + 2^-133 = 2^-132)
    tiny = torch.tensor([0x0001], dtype=torch.int16).view(torch.bfloat16)
    assert int((tiny + tiny).view(torch.int16)) == 0x0002
    n = 1 << 17
    a = np.concatenate([synth.uniform_bits(16, n, 41, 0), synth.fp_values(8, 7, n, 42, 0)]).astype(np.uint32)
    b = np.concatenate([synth.uniform_bits(16, n, 41, 1), synth.fp_values(8, 7, n, 42, 1)]).astype(np.uint32)
    ta = torch.from_numpy(a.astype(np.int32).astype(np.int16)).view(torch.bfloat16)
    tb = torch.from_numpy(b.astype(np.int32).astype(np.int16)).view(torch.bfloat16)
    for op in ("add", "mul", "div"):
        r = {"add": ta + tb, "mul": ta * tb, "div": ta / tb}[op]   # binary32 result rounded: 24 >= 2*8+2
        want = r.view(torch.int16).numpy().astype(np.uint16).astype(np.uint32)
        got = oracle.binop(op, 8, 7, oracle.RN, a, b)
        ok = H.nan_class_equal(8, 7, got, want)
        assert ok.all(), (op, hex(a[~ok][0]), hex(b[~ok][0]))


# ---------------------------------------------------------------------------
# neighbour check of correct rounding, every sweep format
# ---------------------------------------------------------------------------
def _check_rounding(E, M, rnd, v: Fraction, r: int):
    """Assert that encoding r is the RN-even / RZ rounding of nonzero exact v."""
    bias = (1 << (E - 1)) - 1
    emax = (1 << E) - 1
    sign_bit = 1 << (E + M)
    mag = r & (sign_bit - 1)
    s = 1 if v < 0 else 0
    a = -v if s else v
    assert (r >> (E + M)) & 1 == s, "sign"
    inf_code = emax << M
    maxf = H.value(E, M, inf_code - 1)
    ovf = maxf + Fraction(2) ** (emax - 1 - bias - M) / 2
    if rnd == oracle.RZ:
        if a > maxf:
            assert mag == inf_code - 1
            return
        assert mag < inf_code
        lo = H.value(E, M, mag)
        assert lo <= a < H.value(E, M, mag + 1) if mag + 1 < inf_code else lo <= a
        return
    if mag == inf_code:
        assert a >= ovf
        return
    assert mag < inf_code
    x = H.value(E, M, mag)
    if mag > 0:
        lo_mid = (H.value(E, M, mag - 1) + x) / 2
        assert a >= lo_mid and (a != lo_mid or mag % 2 == 0)
    hi_mid = (x + H.value(E, M, mag + 1)) / 2 if mag + 1 < inf_code else ovf
    assert a <= hi_mid and (a != hi_mid or mag % 2 == 0)


SWEEP = [(E, M) for E in range(3, 9) for M in range(2, 24)]


@pytest.mark.parametrize("E", range(3, 9))
def test_sweep_formats_correct_rounding(E):
    n = 120
    for M in range(2, 24):
        a = synth.fp_values(E, M, n, 51 + M, 0).astype(np.uint32)
        b = synth.fp_values(E, M, n, 51 + M, 1).astype(np.uint32)
        b[: n // 4] = a[: n // 4] ^ (1 << (E + M)) ^ (b[: n // 4] & 7)   # near-cancellation
        for rnd in (oracle.RN, oracle.RZ):
            for op in ("add", "mul"):
                got = oracle.binop(op, E, M, rnd, a, b)
                for x, y, r in zip(a, b, got):
                    if any(H.is_nan(E, M, t) or H.is_inf(E, M, t) for t in (x, y)):
                        continue
                    vx, vy = H.value(E, M, x), H.value(E, M, y)
                    v = vx + vy if op == "add" else vx * vy
                    if v == 0:
                        continue
                    _check_rounding(E, M, rnd, v, int(r))


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("E,M", [(3, 2), (4, 4), (5, 7), (6, 9), (8, 23), (3, 23), (8, 2)])
@pytest.mark.parametrize("rnd", [oracle.RN, oracle.RZ])
def test_invariants(E, M, rnd):
    n = 4096
    B = 1 + E + M
    sb = np.uint32(1 << (E + M))
    x = synth.fp_values(E, M, n, 61, 0).astype(np.uint32)
    y = synth.fp_values(E, M, n, 61, 1).astype(np.uint32)
    emask = ((1 << E) - 1) << M
    fmask = (1 << M) - 1
    nan = lambda t: ((t & emask) == emask) & ((t & fmask) != 0)
    fin = lambda t: (t & emask) != emask
    add = lambda p, q: oracle.binop("add", E, M, rnd, p, q)
    mul = lambda p, q: oracle.binop("mul", E, M, rnd, p, q)
    sub = lambda p, q: oracle.binop("sub", E, M, rnd, p, q)
    assert np.array_equal(add(x, y), add(y, x))
    assert np.array_equal(mul(x, y), mul(y, x))
    negz = np.full(n, sb, np.uint32)
    keep = ~nan(x)
    assert np.array_equal(add(x, negz)[keep], x[keep])                  # x + (-0) = x
    one = np.full(n, ((1 << (E - 1)) - 1) << M, np.uint32)
    assert np.array_equal(mul(x, one)[keep], x[keep])                   # x * 1 = x
    f = fin(x)
    assert not sub(x, x)[f].any()                                       # x - x = +0
    r, rn = add(x, y), add(x ^ sb, y ^ sb)
    ok = ~nan(r) & ((r & (sb - 1)) != 0)     # an exact-zero sum is +0 both ways
    assert np.array_equal(rn[ok], (r ^ sb)[ok])                         # sign symmetry
    m1, m2 = mul(x, y), mul(x ^ sb, y)
    ok = ~nan(m1)
    assert np.array_equal(m2[ok], (m1 ^ sb)[ok])
    assert np.array_equal(sub(x, y), add(x, y ^ sb))
    assert B <= 32


# ---------------------------------------------------------------------------
# conversions binary32 <-> 1/E/M
# ---------------------------------------------------------------------------
def _f32_operands(n=1 << 16, seed=81):
    """Uniform binary32 patterns, values near every target's range (exponent
    fields 100..140 cover the normal ranges of 1/5/M and their edges), the
    binary32 subnormals, and the specials."""
    r = synth.splitmix64(seed, 3 * n)
    u = r[:n].astype(np.uint32)
    mid = ((r[n:2 * n] & np.uint64(0x807FFFFF)) | ((np.uint64(100) + r[2 * n:] % np.uint64(41)) << np.uint64(23)))
    sub = (r[2 * n:] & np.uint64(0x807FFFFF)).astype(np.uint32)
    spec = np.array([0, 0x80000000, 0x7F800000, 0xFF800000, 0x7FC00000, 0x7F800001, 0xFFFFFFFF, 0x00000001,
                     0x007FFFFF, 0x00800000, 0x7F7FFFFF, 0x3F800000, 0x477FE000, 0x477FF000, 0x477FF001,
                     0x38800000, 0x387FC000, 0x33800000, 0x33000000, 0x33000001], np.uint32)
    return np.concatenate([u, mid.astype(np.uint32), sub, spec])


@pytest.mark.parametrize("rnd", [oracle.RN, oracle.RZ])
def test_from_f32_binary16_vs_numpy(rnd):
    """1/5/10 from binary32: numpy's binary32 -> binary16 cast rounds to
    nearest even; stepping it one place toward zero when it went away from
    zero gives round toward zero."""
    x = _f32_operands()
    f = x.view(np.float32)
    with np.errstate(all="ignore"):
        h = f.astype(np.float16)
        if rnd == oracle.RZ:
            away = np.abs(h.astype(np.float32)) > np.abs(f)
            h = np.where(away, np.nextafter(h, np.float16(0)), h)
    want = h.view(np.uint16).astype(np.uint32)
    got = oracle.from_f32(5, 10, rnd, x)
    ok = H.nan_class_equal(5, 10, got, want)
    assert ok.all(), "first mismatch %#x got %#x want %#x" % (x[~ok][0], got[~ok][0], want[~ok][0])


def test_from_f32_bfloat16_vs_torch():
    torch = pytest.importorskip("torch")
    x = _f32_operands()
    t = torch.from_numpy(x.view(np.float32).copy()).to(torch.bfloat16)
    want = t.view(torch.int16).numpy().astype(np.uint16).astype(np.uint32)
    got = oracle.from_f32(8, 7, oracle.RN, x)
    ok = H.nan_class_equal(8, 7, got, want)
    assert ok.all(), "first mismatch %#x got %#x want %#x" % (x[~ok][0], got[~ok][0], want[~ok][0])


def test_from_f32_binary32_is_the_identity():
    x = _f32_operands()
    for rnd in (oracle.RN, oracle.RZ):
        got = oracle.from_f32(8, 23, rnd, x)
        ok = H.nan_class_equal(8, 23, got, x)
        assert ok.all()


@pytest.mark.parametrize("E,M", [(2, 1), (3, 2), (4, 3), (5, 2), (3, 4)])
@pytest.mark.parametrize("rnd", [oracle.RN, oracle.RZ, oracle.RN_FTZ, oracle.RZ_FTZ])
def test_from_f32_vs_bruteforce(E, M, rnd):
    F = bf.fmt(E, M)
    x = _f32_operands(1 << 12, 90 + E * 8 + M)
    got = oracle.from_f32(E, M, rnd, x)
    for xi, gi in zip(x, got):
        s, e, fr = (int(xi) >> 31) & 1, (int(xi) >> 23) & 255, int(xi) & 0x7FFFFF
        if e == 255:
            want = F.nan if fr else F.inf(s)
        else:
            v = Fraction(fr if e == 0 else fr + (1 << 23), 1 << 23) * Fraction(2) ** ((e if e else 1) - 127)
            want = F.from_value(-v if s else v, s, rnd)
        assert int(gi) == want, "x=%#x got %#x want %#x" % (xi, gi, want)


def test_to_f32_vs_host_casts():
    """1/5/10 and 1/8/7 widen exactly to binary32 through numpy / torch."""
    torch = pytest.importorskip("torch")
    h = np.arange(1 << 16, dtype=np.uint32)
    want = h.astype(np.uint16).view(np.float16).astype(np.float32).view(np.uint32)
    got = oracle.to_f32(5, 10, oracle.RN, h)
    assert H.nan_class_equal(8, 23, got, want).all()
    t = torch.from_numpy(h.astype(np.uint16).view(np.int16).copy()).view(torch.bfloat16).to(torch.float32)
    want = t.view(torch.int32).numpy().view(np.uint32)
    got = oracle.to_f32(8, 7, oracle.RN, h)
    assert H.nan_class_equal(8, 23, got, want).all()


@pytest.mark.parametrize("E,M", [(2, 1), (3, 2), (4, 3), (6, 9), (7, 13)])
def test_to_f32_round_trips(E, M):
    """Every value of 1/E/M is a binary32 value: converting it to binary32 and
    back (either rounding) returns it, NaNs as the canonical NaN."""
    B = 1 + E + M
    x = (np.arange(1 << B, dtype=np.uint32) if B <= 16 else synth.uniform_bits(B, 1 << 16, 3).astype(np.uint32))
    for rnd in (oracle.RN, oracle.RZ):
        back = oracle.from_f32(E, M, rnd, oracle.to_f32(E, M, rnd, x))
        assert H.nan_class_equal(E, M, back, x).all()
        nan = np.array([H.is_nan(E, M, v) for v in x])
        assert (back[nan] == (((1 << E) - 1) << M | 1 << (M - 1))).all()


# ---------------------------------------------------------------------------
# integer bitslice vectors (Sec. 3)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("w,dt", [(8, np.uint8), (16, np.uint16), (32, np.uint32)])
@pytest.mark.parametrize("op", ["add", "sub", "mul"])
def test_int_ops_vs_numpy_wraparound(w, dt, op):
    """At the machine widths the w-bit operations are numpy's unsigned
    wrap-around arithmetic."""
    n = 1 << 16
    a = synth.uniform_bits(w, n, 111, 0).astype(np.uint32)
    b = synth.uniform_bits(w, n, 111, 1).astype(np.uint32)
    x, y = a.astype(dt), b.astype(dt)
    with np.errstate(over="ignore"):
        want = {"add": x + y, "sub": x - y, "mul": x * y}[op].astype(np.uint32)
    assert (oracle.int_binop(op, w, a, b) == want).all()


@pytest.mark.parametrize("w", [1, 2, 3, 5, 9, 13, 17, 23, 31])
def test_int_ops_invariants(w):
    """Ring laws modulo 2^w: commutativity, 0 and 1, a - a = 0, (a - b) + b = a,
    distributivity, and 2^(w-1) * 2 = 0."""
    n = 1 << 14
    a, b, c = (synth.uniform_bits(w, n, 120 + w, k).astype(np.uint32) for k in range(3))
    add = lambda x, y: oracle.int_binop("add", w, x, y)
    sub = lambda x, y: oracle.int_binop("sub", w, x, y)
    mul = lambda x, y: oracle.int_binop("mul", w, x, y)
    zero, one = np.zeros_like(a), np.ones_like(a)
    assert (add(a, b) == add(b, a)).all() and (mul(a, b) == mul(b, a)).all()
    assert (add(a, zero) == a).all() and (mul(a, one) == a).all() and (mul(a, zero) == 0).all()
    assert (sub(a, a) == 0).all() and (add(sub(a, b), b) == a).all()
    assert (mul(a, add(b, c)) == add(mul(a, b), mul(a, c))).all()
    top = np.full_like(a, 1 << (w - 1))
    assert (mul(top, np.full_like(a, 2)) == 0).all()
    assert (a < (1 << w)).all() and (add(a, b) < (1 << w)).all()
