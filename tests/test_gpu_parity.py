"""Parity of the CUDA path with the oracle, bit for bit, through the C ABI.

Every result is integer logic, so the bar is exact equality of encodings and
of whole plane buffers (padding included).  Operands for the op tests are
packed by the oracle on the host, so each kernel is checked on its own:
pack and unpack against the oracle's bit loops, each op against the oracle's
exact-then-round arithmetic.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_1602_04716_gb300 as bs  # noqa: E402

pytestmark = pytest.mark.gpu

OPS = ["add", "sub", "mul", "fma2", "div"]
RNDS = [oracle.RN, oracle.RZ]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


# ------------------------------------------------------------ helpers ---
def dev(x: np.ndarray):
    x = np.ascontiguousarray(x)
    view = {1: np.uint8, 2: np.int16, 4: np.int32}[x.dtype.itemsize]
    return torch.from_numpy(x.view(view).copy()).cuda()


def host_u32(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def gpu_op(op, E, M, rnd, a, b, c=None, wpt=None, bps=0):
    """Oracle-packed operands -> GPU op -> planes (B, S) on the host."""
    B = 1 + E + M
    f = bs.Format(E, M, rnd)
    n = len(a)
    pa, pb = dev(oracle.pack(B, a)), dev(oracle.pack(B, b))
    pc = dev(oracle.pack(B, c)) if c is not None else None
    out = torch.full_like(pa, -1)
    if wpt is not None:
        bs.bsfp_set_variant(f, op, wpt, bps)
    bs.bsfp_op(op, f, pa, pb, out, n, c=pc)
    torch.cuda.synchronize()
    return host_u32(out).reshape(B, -1)


def want_planes(op, E, M, rnd, a, b, c=None):
    B = 1 + E + M
    return oracle.pack(B, oracle.binop(op, E, M, rnd, a, b, c))


def describe(got, want, B, n, *ins):
    if (got == want).all():
        return ""
    g = oracle.unpack(B, got, n)
    w = oracle.unpack(B, want, n)
    bad = np.nonzero(g != w)[0]
    if not len(bad):
        return "padding differs"
    i = bad[0]
    return "%d/%d mismatches; first at %d: in=%s got=%#x want=%#x" % (
        len(bad), n, i, [hex(int(x[i])) for x in ins if x is not None], g[i], w[i])


def check(op, E, M, rnd, a, b, c=None, **kw):
    B = 1 + E + M
    a = np.asarray(a, np.uint32)
    b = np.asarray(b, np.uint32)
    c = None if c is None else np.asarray(c, np.uint32)
    if op == "fma2" and c is None:
        c = synth.fp_values(E, M, len(a), 99).astype(np.uint32)
    got = gpu_op(op, E, M, rnd, a, b, c, **kw)
    want = want_planes(op, E, M, rnd, a, b, c)
    assert (got == want).all(), "%s 1/%d/%d rnd=%d: %s" % (op, E, M, rnd, describe(got, want, B, len(a), a, b, c))


# ------------------------------------------------------ pack / unpack ---
SIZES = [1, 31, 32, 33, 1023, 1024, 1025, 4097, 65537, 100003]


@pytest.mark.parametrize("E,M", [(4, 3), (2, 1), (4, 4), (5, 10), (8, 7), (8, 23), (3, 12), (6, 17)])
@pytest.mark.parametrize("n", SIZES)
def test_pack_unpack_vs_oracle(E, M, n):
    B = 1 + E + M
    f = bs.Format(E, M)
    cb = bs.bsfp_container_bytes(f)
    cdt = {1: np.uint8, 2: np.uint16, 4: np.uint32}[cb]
    # containers carry junk above bit B: pack must ignore it
    raw = synth.uniform_bits(8 * cb, n, 7 + B, dtype=cdt)
    x = (raw.astype(np.uint64) & ((1 << B) - 1)).astype(np.uint32)
    planes = torch.full((B * bs.bsfp_plane_stride(n),), -1, dtype=torch.int32, device="cuda")
    bs.bsfp_pack(f, dev(raw), n, planes)
    back = torch.full((n,), -1, dtype=bs.container_dtype(f), device="cuda")
    bs.bsfp_unpack(f, planes, n, back)
    torch.cuda.synchronize()
    got_planes = host_u32(planes).reshape(B, -1)
    want_planes_ = oracle.pack(B, x)
    assert (got_planes == want_planes_).all(), "pack differs from the oracle"
    got = back.cpu().numpy().view(cdt).astype(np.uint32)
    assert (got == x).all(), "unpack(pack(x)) != x"


@pytest.mark.parametrize("E,M", [(4, 3), (5, 7), (8, 23), (2, 1), (6, 17)])
@pytest.mark.parametrize("offset", [1, 3])
def test_pack_unpack_standard_array_not_16_byte_aligned(E, M, offset):
    """A standard array aligned only to its container size (here `offset`
    containers past a 16-byte boundary) takes the element-by-element path of
    every tile; results equal the oracle's, and unpack writes exactly n
    containers (the guard containers around the output stay untouched)."""
    B = 1 + E + M
    n = 5 * 1024 + 333
    f = bs.Format(E, M)
    cb = bs.bsfp_container_bytes(f)
    cdt = {1: np.uint8, 2: np.uint16, 4: np.uint32}[cb]
    raw = synth.uniform_bits(8 * cb, n, 41 + B, dtype=cdt)
    x = (raw.astype(np.uint64) & ((1 << B) - 1)).astype(np.uint32)
    base = torch.zeros(n + 16, dtype=bs.container_dtype(f), device="cuda")
    base[offset:offset + n] = dev(raw)
    planes = torch.full((B * bs.bsfp_plane_stride(n),), -1, dtype=torch.int32, device="cuda")
    bs.bsfp_pack(f, base[offset:offset + n], n, planes)
    assert (host_u32(planes).reshape(B, -1) == oracle.pack(B, x)).all()
    guard = torch.full((n + 16,), 0x5A, dtype=bs.container_dtype(f), device="cuda")
    bs.bsfp_unpack(f, planes, n, guard[offset:offset + n])
    g = guard.cpu().numpy().view(cdt).astype(np.uint32)
    assert (g[offset:offset + n] == x).all()
    assert (g[:offset] == 0x5A).all() and (g[offset + n:] == 0x5A).all()


def test_unpack_of_oracle_planes():
    E, M, n = 5, 7, 70001
    x = synth.fp_values(E, M, n, 3).astype(np.uint32)
    planes = dev(oracle.pack(13, x))
    out = torch.empty(n, dtype=torch.int16, device="cuda")
    bs.bsfp_unpack(bs.Format(E, M), planes, n, out)
    assert (out.cpu().numpy().view(np.uint16).astype(np.uint32) == oracle.unpack(13, oracle.pack(13, x), n)).all()


# --------------------------------------------------- exhaustive small ---
SMALL = [(2, 1), (2, 3), (3, 2), (3, 3), (2, 5), (3, 4), (4, 3), (5, 2)]


@pytest.mark.parametrize("E,M", SMALL)
@pytest.mark.parametrize("rnd", RNDS)
def test_exhaustive_pairs_small_formats(E, M, rnd):
    a, b = synth.all_pairs(1 + E + M)
    for op in ("add", "sub", "mul", "div"):
        check(op, E, M, rnd, a, b)


@pytest.mark.parametrize("rnd", RNDS)
def test_exhaustive_pairs_1_4_4(rnd):
    a, b = synth.all_pairs(9)
    for op in ("add", "sub", "mul", "div"):
        check(op, 4, 4, rnd, a, b)


@pytest.mark.parametrize("rnd", RNDS)
def test_fma2_exhaustive_triples_1_4_3(rnd):
    i = np.arange(1 << 24, dtype=np.uint32)
    a, b, c = i >> 16, (i >> 8) & 255, i & 255
    check("fma2", 4, 3, rnd, a, b, c)


# ------------------------------------------------ every compiled format ---
@pytest.mark.parametrize("E", range(2, 9))
def test_every_format_every_op(E):
    """Each of the 23 formats 1/E/1 .. 1/E/23, four ops, both roundings, on
    seeded values of the workload recipe plus uniformly random encodings, at a
    length with a ragged tail."""
    n = 5000 + 17 * E
    for M in range(1, 24):
        B = 1 + E + M
        a = np.concatenate([synth.fp_values(E, M, n, 1000 + M).astype(np.uint32),
                            synth.uniform_bits(B, n, 2000 + M).astype(np.uint32)])
        b = np.concatenate([synth.fp_values(E, M, n, 3000 + M).astype(np.uint32),
                            synth.uniform_bits(B, n, 4000 + M).astype(np.uint32)])
        c = np.concatenate([synth.fp_values(E, M, n, 5000 + M).astype(np.uint32),
                            synth.uniform_bits(B, n, 6000 + M).astype(np.uint32)])
        for rnd in RNDS:
            for op in OPS:
                check(op, E, M, rnd, a, b, c if op == "fma2" else None)


TUNED = [(4, 3), (4, 4), (5, 7), (5, 10), (8, 7), (8, 23)]


@pytest.mark.parametrize("E,M", TUNED)
def test_every_launch_variant(E, M):
    n = 200_000 + 13
    a, b, c = (synth.fp_values(E, M, n, s).astype(np.uint32) for s in (41, 42, 43))
    for op in OPS:
        f = bs.Format(E, M, oracle.RN)
        for wpt in bs.bsfp_variants_compiled(f, op):
            for bps in (0, 1):
                check(op, E, M, oracle.RN, a, b, c if op == "fma2" else None, wpt=wpt, bps=bps)
        bs.bsfp_set_variant(f, op, 0, 0)


# ----------------------------------------------------- flush to zero ---
FTZ_MODES = [oracle.RN_FTZ, oracle.RZ_FTZ]


@pytest.mark.parametrize("rnd", FTZ_MODES)
def test_flush_to_zero_exhaustive_1_4_3(rnd):
    a, b = synth.all_pairs(8)
    for op in ("add", "sub", "mul", "div"):
        check(op, 4, 3, rnd, a, b)
    i = np.arange(1 << 24, dtype=np.uint32)
    check("fma2", 4, 3, rnd, i >> 16, (i >> 8) & 255, i & 255)


@pytest.mark.parametrize("E,M", TUNED)
@pytest.mark.parametrize("rnd", FTZ_MODES)
def test_flush_to_zero_tuned_formats(E, M, rnd):
    """Seeded values of the workload recipe, uniform encodings, and operands
    whose exponent fields sit at the bottom of the range (subnormal operands,
    tiny products and sums), in every compiled launch variant."""
    n = 60_000 + 7
    B = 1 + E + M
    r = synth.splitmix64(7700 + E * 32 + M, 3 * n)
    low = ((r % np.uint64(1 << (M + 1))) | ((r >> np.uint64(40)) % np.uint64(3) << np.uint64(M + 1))
           | ((r >> np.uint64(50)) & np.uint64(1)) << np.uint64(B - 1)).astype(np.uint32)
    a = np.concatenate([synth.fp_values(E, M, n, 71).astype(np.uint32), synth.uniform_bits(B, n, 72).astype(np.uint32),
                        low[:n]])
    b = np.concatenate([synth.fp_values(E, M, n, 73).astype(np.uint32), synth.uniform_bits(B, n, 74).astype(np.uint32),
                        low[n:2 * n]])
    c = np.concatenate([synth.fp_values(E, M, n, 75).astype(np.uint32), synth.uniform_bits(B, n, 76).astype(np.uint32),
                        low[2 * n:]])
    f = bs.Format(E, M, rnd)
    for op in OPS:
        for wpt in bs.bsfp_variants_compiled(f, op):
            check(op, E, M, rnd, a, b, c if op == "fma2" else None, wpt=wpt)
        bs.bsfp_set_variant(f, op, 0, 0)


def test_flush_to_zero_is_refused_where_not_compiled():
    f = bs.Format(6, 9, oracle.RN_FTZ)
    x = torch.zeros(16 * 32, dtype=torch.int32, device="cuda")
    with pytest.raises(bs.BsfpError) as ei:
        bs.bsfp_add(f, x, x, x, 10)
    assert ei.value.status == bs.ERR_UNSUPPORTED


# ------------------------------------------------------------ edge cases ---
@pytest.mark.parametrize("n", [1, 31, 32, 33, 1023, 1025, 32 * 1024 - 1, 32 * 1024 + 1])
def test_tail_lengths(n):
    E, M = 5, 7
    a, b, c = (synth.fp_values(E, M, n, s).astype(np.uint32) for s in (51, 52, 53))
    for op in OPS:
        check(op, E, M, oracle.RN, a, b, c if op == "fma2" else None)


def test_padding_written_as_zero_whatever_the_inputs_hold():
    E, M, n = 4, 4, 1000
    B = 9
    f = bs.Format(E, M)
    S = bs.bsfp_plane_stride(n)
    a = synth.fp_values(E, M, n, 61).astype(np.uint32)
    b = synth.fp_values(E, M, n, 62).astype(np.uint32)
    pa, pb = oracle.pack(B, a), oracle.pack(B, b)
    junk = synth.uniform_bits(32, B * S, 63, dtype=np.uint32).reshape(B, S)
    nw = (n + 31) // 32
    tail = np.uint32((1 << (n % 32)) - 1)
    for p in (pa, pb):
        p[:, nw:] = junk[:, nw:]
        p[:, nw - 1] |= junk[:, nw - 1] & ~tail
    for op in ("add", "mul"):
        out = torch.full((B * S,), -1, dtype=torch.int32, device="cuda")
        bs.bsfp_op(op, f, dev(pa), dev(pb), out, n)
        got = host_u32(out).reshape(B, S)
        assert (got == oracle.pack(B, oracle.binop(op, E, M, 0, a, b))).all()


def test_output_may_alias_an_input():
    E, M, n = 5, 10, 77777
    B = 16
    f = bs.Format(E, M)
    a = synth.fp_values(E, M, n, 71).astype(np.uint32)
    b = synth.fp_values(E, M, n, 72).astype(np.uint32)
    for op in ("add", "sub", "mul"):
        ta, tb = dev(oracle.pack(B, a)), dev(oracle.pack(B, b))
        bs.bsfp_op(op, f, ta, tb, ta, n)
        assert (host_u32(ta).reshape(B, -1) == want_planes(op, E, M, 0, a, b)).all(), op


def test_empty_vector_launches_nothing():
    before = bs.bsfp_launch_count()
    f = bs.Format(5, 7)
    t = torch.zeros(64, dtype=torch.int32, device="cuda")
    for op in ("add", "sub", "mul"):
        bs.bsfp_op(op, f, t, t, t, 0)
    bs.bsfp_pack(f, t, 0, t)
    assert bs.bsfp_launch_count() == before


def test_streams_are_respected():
    E, M, n = 5, 7, 1 << 20
    B = 13
    f = bs.Format(E, M)
    a = synth.fp_values(E, M, n, 81).astype(np.uint32)
    b = synth.fp_values(E, M, n, 82).astype(np.uint32)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ta, tb = dev(oracle.pack(B, a)), dev(oracle.pack(B, b))
        out = torch.empty_like(ta)
        bs.bsfp_mul(f, ta, tb, out, n, stream=s)
    s.synchronize()
    assert (host_u32(out).reshape(B, -1) == want_planes("mul", E, M, 0, a, b)).all()


# ---------------------------------------------------- input generator ---
@pytest.mark.parametrize("E,M", [(4, 3), (4, 4), (5, 7), (8, 23), (3, 2)])
def test_device_generator_matches_host(E, M):
    f = bs.Format(E, M)
    n, start = 100_003, 12345
    out = bs.empty_standard(f, n)
    bs.bsfp_synth_fp_values(f, n, 1602, 3, start, out)
    cdt = {1: np.uint8, 2: np.uint16, 4: np.uint32}[bs.bsfp_container_bytes(f)]
    got = out.cpu().numpy().view(cdt)
    assert (got == synth.fp_values(E, M, n, 1602, 3, start, dtype=cdt)).all()


def test_lop3_probe_runs():
    sink = torch.zeros(4 * 256, dtype=torch.int32, device="cuda")
    bs.bsfp_lop3_probe(sink, 4, 256, 10)
    torch.cuda.synchronize()
    assert int((sink != 0).sum()) > 0


# ------------------------------------------------- full size, every output ---
@pytest.mark.parametrize("E,M", [(4, 4), (5, 7)])
def test_full_size_2_28_every_output(E, M):
    """The benchmark's workload: 2^28 elements generated on the device, packed,
    added and multiplied with the launch shapes the benchmark uses; every one
    of the 2^28 outputs of each op against the oracle, whose inputs come from
    the host generator (in chunks of 2^26 elements)."""
    from bench import apply_tuning
    apply_tuning()
    n = 1 << 28
    chunk = 1 << 26
    f = bs.Format(E, M)
    std = bs.empty_standard(f, n)
    planes = []
    for seed in (synth.SEED_A, synth.SEED_B):
        bs.bsfp_synth_fp_values(f, n, seed, 0, 0, std)
        p = bs.empty_bitslice(f, n)
        bs.bsfp_pack(f, std, n, p)
        planes.append(p)
    out = bs.empty_bitslice(f, n)
    cdt = np.uint16
    got = {}
    for op in ("add", "mul"):
        bs.bsfp_op(op, f, planes[0], planes[1], out, n)
        bs.bsfp_unpack(f, out, n, std)
        got[op] = std.cpu().numpy().view(cdt)
    del planes, out, std
    torch.cuda.empty_cache()
    for start in range(0, n, chunk):
        xa = synth.fp_values(E, M, chunk, synth.SEED_A, 0, start).astype(np.uint32)
        xb = synth.fp_values(E, M, chunk, synth.SEED_B, 0, start).astype(np.uint32)
        for op in ("add", "mul"):
            want = oracle.binop(op, E, M, 0, xa, xb)
            g = got[op][start:start + chunk].astype(np.uint32)
            bad = np.nonzero(g != want)[0]
            assert not len(bad), "%s: %d bad, first idx %d" % (op, len(bad), start + bad[0])


def test_native_autotune_applies_and_records_a_shape(tmp_path):
    f = bs.Format(5, 7, oracle.RN)
    cache = tmp_path / "shapes.txt"
    bs.bsfp_autotune(f, "mul", str(cache))
    lines = [l.split() for l in cache.read_text().splitlines() if not l.startswith("#")]
    assert len(lines) == 1 and lines[0][:4] == ["5", "7", "0", "2"]
    assert bs.bsfp_variant(f, "mul") == int(lines[0][4])
    n = 70_001
    a, b = (synth.fp_values(5, 7, n, s).astype(np.uint32) for s in (81, 82))
    check("mul", 5, 7, oracle.RN, a, b)          # results do not depend on the shape
    bs.bsfp_autotune(f, "add", str(cache))       # a second entry is appended, the first kept
    lines = [l.split() for l in cache.read_text().splitlines() if not l.startswith("#")]
    assert sorted(l[3] for l in lines) == ["0", "2"]
    bs.bsfp_set_variant(f, "mul", 0, 0)
    bs.bsfp_set_variant(f, "add", 0, 0)


# ------------------------------------------------------- guard words ---
def test_no_kernel_writes_outside_its_output():
    """Every kernel family writes into a buffer framed by 4 KiB of guard words
    on each side (compute-sanitizer is closed on this machine): the guards must
    come back untouched and the payload must match the oracle."""
    G = 1024   # guard words on each side
    pat = np.int32(0x5A5A5A5A)

    def framed(words):
        t = torch.full((words + 2 * G,), int(pat), dtype=torch.int32, device="cuda")
        return t, t[G:G + words]

    def guards_ok(t, words):
        h = t.cpu().numpy()
        return (h[:G] == pat).all() and (h[G + words:] == pat).all()

    for E, M, n in ((5, 7, 1000), (4, 3, 33), (8, 23, 4097), (6, 9, 70001)):
        B = 1 + E + M
        S = bs.bsfp_plane_stride(n)
        a, b = (synth.fp_values(E, M, n, s).astype(np.uint32) for s in (91, 92))
        pa, pb = dev(oracle.pack(B, a)), dev(oracle.pack(B, b))
        for op in ("add", "mul", "div"):
            t, out = framed(B * S)
            bs.bsfp_op(op, bs.Format(E, M), pa, pb, out, n)
            torch.cuda.synchronize()
            assert guards_ok(t, B * S), "%s 1/%d/%d wrote outside" % (op, E, M)
        std_words = (n * bs.bsfp_container_bytes(bs.Format(E, M)) + 3) // 4
        t, out = framed(std_words)
        bs.bsfp_unpack(bs.Format(E, M), pa, n, out)
        torch.cuda.synchronize()
        assert guards_ok(t, std_words), "unpack 1/%d/%d wrote outside" % (E, M)
        t, out = framed(n)
        bs.bsfp_to_float(bs.Format(E, M), pa, n, out)
        torch.cuda.synchronize()
        assert guards_ok(t, n), "to_float 1/%d/%d wrote outside" % (E, M)
        src = torch.zeros(n, dtype=torch.float32, device="cuda")
        t, out = framed(B * S)
        bs.bsfp_from_float(bs.Format(E, M), src, n, out)
        torch.cuda.synchronize()
        assert guards_ok(t, B * S), "from_float 1/%d/%d wrote outside" % (E, M)
    for w, n in ((5, 100), (13, 4097), (32, 33)):
        S = bs.bsfp_plane_stride(n)
        x = torch.zeros(w * S, dtype=torch.int32, device="cuda")
        t, out = framed(w * S)
        bs.bsfp_int_op("mul", w, x, x, out, n)
        torch.cuda.synchronize()
        assert guards_ok(t, w * S), "int mul w=%d wrote outside" % w
