"""Parity of the streamed kernels (variant BSFP_VARIANT_STREAMED: a producer
warp brings the operands' planes into a shared-memory ring with TMA bulk
copies; consumer warps run the circuits from it) through the C ABI.

The circuits are those of the grid-stride kernels; what is new is the data
movement -- tiles of TW word columns handed to blocks round-robin, a ring of
NST stages per block, bounded mbarrier waits.  So the cases are chosen by
tile geometry: sizes inside one tile, on both sides of a tile boundary, with
a ragged last tile; and sizes at which every block goes round its ring
several times.  Small sizes are compared with the oracle element by element
(whole plane buffers, padding included); the large ones bit for bit with the
grid-stride kernel over whole plane buffers and with the oracle on sampled
elements.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_1602_04716_gb300 as bs  # noqa: E402

pytestmark = pytest.mark.gpu

STREAM_FORMATS = [(4, 3), (4, 4), (5, 7), (5, 10), (8, 7)]
MODES = [oracle.RN, oracle.RZ, oracle.RN_FTZ, oracle.RZ_FTZ]
OPS = ["add", "sub", "mul", "div"]


def shape(E, M, op="add"):
    """(tile words per plane, ring stages) of the streamed kernel."""
    return bs.bsfp_stream_shape(bs.Format(E, M), op)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    bs.bsfp_fault_status(clear=True)
    bs.bsfp_set_stream_min_tiles(0)   # take the streamed kernel at every size
    yield
    bs.bsfp_set_stream_min_tiles(2)
    torch.cuda.synchronize()
    for E, M in STREAM_FORMATS:
        for rnd in MODES:
            for op in OPS + ["fma2"]:
                bs.bsfp_set_variant(bs.Format(E, M, rnd), op, 0, 0)


def dev(x: np.ndarray):
    x = np.ascontiguousarray(x)
    view = {1: np.uint8, 2: np.int16, 4: np.int32}[x.dtype.itemsize]
    return torch.from_numpy(x.view(view).copy()).cuda()


def test_streamed_variant_is_compiled_where_documented():
    for E, M in STREAM_FORMATS:
        for rnd in MODES:
            f = bs.Format(E, M, rnd)
            for op in OPS:
                assert bs.VARIANT_STREAMED in bs.bsfp_variants_compiled(f, op), (E, M, rnd, op)
            assert (bs.VARIANT_STREAMED in bs.bsfp_variants_compiled(f, "fma2")) == (1 + E + M >= 10)
    for E, M in [(8, 23), (3, 2)]:
        for op in ("mul", "fma2", "div"):
            assert bs.VARIANT_STREAMED not in bs.bsfp_variants_compiled(bs.Format(E, M), op)
    # outside the tuned set (RN, RZ): the streamed mul for 12..24 planes, fma2 for 10..19 and division
    # for 8..24, no streamed add
    assert bs.VARIANT_STREAMED in bs.bsfp_variants_compiled(bs.Format(6, 9, 1), "mul")
    assert bs.VARIANT_STREAMED in bs.bsfp_variants_compiled(bs.Format(6, 9, 1), "fma2")
    assert bs.VARIANT_STREAMED in bs.bsfp_variants_compiled(bs.Format(6, 9, 1), "div")
    assert bs.VARIANT_STREAMED not in bs.bsfp_variants_compiled(bs.Format(6, 9), "add")
    with pytest.raises(bs.BsfpError):
        bs.bsfp_set_variant(bs.Format(6, 9), "add", bs.VARIANT_STREAMED)
    with pytest.raises(bs.BsfpError):
        bs.bsfp_set_variant(bs.Format(3, 2), "mul", bs.VARIANT_STREAMED)


@pytest.mark.parametrize("E,M", STREAM_FORMATS)
@pytest.mark.parametrize("rnd", MODES)
def test_tile_geometry_vs_oracle(E, M, rnd):
    """n inside the first tile, either side of the first tile boundary, and
    three tiles plus a ragged tail; every word of every output plane
    (padding included) against the oracle."""
    B = 1 + E + M
    f = bs.Format(E, M, rnd)
    sizes = sorted({m for op in OPS for TW in [shape(E, M, op)[0]]
                    for m in (1, 33, 32 * TW - 1, 32 * TW + 1, 3 * 32 * TW + 77)})
    for n in sizes:
        a = synth.fp_values(E, M, n, 501 + n % 7).astype(np.uint32)
        b = synth.fp_values(E, M, n, 601 + n % 5).astype(np.uint32)
        pa, pb = dev(oracle.pack(B, a)), dev(oracle.pack(B, b))
        for op in OPS:
            bs.bsfp_set_variant(f, op, bs.VARIANT_STREAMED)
            assert bs.bsfp_variant(f, op) == bs.VARIANT_STREAMED
            out = torch.full_like(pa, -1)
            bs.bsfp_op(op, f, pa, pb, out, n)
            got = out.cpu().numpy().view(np.uint32).reshape(B, -1)
            want = oracle.pack(B, oracle.binop(op, E, M, rnd, a, b))
            assert (got == want).all(), "%s 1/%d/%d rnd=%d n=%d" % (op, E, M, rnd, n)
    assert bs.bsfp_fault_status() == 0


@pytest.mark.parametrize("E,M", STREAM_FORMATS)
def test_several_rounds_of_the_ring(E, M):
    """Every block takes NST + 2 tiles (the refill path of the ring) and the
    last tile is ragged: the streamed and grid-stride kernels agree on every
    word of the output planes, and 4,096 sampled elements plus the tail agree
    with the oracle, in all four modes."""
    B = 1 + E + M
    # every op class gets NST + 2 tiles per block or more
    TW, NST = max((shape(E, M, op) for op in ("add", "mul", "div")), key=lambda s: s[0] * (s[1] + 2))
    n = bs.bsfp_num_sms() * (NST + 2) * 32 * TW - 3 * 32 * TW // 2 + 12345
    cdt = {1: np.uint8, 2: np.uint16, 4: np.uint32}[bs.bsfp_container_bytes(bs.Format(E, M))]
    std = bs.empty_standard(bs.Format(E, M), n)
    planes = []
    for seed in (7001, 7002):
        bs.bsfp_synth_fp_values(bs.Format(E, M), n, seed, 0, 0, std)
        p = bs.empty_bitslice(bs.Format(E, M), n)
        bs.bsfp_pack(bs.Format(E, M), std, n, p)
        planes.append(p)
    rng = np.random.default_rng(E * 64 + M)
    idx = np.unique(np.concatenate([rng.integers(0, n, 4096), np.arange(n - 64, n)])).astype(np.int64)
    xa = synth.fp_values_at(E, M, idx, 7001)
    xb = synth.fp_values_at(E, M, idx, 7002)
    idx_t = torch.from_numpy(idx).cuda()
    ref = bs.empty_bitslice(bs.Format(E, M), n)
    got = bs.empty_bitslice(bs.Format(E, M), n)
    for rnd in MODES:
        f = bs.Format(E, M, rnd)
        for op in OPS:
            bs.bsfp_set_variant(f, op, bs.bsfp_variants_compiled(f, op)[0])
            bs.bsfp_op(op, f, planes[0], planes[1], ref, n)
            bs.bsfp_set_variant(f, op, bs.VARIANT_STREAMED)
            got.fill_(-1)
            bs.bsfp_op(op, f, planes[0], planes[1], got, n)
            assert torch.equal(got, ref), "%s 1/%d/%d rnd=%d: streamed != grid-stride" % (op, E, M, rnd)
            bs.bsfp_unpack(f, got, n, std)
            res = std[idx_t].cpu().numpy().view(cdt).astype(np.uint32)
            want = oracle.binop(op, E, M, rnd, xa, xb)
            bad = np.nonzero(res != want)[0]
            assert not len(bad), "%s 1/%d/%d rnd=%d: %d bad, first idx %d" % (op, E, M, rnd, len(bad), idx[bad[0]])
    assert bs.bsfp_fault_status() == 0
    del planes, ref, got, std
    torch.cuda.empty_cache()


FMA2_STREAM_FORMATS = [(E, M) for E, M in STREAM_FORMATS if 1 + E + M >= 10]


@pytest.mark.parametrize("E,M", FMA2_STREAM_FORMATS)
@pytest.mark.parametrize("rnd", MODES)
def test_streamed_fma2_tile_geometry_vs_oracle(E, M, rnd):
    """The streamed fma2 (product first, then the addend: from the ring up to
    13 planes, from global memory beyond) at the tile-geometry sizes, every
    word of the output planes against the oracle, in all four modes."""
    B = 1 + E + M
    f = bs.Format(E, M, rnd)
    TW, _ = shape(E, M, "fma2")
    for n in (1, 33, 32 * TW - 1, 32 * TW + 1, 3 * 32 * TW + 77):
        a, b, c = (synth.fp_values(E, M, n, seed + n % 7).astype(np.uint32) for seed in (811, 822, 833))
        pa, pb, pc = dev(oracle.pack(B, a)), dev(oracle.pack(B, b)), dev(oracle.pack(B, c))
        bs.bsfp_set_variant(f, "fma2", bs.VARIANT_STREAMED)
        out = torch.full_like(pa, -1)
        bs.bsfp_fma2(f, pa, pb, pc, out, n)
        got = out.cpu().numpy().view(np.uint32).reshape(B, -1)
        want = oracle.pack(B, oracle.fma2(E, M, rnd, a, b, c))
        assert (got == want).all(), "fma2 1/%d/%d rnd=%d n=%d" % (E, M, rnd, n)
    bs.bsfp_set_variant(f, "fma2", 0, 0)
    assert bs.bsfp_fault_status() == 0


@pytest.mark.parametrize("E,M", FMA2_STREAM_FORMATS)
def test_streamed_fma2_several_rounds_of_the_ring(E, M):
    """NST + 2 tiles per block and a ragged last tile: streamed and
    grid-stride fma2 agree on every word of the output planes in all four
    modes, and sampled elements plus the tail agree with the oracle."""
    B = 1 + E + M
    TW, NST = shape(E, M, "fma2")
    n = bs.bsfp_num_sms() * (NST + 2) * 32 * TW - 3 * 32 * TW // 2 + 4321
    cdt = {1: np.uint8, 2: np.uint16, 4: np.uint32}[bs.bsfp_container_bytes(bs.Format(E, M))]
    std = bs.empty_standard(bs.Format(E, M), n)
    planes = []
    for seed in (7101, 7102, 7103):
        bs.bsfp_synth_fp_values(bs.Format(E, M), n, seed, 0, 0, std)
        p = bs.empty_bitslice(bs.Format(E, M), n)
        bs.bsfp_pack(bs.Format(E, M), std, n, p)
        planes.append(p)
    rng = np.random.default_rng(E * 64 + M + 1)
    idx = np.unique(np.concatenate([rng.integers(0, n, 4096), np.arange(n - 64, n)])).astype(np.int64)
    xs = [synth.fp_values_at(E, M, idx, seed) for seed in (7101, 7102, 7103)]
    idx_t = torch.from_numpy(idx).cuda()
    ref = bs.empty_bitslice(bs.Format(E, M), n)
    got = bs.empty_bitslice(bs.Format(E, M), n)
    for rnd in MODES:
        f = bs.Format(E, M, rnd)
        bs.bsfp_set_variant(f, "fma2", bs.bsfp_variants_compiled(f, "fma2")[0])
        bs.bsfp_fma2(f, planes[0], planes[1], planes[2], ref, n)
        bs.bsfp_set_variant(f, "fma2", bs.VARIANT_STREAMED)
        got.fill_(-1)
        bs.bsfp_fma2(f, planes[0], planes[1], planes[2], got, n)
        bs.bsfp_set_variant(f, "fma2", 0, 0)
        assert torch.equal(got, ref), "fma2 1/%d/%d rnd=%d: streamed != grid-stride" % (E, M, rnd)
        bs.bsfp_unpack(f, got, n, std)
        res = std[idx_t].cpu().numpy().view(cdt).astype(np.uint32)
        want = oracle.fma2(E, M, rnd, *xs)
        bad = np.nonzero(res != want)[0]
        assert not len(bad), "fma2 1/%d/%d rnd=%d: %d bad, first idx %d" % (E, M, rnd, len(bad), idx[bad[0]])
    assert bs.bsfp_fault_status() == 0
    del planes, ref, got, std
    torch.cuda.empty_cache()


@pytest.mark.parametrize("E,M,op", [(4, 4, "add"), (4, 4, "mul"), (5, 7, "add"), (5, 7, "mul"), (5, 7, "div"),
                                     (5, 7, "fma2"), (8, 7, "fma2"), (6, 9, "div")])
def test_uneven_rounds_of_tiles(E, M, op):
    """2.4 tiles per block: some blocks take three tiles and others two, and
    the last tile is ragged.  For the adder, the multiplier, the divider and
    fma2 (with the addend in the ring and from global memory): streamed
    against grid-stride on every word of the output planes (RN and RZ), and
    sampled elements against the oracle."""
    B = 1 + E + M
    TW, _ = shape(E, M, op)
    n = int(2.4 * bs.bsfp_num_sms() * 32 * TW) + 333
    f0 = bs.Format(E, M)
    planes = []
    std = bs.empty_standard(f0, n)
    for seed in (7301, 7302, 7303):
        bs.bsfp_synth_fp_values(f0, n, seed, 0, 0, std)
        p = bs.empty_bitslice(f0, n)
        bs.bsfp_pack(f0, std, n, p)
        planes.append(p)
    cdt = {1: np.uint8, 2: np.uint16, 4: np.uint32}[bs.bsfp_container_bytes(f0)]
    rng = np.random.default_rng(B * 7 + len(op))
    idx = np.unique(np.concatenate([rng.integers(0, n, 2048), np.arange(n - 40, n)])).astype(np.int64)
    xs = [synth.fp_values_at(E, M, idx, seed) for seed in (7301, 7302, 7303)]
    idx_t = torch.from_numpy(idx).cuda()
    ref = bs.empty_bitslice(f0, n)
    got = bs.empty_bitslice(f0, n)
    for rnd in (0, 1):
        f = bs.Format(E, M, rnd)
        c = planes[2] if op == "fma2" else None
        bs.bsfp_set_variant(f, op, bs.bsfp_variants_compiled(f, op)[0])
        bs.bsfp_op(op, f, planes[0], planes[1], ref, n, c=c)
        bs.bsfp_set_variant(f, op, bs.VARIANT_STREAMED)
        assert bs.bsfp_variant_for(f, op, n) == bs.VARIANT_STREAMED
        got.fill_(-1)
        bs.bsfp_op(op, f, planes[0], planes[1], got, n, c=c)
        bs.bsfp_set_variant(f, op, 0, 0)
        assert torch.equal(got, ref), "%s 1/%d/%d rnd=%d: streamed != grid-stride" % (op, E, M, rnd)
        bs.bsfp_unpack(f, got, n, std)
        res = std[idx_t].cpu().numpy().view(cdt).astype(np.uint32)
        want = oracle.binop(op, E, M, rnd, xs[0], xs[1], xs[2])
        bad = np.nonzero(res != want)[0]
        assert not len(bad), "%s 1/%d/%d rnd=%d: %d bad, first idx %d" % (op, E, M, rnd, len(bad), idx[bad[0]])
    assert bs.bsfp_fault_status() == 0
    del planes, ref, got, std
    torch.cuda.empty_cache()


def test_streamed_writes_nothing_outside_its_output():
    """Guard words of 4 KiB on both sides of the output planes survive a
    streamed launch whose last tile is ragged."""
    E, M = 5, 7
    B = 1 + E + M
    f = bs.Format(E, M)
    TW, _ = shape(E, M)
    n = 5 * 32 * TW + 1000
    S = bs.bsfp_plane_stride(n)
    a = synth.fp_values(E, M, n, 11).astype(np.uint32)
    b = synth.fp_values(E, M, n, 12).astype(np.uint32)
    pa, pb = dev(oracle.pack(B, a)), dev(oracle.pack(B, b))
    G = 1024
    buf = torch.full((B * S + 2 * G,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    out = buf[G:G + B * S]
    for op in OPS:
        bs.bsfp_set_variant(f, op, bs.VARIANT_STREAMED)
        bs.bsfp_op(op, f, pa, pb, out, n)
        torch.cuda.synchronize()
        assert bool((buf[:G] == 0x5A5A5A5A).all()) and bool((buf[G + B * S:] == 0x5A5A5A5A).all()), op
        want = oracle.pack(B, oracle.binop(op, E, M, 0, a, b))
        assert (out.cpu().numpy().view(np.uint32).reshape(B, -1) == want).all(), op


def test_fault_word_is_clear_after_the_streamed_runs():
    assert bs.bsfp_fault_status(clear=True) == 0
    assert bs.bsfp_fault_status() == 0


def test_small_calls_fall_back_to_the_grid_stride_kernel():
    """With the default threshold (2 tiles per SM) a call too small to fill
    the ring runs the default grid-stride variant; results do not change."""
    E, M = 5, 7
    f = bs.Format(E, M)
    TW, _ = shape(E, M, "mul")
    sms = bs.bsfp_num_sms()
    bs.bsfp_set_variant(f, "mul", bs.VARIANT_STREAMED)
    try:
        bs.bsfp_set_stream_min_tiles(2)
        small, big = 32 * TW * sms, 2 * 32 * TW * sms
        assert bs.bsfp_variant_for(f, "mul", small) not in (bs.VARIANT_STREAMED, 0, -1)
        assert bs.bsfp_variant_for(f, "mul", big) == bs.VARIANT_STREAMED
        bs.bsfp_set_stream_min_tiles(0)
        assert bs.bsfp_variant_for(f, "mul", 1) == bs.VARIANT_STREAMED
    finally:
        bs.bsfp_set_stream_min_tiles(0)
        bs.bsfp_set_variant(f, "mul", 0, 0)


def test_bounded_wait_runs_out_and_reports():
    """The failure path of the streamed kernel's waits: the copies of one tile
    are withheld and the waits are bounded at 2^22 cycles (about 2 ms), so
    the waits on that tile run out.  The block stops, the fault word becomes
    1, the device stays usable, and the next normal call is exact."""
    E, M = 5, 7
    B = 1 + E + M
    f = bs.Format(E, M)
    TW, NST = shape(E, M, "mul")
    n = bs.bsfp_num_sms() * (NST + 2) * 32 * TW
    a = torch.zeros(B * bs.bsfp_plane_stride(n), dtype=torch.int32, device="cuda")
    b = torch.zeros_like(a)
    out = torch.zeros_like(a)
    assert bs.bsfp_fault_status(clear=True) == 0
    tiles = (bs.bsfp_plane_stride(n) + TW - 1) // TW
    with pytest.raises(bs.BsfpError):
        bs.bsfp_stream_selftest(f, "mul", a, b, out, n, tiles, 1 << 22)    # tile out of range
    with pytest.raises(bs.BsfpError):
        bs.bsfp_stream_selftest(f, "fma2", a, b, out, n, 0, 1 << 22)       # add/sub and mul only
    bs.bsfp_stream_selftest(f, "mul", a, b, out, n, -1, 1 << 22)           # nothing withheld
    assert bs.bsfp_fault_status() == 0
    bs.bsfp_stream_selftest(f, "mul", a, b, out, n, tiles // 2, 1 << 22)
    assert bs.bsfp_fault_status(clear=True) == 1
    assert bs.bsfp_fault_status() == 0
    # the context still computes: a normal streamed call, exact against the oracle
    m = 3 * 32 * TW + 5
    x = synth.fp_values(E, M, m, 91).astype(np.uint32)
    y = synth.fp_values(E, M, m, 92).astype(np.uint32)
    px, py = dev(oracle.pack(B, x)), dev(oracle.pack(B, y))
    o = torch.full_like(px, -1)
    bs.bsfp_set_variant(f, "mul", bs.VARIANT_STREAMED)
    bs.bsfp_mul(f, px, py, o, m)
    assert (o.cpu().numpy().view(np.uint32).reshape(B, -1) == oracle.pack(B, oracle.binop("mul", E, M, 0, x, y))).all()
    assert bs.bsfp_fault_status() == 0
    bs.bsfp_set_variant(f, "mul", 0, 0)


@pytest.mark.parametrize("E,M,op,alias", [(5, 7, "add", 0), (5, 7, "mul", 0), (5, 7, "div", 0), (5, 7, "mul", 1),
                                           (5, 7, "fma2", 0), (5, 7, "fma2", 2), (8, 7, "fma2", 0),
                                           (8, 7, "fma2", 2)])
def test_in_place_output(E, M, op, alias):
    """out may equal an input (the C ABI allows exact aliasing): the streamed
    kernel reads a tile into shared memory before any of its columns is
    written, and fma2 with the addend from global memory (16 planes) reads
    each thread's addend columns before it stores them, so out = a, b or c
    gives the same result as a separate output."""
    B = 1 + E + M
    f = bs.Format(E, M)
    TW, NST = shape(E, M, op)
    n = bs.bsfp_num_sms() * (NST + 1) * 32 * TW + 999
    x = [synth.fp_values(E, M, n, seed).astype(np.uint32) for seed in (61, 62, 63)]
    p = [dev(oracle.pack(B, v)) for v in x]
    bs.bsfp_set_variant(f, op, bs.VARIANT_STREAMED)
    bs.bsfp_op(op, f, p[0], p[1], p[alias], n, c=p[2] if op == "fma2" else None)
    torch.cuda.synchronize()
    bs.bsfp_set_variant(f, op, 0, 0)
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([rng.integers(0, n, 20000), np.arange(n - 100, n)]))
    got = oracle.unpack(B, p[alias].cpu().numpy().view(np.uint32), n)[idx]
    assert (got == oracle.binop(op, E, M, 0, x[0][idx], x[1][idx], x[2][idx])).all()


BANDS = {"mul": (12, 24, 1), "fma2": (10, 19, 4), "div": (8, 24, 3)}   # planes from, to; fewest fraction bits


def _streamed_band_formats(op):
    fm = []
    for E in range(2, 9):
        for M in range(1, 24):
            if 1 + E + M <= 32 and (E, M) not in STREAM_FORMATS and \
                    bs.VARIANT_STREAMED in bs.bsfp_variants_compiled(bs.Format(E, M), op):
                fm.append((E, M))
    return fm


@pytest.mark.parametrize("op", ["mul", "fma2", "div"])
def test_streamed_band_covers_its_plane_counts(op):
    """mul: the formats of 12..24 planes outside the tuned set; fma2: those
    of 10..19 planes with 4 fraction bits or more; division: those of 8..24
    planes with 3 fraction bits or more."""
    lo, hi, mlo = BANDS[op]
    fm = _streamed_band_formats(op)
    assert fm and all(lo <= 1 + E + M <= hi and M >= mlo for E, M in fm)
    assert len(fm) == sum(1 for E in range(2, 9) for M in range(1, 24)
                          if lo <= 1 + E + M <= hi and M >= mlo and (E, M) not in STREAM_FORMATS + [(8, 23)])


@pytest.mark.parametrize("op", ["mul", "fma2", "div"])
@pytest.mark.parametrize("E", range(2, 9))
def test_streamed_band_of_every_format_vs_oracle(op, E):
    """Formats outside the tuned set with a streamed mul (12..24 planes: the
    default up to 20, the autotuner's choice beyond), fma2 (10..19 planes, 4
    fraction bits or more, the default; the addend's planes in the ring up to
    13 planes, loaded from global memory beyond) or division (8..24 planes, 3 fraction bits or more:
    the default from 4).  For each of them, RN and RZ, forced
    streamed at every size: inside one tile, and three tiles plus a ragged
    tail, every word of the output planes (padding included) against the
    oracle."""
    for (e, M) in _streamed_band_formats(op):
        if e != E:
            continue
        B = 1 + E + M
        TW, _ = shape(E, M, op)
        for n in (77, 3 * 32 * TW + 77):
            a = synth.fp_values(E, M, n, 900 + M).astype(np.uint32)
            b = synth.fp_values(E, M, n, 950 + M).astype(np.uint32)
            c = synth.fp_values(E, M, n, 975 + M).astype(np.uint32)
            pa, pb, pc = dev(oracle.pack(B, a)), dev(oracle.pack(B, b)), dev(oracle.pack(B, c))
            for rnd in (0, 1):
                f = bs.Format(E, M, rnd)
                bs.bsfp_set_variant(f, op, bs.VARIANT_STREAMED)
                out = torch.full_like(pa, -1)
                if op == "fma2":
                    bs.bsfp_fma2(f, pa, pb, pc, out, n)
                else:
                    bs.bsfp_op(op, f, pa, pb, out, n)
                bs.bsfp_set_variant(f, op, 0, 0)
                got = out.cpu().numpy().view(np.uint32).reshape(B, -1)
                want = oracle.pack(B, oracle.fma2(E, M, rnd, a, b, c) if op == "fma2" else
                                   oracle.binop(op, E, M, rnd, a, b))
                assert (got == want).all(), "%s 1/%d/%d rnd=%d n=%d" % (op, E, M, rnd, n)
    assert bs.bsfp_fault_status() == 0
