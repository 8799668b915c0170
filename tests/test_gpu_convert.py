"""The fused float conversions on the GPU, bit for bit against the oracle:
binary32 / bfloat16 / binary16 arrays straight to bitslice planes of a
format (one rounding, every mode), and bitslice planes back to binary32
(exact), at ragged lengths, with subnormals, overflow, NaN and Inf among the
inputs; padding planes must come out zero."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_1602_04716_gb300 as bs  # noqa: E402

pytestmark = pytest.mark.gpu

TUNED = [(4, 3), (4, 4), (5, 7), (5, 10), (8, 7), (8, 23)]
OTHER = [(2, 1), (3, 2), (6, 9), (7, 13), (3, 23), (8, 1)]


def _f32_inputs(n, seed):
    r = synth.splitmix64(seed, 3 * n)
    near = ((r[n:2 * n] & np.uint64(0x807FFFFF)) | ((np.uint64(96) + r[2 * n:] % np.uint64(48)) << np.uint64(23)))
    spec = np.array([0, 0x80000000, 0x7F800000, 0xFF800000, 0x7FC00000, 0x7F800001, 0x00000001, 0x007FFFFF,
                     0x00800000, 0x7F7FFFFF, 0x3F800000, 0x477FF000, 0x477FF001], np.uint32)
    x = np.concatenate([r[:n].astype(np.uint32), near.astype(np.uint32),
                        (r[2 * n:] & np.uint64(0x807FFFFF)).astype(np.uint32), spec])
    return x[: 3 * n + 7]     # a ragged length


def _as_f32_bits(x, src):
    """The binary32 bit patterns a 16-bit source holds exactly."""
    if src == bs.BFLOAT16:
        return (x >> 16) << 16
    if src == bs.FLOAT16:
        h = (x >> 16).astype(np.uint16)
        return h.view(np.float16).astype(np.float32).view(np.uint32)
    return x


def _dev_src(x, src):
    if src == bs.FLOAT32:
        return torch.from_numpy(x.view(np.float32).copy()).cuda()
    h = (x >> 16).astype(np.uint16).view(np.int16).copy()
    t = torch.from_numpy(h).cuda()
    return t.view(torch.bfloat16 if src == bs.BFLOAT16 else torch.float16)


@pytest.mark.parametrize("E,M", TUNED + OTHER)
def test_from_float_matches_oracle(E, M):
    B = 1 + E + M
    x = _f32_inputs(20_000, 500 + 32 * E + M)
    n = x.size
    modes = (0, 1, 2, 3) if (E, M) in TUNED else (0, 1)
    for src in (bs.FLOAT32, bs.BFLOAT16, bs.FLOAT16):
        xs = _as_f32_bits(x, src)
        d = _dev_src(x, src)
        for rnd in modes:
            f = bs.Format(E, M, rnd)
            out = torch.full((B * bs.bsfp_plane_stride(n),), -1, dtype=torch.int32, device="cuda")
            bs.bsfp_from_float(f, d, n, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy().view(np.uint32).reshape(B, -1)
            want = oracle.pack(B, oracle.from_f32(E, M, rnd, xs))
            if not (got == want).all():
                g = oracle.unpack(B, got, n)
                w = oracle.unpack(B, want, n)
                bad = np.nonzero(g != w)[0]
                raise AssertionError("1/%d/%d rnd=%d src=%d: %d bad, first x=%#x got %#x want %#x" % (
                    E, M, rnd, src, len(bad), xs[bad[0]] if len(bad) else 0, g[bad[0]] if len(bad) else 0,
                    w[bad[0]] if len(bad) else 0))


@pytest.mark.parametrize("E,M", TUNED + OTHER)
def test_to_float_matches_oracle(E, M):
    B = 1 + E + M
    n = 70_001
    x = np.concatenate([synth.uniform_bits(B, n, 600 + M).astype(np.uint32),
                        synth.fp_values(E, M, n, 601 + M).astype(np.uint32)])
    planes = torch.from_numpy(oracle.pack(B, x).view(np.int32).copy()).cuda()
    for rnd in ((0, 2) if (E, M) in TUNED else (0,)):
        out = torch.full((x.size,), -1, dtype=torch.int32, device="cuda")
        bs.bsfp_to_float(bs.Format(E, M, rnd), planes, x.size, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        want = oracle.to_f32(E, M, rnd, x)
        bad = np.nonzero(got != want)[0]
        assert not len(bad), "1/%d/%d rnd=%d: first x=%#x got %#x want %#x" % (E, M, rnd, x[bad[0]], got[bad[0]],
                                                                             want[bad[0]])


@pytest.mark.parametrize("E,M", [(5, 7), (4, 3), (8, 23)])
def test_conversions_of_arrays_not_16_byte_aligned(E, M):
    """Source and destination float arrays one element past a 16-byte
    boundary take the element-by-element path of every tile: same results as
    the oracle, and to_float writes exactly n values."""
    B = 1 + E + M
    x = _f32_inputs(3000, 700 + E * 32 + M)
    n = x.size
    f = bs.Format(E, M, 0)
    for src in (bs.FLOAT32, bs.BFLOAT16, bs.FLOAT16):
        xs = _as_f32_bits(x, src)
        d = _dev_src(x, src)
        base = torch.zeros(n + 8, dtype=d.dtype, device="cuda")
        base[1:n + 1] = d
        out = torch.full((B * bs.bsfp_plane_stride(n),), -1, dtype=torch.int32, device="cuda")
        bs.bsfp_from_float(f, base[1:n + 1], n, out)
        got = out.cpu().numpy().view(np.uint32).reshape(B, -1)
        assert (got == oracle.pack(B, oracle.from_f32(E, M, 0, xs))).all(), "src=%d" % src
    planes = torch.from_numpy(oracle.pack(B, synth.fp_values(E, M, n, 9).astype(np.uint32)).view(np.int32).copy()).cuda()
    guard = torch.full((n + 8,), 7, dtype=torch.int32, device="cuda")
    bs.bsfp_to_float(f, planes, n, guard[1:n + 1])
    g = guard.cpu().numpy().view(np.uint32)
    assert (g[1:n + 1] == oracle.to_f32(E, M, 0, synth.fp_values(E, M, n, 9).astype(np.uint32))).all()
    assert g[0] == 7 and (g[n + 1:] == 7).all()


def test_round_trip_at_scale():
    """2^24 + 5 binary32 values -> 1/5/10 -> binary32 equals numpy's
    binary32 -> binary16 -> binary32 (round to nearest even)."""
    n = (1 << 24) + 5
    x = synth.splitmix64(77, n).astype(np.uint32)
    f = bs.Format(5, 10, 0)
    d = torch.from_numpy(x.view(np.float32).copy()).cuda()
    planes = torch.empty(16 * bs.bsfp_plane_stride(n), dtype=torch.int32, device="cuda")
    back = torch.empty(n, dtype=torch.float32, device="cuda")
    bs.bsfp_from_float(f, d, n, planes)
    bs.bsfp_to_float(f, planes, n, back)
    torch.cuda.synchronize()
    with np.errstate(all="ignore"):
        want = x.view(np.float32).astype(np.float16).astype(np.float32)
    got = back.cpu().numpy()
    nan = np.isnan(want)
    assert (np.isnan(got) == nan).all()
    assert (got.view(np.uint32)[~nan] == want.view(np.uint32)[~nan]).all()


def test_conversion_errors():
    x = torch.zeros(64, dtype=torch.float32, device="cuda")
    p = torch.zeros(32 * 32, dtype=torch.int32, device="cuda")
    with pytest.raises(bs.BsfpError) as ei:
        bs.bsfp_from_float(bs.Format(5, 7), x, 64, p, src_type=3)
    assert ei.value.status == bs.ERR_UNSUPPORTED
    with pytest.raises(bs.BsfpError) as ei:
        bs.bsfp_from_float(bs.Format(6, 9, bs.RN_FTZ), x, 64, p)
    assert ei.value.status == bs.ERR_UNSUPPORTED
    with pytest.raises(bs.BsfpError) as ei:
        bs.bsfp_from_float(bs.Format(5, 7), x.data_ptr() + 2, 8, p, src_type=bs.FLOAT32)
    assert ei.value.status == bs.ERR_ALIGN
