"""Integer bitslice vectors (Sec. 3) on the GPU: w-bit add, sub and mul
modulo 2^w for every width 1..32, bit-exact against the oracle (every pair
for small widths, seeded samples with a ragged length otherwise), pack /
unpack at every width, and padding written as zero."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_1602_04716_gb300 as bs  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int32).copy()).cuda()


@pytest.mark.parametrize("w", range(1, 33))
def test_integer_ops_every_width(w):
    if w <= 8:
        a, b = (v.astype(np.uint32) for v in synth.all_pairs(w))
    else:
        n = 40_000 + 13
        a, b = (synth.uniform_bits(w, n, 900 + w, k).astype(np.uint32) for k in range(2))
    n = a.size
    pa, pb = _dev(oracle.pack(w, a)), _dev(oracle.pack(w, b))
    for op in ("add", "sub", "mul"):
        out = torch.full_like(pa, -1)
        bs.bsfp_int_op(op, w, pa, pb, out, n)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32).reshape(w, -1)
        want = oracle.pack(w, oracle.int_binop(op, w, a, b))
        assert (got == want).all(), "%s w=%d" % (op, w)


@pytest.mark.parametrize("w", [1, 5, 8, 9, 13, 16, 17, 31, 32])
def test_integer_pack_unpack(w):
    n = 100_003
    x = synth.uniform_bits(w, n, 950 + w).astype(np.uint32)
    cdt = synth.container_dtype(w)
    std = torch.from_numpy(x.astype(cdt).view({1: np.uint8, 2: np.int16, 4: np.int32}[np.dtype(cdt).itemsize])
                           .copy()).cuda()
    planes = torch.full((w * bs.bsfp_plane_stride(n),), -1, dtype=torch.int32, device="cuda")
    bs.bsfp_int_pack(w, std, n, planes)
    back = torch.empty_like(std)
    bs.bsfp_int_unpack(w, planes, n, back)
    torch.cuda.synchronize()
    assert (planes.cpu().numpy().view(np.uint32).reshape(w, -1) == oracle.pack(w, x)).all()
    assert torch.equal(back, std)


def test_integer_errors():
    x = torch.zeros(64, dtype=torch.int32, device="cuda")
    for bad in (0, 33):
        with pytest.raises(bs.BsfpError) as ei:
            bs.bsfp_int_op("add", bad, x, x, x, 10)
        assert ei.value.status == bs.ERR_FORMAT
