"""The README's example runs as written and its results are the oracle's."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
import paper_1602_04716_gb300 as bs  # noqa: E402

pytestmark = pytest.mark.gpu


def test_readme_example():
    torch.manual_seed(0)
    f = bs.Format(5, 7, bs.RN)
    x = torch.randn(1 << 20, device="cuda")
    a, b, out = (bs.empty_bitslice(f, x.numel()) for _ in range(3))
    bs.bsfp_from_float(f, x, x.numel(), a)
    bs.bsfp_from_float(f, x * 3, x.numel(), b)
    bs.bsfp_mul(f, a, b, out, x.numel())
    y = torch.empty_like(x)
    bs.bsfp_to_float(f, out, x.numel(), y)
    torch.cuda.synchronize()
    xs = x.cpu().numpy().view(np.uint32)
    x3 = (x * 3).cpu().numpy().view(np.uint32)
    ca, cb = oracle.from_f32(5, 7, 0, xs), oracle.from_f32(5, 7, 0, x3)
    want = oracle.to_f32(5, 7, 0, oracle.binop("mul", 5, 7, 0, ca, cb))
    assert (y.cpu().numpy().view(np.uint32) == want).all()
