"""The host-to-host pipeline: standard arrays in host memory, every chunk
copied in, packed, run through each requested op, unpacked and copied back
over rotating streams.  Results must equal the oracle bit for bit, for
lengths that end mid-chunk and mid-word, for pageable and page-locked host
arrays, and for several ops sharing one transfer of the inputs."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_1602_04716_gb300 as bs  # noqa: E402

pytestmark = pytest.mark.gpu


def _host(E, M, n, seed, pinned):
    x = synth.fp_values(E, M, n, seed)
    if not pinned:
        return x
    t = torch.empty(n, dtype={1: torch.uint8, 2: torch.int16, 4: torch.int32}[x.itemsize], pin_memory=True)
    t.numpy()[:] = x.view(t.numpy().dtype)
    return t


def _np(x, dtype):
    return x.numpy().view(dtype) if hasattr(x, "numpy") else x


@pytest.mark.parametrize("E,M", [(4, 3), (5, 7), (8, 23), (6, 9)])
@pytest.mark.parametrize("pinned", [False, True])
def test_pipeline_matches_oracle(E, M, pinned):
    pipe = bs.Pipeline(chunk=4096, depth=3)
    dt = synth.container_dtype(1 + E + M)
    for n in (1, 1000, 4096, 4097, 50_001):
        for rnd in (0, 1):
            f = bs.Format(E, M, rnd)
            a, b, c = (_host(E, M, n, 100 * n + s, pinned) for s in (1, 2, 3))
            av, bv, cv = (_np(x, dt).astype(np.uint32) for x in (a, b, c))
            for ops in (["add", "sub", "mul", "fma2"], ["div"]):
                outs = [_host(E, M, n, 0, pinned) for _ in ops]
                pipe.run(f, ops, a, b, outs, n, c=c)
                for op, o in zip(ops, outs):
                    want = oracle.binop(op, E, M, rnd, av, bv, cv)
                    got = _np(o, dt).astype(np.uint32)
                    assert (got == want).all(), "%s 1/%d/%d rnd=%d n=%d" % (op, E, M, rnd, n)
    pipe.close()


def test_pipeline_default_chunks_and_growth():
    """A long vector in default-sized chunks, then a wider format that makes
    the pipeline grow its buffers."""
    pipe = bs.Pipeline()
    for E, M, n in ((4, 4, (1 << 24) + 12345), (8, 23, 300_000)):
        f = bs.Format(E, M, 0)
        a, b = (_host(E, M, n, s, True) for s in (7, 8))
        out = _host(E, M, n, 0, True)
        pipe.run(f, ["mul"], a, b, [out], n)
        dt = synth.container_dtype(1 + E + M)
        idx = np.unique(np.concatenate([np.arange(0, n, 9973), [n - 1]]))
        av, bv = (_np(x, dt)[idx].astype(np.uint32) for x in (a, b))
        want = oracle.binop("mul", E, M, 0, av, bv)
        assert (_np(out, dt)[idx].astype(np.uint32) == want).all()
    pipe.close()


def test_pipeline_submissions_back_to_back():
    """Several vectors of different formats, op lists and lengths submitted
    back to back and waited for once: the chunks keep rotating over the
    streams across the submissions (chunk counts not multiples of the
    depth, a buffer growth in the middle), and every result equals the
    oracle.  Then a failing submission is reported by its own return and a
    later wait is clean."""
    pipe = bs.Pipeline(chunk=4096, depth=3)
    cases = [((4, 4), 4096 * 5 + 17, ["add", "mul"]), ((5, 7), 4096 * 4 + 1, ["mul", "sub", "fma2"]),
             ((8, 23), 4096 * 2 + 300, ["div"]), ((4, 3), 999, ["add"]), ((5, 10), 4096 * 7, ["fma2", "add"])]
    keep = []
    for (E, M), n, ops in cases:
        f = bs.Format(E, M, n % 2)
        a, b, c = (_host(E, M, n, 31 * n + s, True) for s in (1, 2, 3))
        outs = [_host(E, M, n, 0, True) for _ in ops]
        pipe.submit(f, ops, a, b, outs, n, c=c)
        keep.append((E, M, n % 2, n, ops, a, b, c, outs))
    pipe.wait()
    for E, M, rnd, n, ops, a, b, c, outs in keep:
        dt = synth.container_dtype(1 + E + M)
        av, bv, cv = (_np(x, dt).astype(np.uint32) for x in (a, b, c))
        for op, o in zip(ops, outs):
            want = oracle.binop(op, E, M, rnd, av, bv, cv)
            assert (_np(o, dt).astype(np.uint32) == want).all(), "%s 1/%d/%d n=%d" % (op, E, M, n)
    x = np.zeros(10, np.uint8)
    with pytest.raises(bs.BsfpError) as ei:
        pipe.submit(bs.Format(4, 3), ["fma2"], x, x, [x.copy()], 10)   # no addend
    assert ei.value.status == bs.ERR_NULL
    pipe.wait()
    pipe.close()


def test_pipeline_validation():
    pipe = bs.Pipeline(chunk=1024, depth=2)
    f = bs.Format(4, 3)
    a = np.zeros(10, np.uint8)
    with pytest.raises(bs.BsfpError) as ei:
        pipe.run(f, [], a, a, [], 10)
    assert ei.value.status == bs.ERR_SIZE
    with pytest.raises(bs.BsfpError) as ei:
        pipe.run(f, ["fma2"], a, a, [a.copy()], 10)
    assert ei.value.status == bs.ERR_NULL
    with pytest.raises(bs.BsfpError) as ei:
        pipe.run(f, [9], a, a, [a.copy()], 10)
    assert ei.value.status == bs.ERR_UNSUPPORTED
    pipe.run(f, ["add"], a, a, [a.copy()], 0)   # n == 0: nothing to do
    pipe.close()
