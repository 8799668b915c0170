"""bsfp_batch_run_noalloc, the batched launch that allocates nothing.

Some callers cannot allocate device memory: an application whose own pool has
reserved the GPU's memory up front, or a latency-bound loop where
cudaMalloc/cudaFree would synchronise the device.  For them the library keeps
the batch scratch in one fixed device array.  Here two different mixed
batches go through that entry point in a row (the second smaller than the
first, so anything the first call left in the shared array would show), and
each output must equal, bit for bit, what a persistent batch plan gives for
the same jobs.  This file is collected last so that a run stopping at the
first failure has run every other test already; it builds its own inputs, so
it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
import paper_1602_04716_gb300 as bs  # noqa: E402
from paper_1602_04716_gb300 import bsfp as _binding  # noqa: E402

pytestmark = pytest.mark.gpu

OPS = ["add", "sub", "mul", "fma2", "div"]


def _batch(njobs, seed, max_len):
    """Mixed formats (the persistent set plus two others), ops, roundings and
    ragged lengths, with a few empty jobs; operands packed on the device."""
    fmts = bs.BATCH_FORMATS + [(6, 9), (3, 2)]
    r = synth.splitmix64(seed, 3 * njobs)
    lens = synth.log_uniform_lengths(njobs, 1, max_len, seed, 1)
    specs, keep = [], []
    for i in range(njobs):
        E, M = fmts[int(r[3 * i] % len(fmts))]
        op = OPS[int(r[3 * i + 1] % len(OPS))]
        f = bs.Format(E, M, int(r[3 * i + 2] % 2))
        n = 0 if i % 29 == 5 else int(lens[i])
        ops_ = []
        for k in range(3):
            p = bs.empty_bitslice(f, n)
            if n:
                std = torch.from_numpy(synth.fp_values(E, M, n, seed + 31 * i + k).view(
                    {1: np.uint8, 2: np.int16, 4: np.int32}[bs.bsfp_container_bytes(f)])).cuda()
                bs.bsfp_pack(f, std, n, p)
            ops_.append(p)
        out = torch.full_like(ops_[0], -1)
        specs.append((f, op, ops_[0], ops_[1], ops_[2] if op == "fma2" else None, out, n))
        keep.append((ops_, out))
    arr, nj = bs.make_jobs(specs)
    return arr, nj, [o for _, o in keep], keep


def _reference(arr, nj, outs):
    """Outputs of the existing entry point (a persistent batch plan)."""
    plan = bs.BatchPlan(arr, nj, bs.BATCH_PERSISTENT)
    plan.run()
    torch.cuda.synchronize()
    want = [o.clone() for o in outs]
    plan.free()
    for o in outs:
        o.fill_(-1)
    torch.cuda.synchronize()
    return want


def test_noalloc_matches_batch_plan_on_two_calls_in_a_row():
    torch.cuda.set_device(0)
    first = _batch(300, 424242, 1 << 18)
    second = _batch(90, 171717, 1 << 14)
    want1 = _reference(first[0], first[1], first[2])
    want2 = _reference(second[0], second[1], second[2])

    before = bs.bsfp_launch_count()
    bs.bsfp_batch_run_noalloc(first[0], first[1])
    bs.bsfp_batch_run_noalloc(second[0], second[1])
    torch.cuda.synchronize()
    assert bs.bsfp_launch_count() > before

    # bit-exact: this is integer logic, the tolerance is zero
    for call, (batch, want) in enumerate(((first, want1), (second, want2))):
        for i, (o, w) in enumerate(zip(batch[2], want)):
            assert torch.equal(o, w), "call %d job %d differs from the batch plan" % (call + 1, i)


def test_noalloc_rejects_sizes_beyond_its_scratch_before_launching():
    L = _binding._lib()
    jobs = (bs.bsfp_job * 1)()
    assert L.bsfp_batch_run_noalloc(jobs, bs.NOALLOC_MAX_JOBS + 1, None) == bs.ERR_SIZE
    assert L.bsfp_batch_run_noalloc(jobs, -1, None) == bs.ERR_SIZE
    assert L.bsfp_batch_run_noalloc(ctypes.cast(None, ctypes.POINTER(bs.bsfp_job)), 3, None) == bs.ERR_NULL
    # one job of 2^40 elements needs 2^25 tiles: refused by the host-side
    # check, so the (aligned, never dereferenced) addresses are not touched
    big, nj = bs.make_jobs([(bs.Format(4, 3), "add", 256, 512, None, 768, 1 << 40)])
    before = bs.bsfp_launch_count()
    assert L.bsfp_batch_run_noalloc(big, nj, None) == bs.ERR_SIZE
    assert bs.bsfp_launch_count() == before
