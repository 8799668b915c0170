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
    # one job of 2^40 elements needs 2^27 tiles: refused by the host-side
    # check, so the (aligned, never dereferenced) addresses are not touched
    big, nj = bs.make_jobs([(bs.Format(4, 3), "add", 256, 512, None, 768, 1 << 40)])
    before = bs.bsfp_launch_count()
    assert L.bsfp_batch_run_noalloc(big, nj, None) == bs.ERR_SIZE
    assert bs.bsfp_launch_count() == before


def test_noalloc_checks_every_job_before_launching_any():
    """A bad job anywhere in the array (here a misaligned operand in job 7 of
    12) is refused before anything is copied or launched."""
    arr, nj, outs, keep = _batch(12, 9090, 1 << 12)
    arr[7].out = (arr[7].out or 256) + 4
    before = bs.bsfp_launch_count()
    L = _binding._lib()
    assert L.bsfp_batch_run_noalloc(arr, nj, None) == bs.ERR_ALIGN
    torch.cuda.synchronize()
    assert bs.bsfp_launch_count() == before
    for o in outs:
        assert bool((o == -1).all())


def test_noalloc_with_no_persistent_job_runs_the_plain_kernels():
    """Only division and flush-to-zero jobs: no tile for the persistent
    kernels (the scratch is not used at all), every job as its plain kernel;
    outputs equal the batch plan's."""
    specs, keep = [], []
    for i, (E, M, rnd, op) in enumerate([(5, 7, 0, "div"), (4, 4, 2, "add"), (5, 10, 3, "mul"), (8, 7, 1, "div"),
                                         (4, 3, 2, "fma2"), (6, 9, 0, "div")]):
        f = bs.Format(E, M, rnd)
        n = 1000 + 977 * i
        ops_ = []
        for k in range(3):
            p = bs.empty_bitslice(f, n)
            std = torch.from_numpy(synth.fp_values(E, M, n, 600 + 7 * i + k).view(
                {1: np.uint8, 2: np.int16, 4: np.int32}[bs.bsfp_container_bytes(f)])).cuda()
            bs.bsfp_pack(f, std, n, p)
            ops_.append(p)
        out = torch.full_like(ops_[0], -1)
        specs.append((f, op, ops_[0], ops_[1], ops_[2] if op == "fma2" else None, out, n))
        keep.append((ops_, out))
    arr, nj = bs.make_jobs(specs)
    outs = [o for _, o in keep]
    want = _reference(arr, nj, outs)
    bs.bsfp_batch_run_noalloc(arr, nj)
    torch.cuda.synchronize()
    for i, (o, w) in enumerate(zip(outs, want)):
        assert torch.equal(o, w), "job %d differs from the batch plan" % i


def test_noalloc_jobs_changed_before_their_copy_skip_the_work_and_raise_the_fault_word():
    """Page-locked jobs changed after the call returns but before the stream
    reaches its copy: the kernels read jobs other than the validated ones.
    The prologue sees its totals differ from the host's, so the persistent
    kernels take no tile and the fault word becomes 1.  The change only
    shortens a job, so every address stays inside its buffers even if the
    check were missing.  The stream is kept busy first with ordinary adds so
    that the copy starts well after the change."""
    arr, nj, outs, keep = _batch(40, 31415, 1 << 16)
    sz = ctypes.sizeof(bs.bsfp_job) * nj
    pinned = torch.empty(sz, dtype=torch.uint8, pin_memory=True)
    ctypes.memmove(pinned.data_ptr(), ctypes.addressof(arr), sz)
    jobs_p = ctypes.cast(pinned.data_ptr(), ctypes.POINTER(bs.bsfp_job))
    # the same jobs once, unchanged: every map entry of this layout is valid
    bs.bsfp_batch_run_noalloc(jobs_p, nj)
    torch.cuda.synchronize()
    assert bs.bsfp_fault_status(clear=True) == 0
    persistent = {(E, M) for E, M in bs.BATCH_FORMATS}
    k = max((i for i in range(nj) if jobs_p[i].n > 40000 and jobs_p[i].f.rnd in (0, 1) and jobs_p[i].op != 4
             and (jobs_p[i].f.exp_bits, jobs_p[i].f.man_bits) in persistent), default=None)
    assert k is not None
    f = bs.Format(5, 7)
    big = 1 << 28
    xa = torch.zeros(13 * bs.bsfp_plane_stride(big), dtype=torch.int32, device="cuda")
    xo = torch.empty_like(xa)
    for _ in range(20):   # about 4 ms of work ahead of the copy on this stream
        bs.bsfp_add(f, xa, xa, xo, big)
    bs.bsfp_batch_run_noalloc(jobs_p, nj)
    jobs_p[k].n = 40   # one tile instead of several
    torch.cuda.synchronize()
    assert bs.bsfp_fault_status(clear=True) == 1
    assert bs.bsfp_fault_status() == 0
    del xa, xo
