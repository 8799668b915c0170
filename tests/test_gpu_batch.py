"""The batched launch: every job of a mixed batch (formats, ops, roundings,
lengths from 0 to tens of thousands, plus formats outside the persistent set)
is bit-identical to the oracle and to the same job run alone, in the
persistent plan, in the graph of plain launches and as plain launches without
a graph; graph replays give the same result again."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_1602_04716_gb300 as bs  # noqa: E402

pytestmark = pytest.mark.gpu

OPS = ["add", "sub", "mul", "fma2", "div"]
FTZ_FORMATS = [(4, 3), (4, 4), (5, 7), (5, 10), (8, 7), (8, 23)]


def _dev(x: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int32).copy()).cuda()


def _make_batch(njobs, seed, max_len=1 << 16, extra_formats=((6, 9), (3, 2), (8, 23))):
    r = synth.splitmix64(seed, 4 * njobs)
    fmts = bs.BATCH_FORMATS + list(extra_formats)
    lens = synth.log_uniform_lengths(njobs, 1, max_len, seed, 1)
    jobs = []
    for i in range(njobs):
        E, M = fmts[int(r[4 * i] % len(fmts))]
        op = OPS[int(r[4 * i + 1] % len(OPS))]
        # flush-to-zero modes where compiled (they run as plain kernels in a plan)
        rnd = int(r[4 * i + 2] % (4 if (E, M) in FTZ_FORMATS else 2))
        n = int(lens[i]) if i % 17 else (0 if i % 34 == 0 else int(lens[i]) + 31)
        B = 1 + E + M
        a, b, c = (synth.fp_values(E, M, n, seed + 10 * i + k).astype(np.uint32) for k in (1, 2, 3))
        t = {k: _dev(oracle.pack(B, v)) for k, v in (("a", a), ("b", b), ("c", c))}
        t["out"] = torch.full_like(t["a"], -1)
        jobs.append(dict(E=E, M=M, op=op, rnd=rnd, n=n, a=a, b=b, c=c, t=t))
    return jobs


def _ctypes_jobs(jobs):
    return bs.make_jobs((bs.Format(j["E"], j["M"], j["rnd"]), j["op"], j["t"]["a"], j["t"]["b"],
                         j["t"]["c"] if j["op"] == "fma2" else None, j["t"]["out"], j["n"]) for j in jobs)


def _check_all(jobs):
    for i, j in enumerate(jobs):
        B = 1 + j["E"] + j["M"]
        want = oracle.pack(B, oracle.binop(j["op"], j["E"], j["M"], j["rnd"], j["a"], j["b"], j["c"]))
        got = j["t"]["out"].cpu().numpy().view(np.uint32).reshape(B, -1)
        if j["n"] == 0:
            continue
        assert (got == want).all(), "job %d: %s 1/%d/%d rnd=%d n=%d" % (i, j["op"], j["E"], j["M"], j["rnd"], j["n"])


def _clear(jobs):
    for j in jobs:
        j["t"]["out"].fill_(-1)


@pytest.mark.parametrize("wpt", [1, 2])
def test_persistent_plan_matches_oracle_and_replays(wpt):
    jobs = _make_batch(220, 5000 + wpt)
    arr, nj = _ctypes_jobs(jobs)
    plan = bs.BatchPlan(arr, nj, bs.BATCH_PERSISTENT, wpt)
    n_plain = sum(1 for j in jobs if (j["E"], j["M"]) not in bs.BATCH_FORMATS and j["n"] > 0)
    assert plan.launches >= n_plain + 1
    for _ in range(2):   # the second run replays the graph with the counters cleared again
        _clear(jobs)
        plan.run()
        torch.cuda.synchronize()
        _check_all(jobs)
    plan.free()


@pytest.mark.parametrize("blocks_per_sm", [1, 2])
def test_persistent_plan_small_grids(blocks_per_sm):
    """Few resident CTAs: every CTA loops over many tiles."""
    jobs = _make_batch(60, 7100 + blocks_per_sm, max_len=1 << 18, extra_formats=())
    arr, nj = _ctypes_jobs(jobs)
    plan = bs.BatchPlan(arr, nj, bs.BATCH_PERSISTENT, 2, blocks_per_sm)
    plan.run()
    torch.cuda.synchronize()
    _check_all(jobs)
    plan.free()


def test_streamed_plan_matches_oracle_and_replays():
    """BSFP_BATCH_STREAMED: add/sub/mul jobs of the five batched formats (all
    four rounding modes) run as one streamed kernel per (format, rounding, op
    class) over the tiles of all its jobs, fma2 as the persistent kernels,
    everything else as plain launches; every job exact, and again on a
    replay of the graph."""
    jobs = _make_batch(220, 5100)
    arr, nj = _ctypes_jobs(jobs)
    bs.bsfp_set_batch_stream_min_tiles(0)   # every group streamed, however small
    try:
        plan = bs.BatchPlan(arr, nj, bs.BATCH_STREAMED)
    finally:
        bs.bsfp_set_batch_stream_min_tiles(8)
    groups = {(j["E"], j["M"], j["rnd"], j["op"] == "mul") for j in jobs
              if (j["E"], j["M"]) in bs.BATCH_FORMATS and j["op"] in ("add", "sub", "mul") and j["n"] > 0}
    n_plain = sum(1 for j in jobs if j["n"] > 0 and ((j["E"], j["M"]) not in bs.BATCH_FORMATS or j["op"] == "div" or
                                                     (j["op"] == "fma2" and j["rnd"] > 1)))
    n_persistent = 1 if any(j["op"] == "fma2" and j["rnd"] < 2 and (j["E"], j["M"]) in bs.BATCH_FORMATS and j["n"] > 0
                            for j in jobs) else 0
    assert plan.launches == len(groups) + n_persistent + n_plain
    for _ in range(2):
        _clear(jobs)
        plan.run()
        torch.cuda.synchronize()
        _check_all(jobs)
    assert bs.bsfp_fault_status() == 0
    plan.free()


def test_streamed_plan_many_tiles_per_block():
    """Jobs up to 2^20 elements of the batched formats only: each streamed
    group has more tiles than SMs, so every block goes round its ring."""
    jobs = _make_batch(48, 7300, max_len=1 << 20, extra_formats=())
    for j in jobs:
        if j["op"] in ("fma2", "div"):
            j["op"] = "mul"
    arr, nj = _ctypes_jobs(jobs)
    bs.bsfp_set_batch_stream_min_tiles(0)
    try:
        plan = bs.BatchPlan(arr, nj, bs.BATCH_STREAMED)
    finally:
        bs.bsfp_set_batch_stream_min_tiles(8)
    plan.run()
    torch.cuda.synchronize()
    _check_all(jobs)
    assert bs.bsfp_fault_status() == 0
    plan.free()


def test_streamed_plan_sends_small_groups_to_the_persistent_kernels():
    """With the default threshold (8 tiles per SM per group on average) the
    RN/RZ groups of a small batch all run in the persistent kernels (one
    launch per op class); the flush-to-zero groups, which the persistent
    kernels do not cover, stay streamed.  Every job exact."""
    jobs = _make_batch(220, 5200)
    arr, nj = _ctypes_jobs(jobs)
    plan = bs.BatchPlan(arr, nj, bs.BATCH_STREAMED)
    live = [j for j in jobs if j["n"] > 0]
    batch = [j for j in live if (j["E"], j["M"]) in bs.BATCH_FORMATS]
    stream_groups = {(j["E"], j["M"], j["rnd"], j["op"] == "mul") for j in batch
                     if j["op"] in ("add", "sub", "mul") and j["rnd"] > 1}
    persistent = {("mul" if j["op"] == "mul" else "fma2" if j["op"] == "fma2" else "add") for j in batch
                  if j["op"] in ("add", "sub", "mul", "fma2") and j["rnd"] < 2}
    plain = [j for j in live if (j["E"], j["M"]) not in bs.BATCH_FORMATS or j["op"] == "div" or
             (j["op"] == "fma2" and j["rnd"] > 1)]
    assert plan.launches == len(stream_groups) + len(persistent) + len(plain)
    _clear(jobs)
    plan.run()
    torch.cuda.synchronize()
    _check_all(jobs)
    plan.free()


def test_unified_plan_matches_oracle_and_replays():
    """BSFP_BATCH_UNIFIED: the RN/RZ add/sub jobs of the five batched formats
    in one streamed launch and their mul jobs in another, whatever the
    format; tiles (of a width per format) from an atomic counter.  The other
    jobs go as in the streamed plan.  Every job exact, and again on a replay
    (the counters are cleared by the graph)."""
    jobs = _make_batch(220, 5300)
    arr, nj = _ctypes_jobs(jobs)
    plan = bs.BatchPlan(arr, nj, bs.BATCH_UNIFIED)
    live = [j for j in jobs if j["n"] > 0]
    batch = [j for j in live if (j["E"], j["M"]) in bs.BATCH_FORMATS]
    unified = {j["op"] == "mul" for j in batch if j["op"] in ("add", "sub", "mul") and j["rnd"] < 2}
    ftz_groups = {(j["E"], j["M"], j["rnd"], j["op"] == "mul") for j in batch
                  if j["op"] in ("add", "sub", "mul") and j["rnd"] > 1}
    persistent = 1 if any(j["op"] == "fma2" and j["rnd"] < 2 for j in batch) else 0
    plain = [j for j in live if (j["E"], j["M"]) not in bs.BATCH_FORMATS or j["op"] == "div" or
             (j["op"] == "fma2" and j["rnd"] > 1)]
    assert plan.launches == len(unified) + len(ftz_groups) + persistent + len(plain)
    for _ in range(2):
        _clear(jobs)
        plan.run()
        torch.cuda.synchronize()
        _check_all(jobs)
    assert bs.bsfp_fault_status() == 0
    plan.free()


def test_unified_plan_many_tiles_per_block():
    """Jobs up to 2^20 elements of the batched formats, RN/RZ add, sub and
    mul only: many more tiles than SMs, of every kind interleaved, so every
    block goes round its ring many times and the last tile of many jobs is
    ragged."""
    jobs = _make_batch(64, 7400, max_len=1 << 20, extra_formats=())
    for i, j in enumerate(jobs):
        j["rnd"] = j["rnd"] & 1
        if j["op"] in ("fma2", "div"):
            j["op"] = ("add", "sub", "mul")[i % 3]
    arr, nj = _ctypes_jobs(jobs)
    plan = bs.BatchPlan(arr, nj, bs.BATCH_UNIFIED)
    assert plan.launches == len({j["op"] == "mul" for j in jobs if j["n"] > 0})
    _clear(jobs)
    plan.run()
    torch.cuda.synchronize()
    _check_all(jobs)
    assert bs.bsfp_fault_status() == 0
    plan.free()


def test_plain_graph_and_plain_launches_match():
    jobs = _make_batch(120, 8000)
    arr, nj = _ctypes_jobs(jobs)
    plan = bs.BatchPlan(arr, nj, bs.BATCH_PLAIN)
    assert plan.launches == sum(1 for j in jobs if j["n"] > 0)
    plan.run()
    torch.cuda.synchronize()
    _check_all(jobs)
    plan.free()
    _clear(jobs)
    before = bs.bsfp_launch_count()
    bs.bsfp_launch_jobs(arr, nj)
    torch.cuda.synchronize()
    assert bs.bsfp_launch_count() - before == sum(1 for j in jobs if j["n"] > 0)
    _check_all(jobs)


def test_each_job_alone_equals_the_mix():
    jobs = _make_batch(40, 9000)
    arr, nj = _ctypes_jobs(jobs)
    plan = bs.BatchPlan(arr, nj)
    plan.run()
    torch.cuda.synchronize()
    mixed = [j["t"]["out"].clone() for j in jobs]
    plan.free()
    for j, m in zip(jobs, mixed):
        j["t"]["out"].fill_(-1)
        bs.bsfp_op(j["op"], bs.Format(j["E"], j["M"], j["rnd"]), j["t"]["a"], j["t"]["b"], j["t"]["out"], j["n"],
                   c=j["t"]["c"])
        torch.cuda.synchronize()
        if j["n"]:
            assert torch.equal(j["t"]["out"], m)


def test_invalid_job_rejected_before_anything_runs():
    jobs = _make_batch(5, 9100, extra_formats=())
    arr, nj = _ctypes_jobs(jobs)
    arr[3].f.exp_bits = 9
    with pytest.raises(bs.BsfpError) as ei:
        bs.BatchPlan(arr, nj)
    assert ei.value.status == bs.ERR_FORMAT
    arr[3].f.exp_bits = 4
    arr[2].a = arr[2].a + 4 if arr[2].a else 4
    with pytest.raises(bs.BsfpError) as ei:
        bs.BatchPlan(arr, nj)
    assert ei.value.status in (bs.ERR_ALIGN, bs.ERR_NULL)
