"""The request server (continuous batching): every result of a request served
in a mix of concurrent, mixed-format, mixed-length requests is bit-identical
to the same op run alone; admission never exceeds the result budget and keeps
arrival order; waits are bounded."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_1602_04716_gb300 as bs  # noqa: E402

pytestmark = pytest.mark.gpu

OPS = ["add", "sub", "mul", "fma2", "div"]


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int32).copy()).cuda()


def _requests(nreq, seed, lo=1, hi=1 << 16, fmts=None):
    fmts = fmts or (bs.BATCH_FORMATS + [(6, 9), (3, 2)])
    r = synth.splitmix64(seed, 3 * nreq)
    lens = synth.log_uniform_lengths(nreq, lo, hi, seed, 1)
    reqs = []
    for i in range(nreq):
        E, M = fmts[int(r[3 * i] % len(fmts))]
        op = OPS[int(r[3 * i + 1] % len(OPS))]
        rnd = int(r[3 * i + 2] % 2)
        n = 0 if i % 37 == 3 else int(lens[i])
        B = 1 + E + M
        vals = [synth.fp_values(E, M, n, seed + 17 * i + k).astype(np.uint32) for k in range(3)]
        t = [_dev(oracle.pack(B, v)) for v in vals]
        reqs.append(dict(f=bs.Format(E, M, rnd), op=op, n=n, B=B, vals=vals, t=t))
    return reqs


def _alone(q):
    out = torch.empty_like(q["t"][0])
    bs.bsfp_op(q["op"], q["f"], q["t"][0], q["t"][1], out, q["n"], c=q["t"][2])
    torch.cuda.synchronize()
    return out


def _jobs(reqs):
    return bs.make_jobs((q["f"], q["op"], q["t"][0], q["t"][1], q["t"][2] if q["op"] == "fma2" else None, None,
                         q["n"]) for q in reqs)


def test_results_in_the_mix_equal_alone_and_the_oracle():
    reqs = _requests(240, 31337)
    arr, nj = _jobs(reqs)
    srv = bs.Server(1 << 30, slots=4)
    # 240 requests over ~6 ms: several micro-batches in flight at once
    arrivals = np.cumsum(synth.uniform01(nj, 4242) * 50_000).astype(np.int64)
    done = srv.replay(arr, nj, arrivals, release=False)
    st = srv.stats()
    assert st["completed"] == nj and st["failed"] == 0 and st["pending"] == 0
    for i, q in enumerate(reqs):
        c = done[i]
        assert c.status == 0 and c.n == q["n"]
        assert c.t_submit_ns <= c.t_admit_ns <= c.t_done_ns
        if q["n"] == 0:
            srv.release(c.id)
            continue
        got = bs.Server.result(c, q["f"]).clone()
        assert torch.equal(got, _alone(q).flatten()), "request %d differs from the op alone" % i
        if i % 8 == 0:
            E, M = q["f"].exp_bits, q["f"].man_bits
            want = oracle.pack(q["B"], oracle.binop(q["op"], E, M, q["f"].rnd, *q["vals"]))
            assert (got.cpu().numpy().view(np.uint32).reshape(q["B"], -1) == want).all()
        srv.release(c.id)
    assert srv.stats()["arena_bytes_in_use"] == 0
    srv.close()


def test_admission_stays_within_the_budget_and_in_order():
    reqs = _requests(60, 777, lo=1 << 12, hi=1 << 16, fmts=bs.BATCH_FORMATS)
    biggest = max(bs.bsfp_bitslice_bytes(q["f"], q["n"]) for q in reqs)
    budget = 3 * ((biggest + 255) // 256 * 256)
    srv = bs.Server(budget, slots=4)
    ids = [srv.submit(q["f"], q["op"], q["t"][0], q["t"][1], q["n"], c=q["t"][2]) for q in reqs]
    seen, admitted = {}, {}
    import time
    t_end = time.time() + 30
    while len(seen) < len(ids) and time.time() < t_end:
        for c in srv.poll():
            assert c.status == 0
            k = ids.index(c.id)
            seen[c.id] = bs.Server.result(c, reqs[k]["f"]).clone()
            admitted[c.id] = c.t_admit_ns
            srv.release(c.id)
    assert len(seen) == len(ids)
    st = srv.stats()
    assert st["arena_peak_bytes"] <= budget and st["arena_bytes_in_use"] == 0
    assert st["batches"] > 1   # the budget forced several admissions
    # strictly in arrival order: admission times never decrease along the ids
    adm = [admitted[r] for r in ids]
    assert adm == sorted(adm)
    for k, rid in enumerate(ids):
        assert torch.equal(seen[rid], _alone(reqs[k]).flatten())
    srv.close()


def test_caller_owned_results_use_no_arena_memory():
    reqs = _requests(20, 99, fmts=[(4, 3), (5, 10), (8, 23)])
    srv = bs.Server(1 << 20)
    outs = []
    for q in reqs:
        o = torch.full_like(q["t"][0], -1)
        outs.append(o)
        srv.submit(q["f"], q["op"], q["t"][0], q["t"][1], q["n"], c=q["t"][2], out=o)
    srv.drain(10000)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["arena_peak_bytes"] == 0
    for q, o in zip(reqs, outs):
        if q["n"]:
            assert torch.equal(o, _alone(q))
    srv.close()


def test_budget_errors_and_bounded_drain():
    q = _requests(1, 5, lo=1 << 16, hi=1 << 16, fmts=[(5, 7)])[0]
    need = bs.bsfp_bitslice_bytes(q["f"], q["n"])
    small = bs.Server(need // 2)
    with pytest.raises(bs.BsfpError) as ei:
        small.submit(q["f"], q["op"], q["t"][0], q["t"][1], q["n"], c=q["t"][2])
    assert ei.value.status == bs.ERR_BUDGET
    small.close()
    # room for exactly one result: the second waits until the first is released
    one = bs.Server((need + 255) // 256 * 256)
    r1 = one.submit(q["f"], q["op"], q["t"][0], q["t"][1], q["n"], c=q["t"][2])
    r2 = one.submit(q["f"], q["op"], q["t"][0], q["t"][1], q["n"], c=q["t"][2])
    with pytest.raises(bs.BsfpError) as ei:
        one.drain(300)
    assert ei.value.status == bs.ERR_TIMEOUT
    done = one.poll()
    assert [c.id for c in done] == [r1]
    with pytest.raises(bs.BsfpError):
        one.release(r2)           # not finished yet
    one.release(r1)
    one.drain(10000)
    done = one.poll()
    assert [c.id for c in done] == [r2]
    one.release(r2)
    with pytest.raises(bs.BsfpError):
        one.release(r2)           # released twice
    assert one.stats()["arena_peak_bytes"] <= (need + 255) // 256 * 256
    one.close()


def test_allocation_failure_is_reported_and_leaves_nothing_behind():
    """A budget far beyond the device's memory: creation fails with
    BSFP_ERR_CUDA (a refused cudaMalloc, not a fault), and the device stays
    usable with its free memory unchanged."""
    free0, _ = torch.cuda.mem_get_info()
    with pytest.raises(bs.BsfpError) as ei:
        bs.Server(1 << 50)
    assert ei.value.status == bs.ERR_CUDA
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < (64 << 20)
    srv = bs.Server(1 << 20)      # still works afterwards
    srv.close()


def test_burst_submission_is_batched_and_exact():
    """A burst submitted in one call (bsfp_server_submit_n) is admitted many
    requests at a time -- a handful of micro-batches for 400 requests -- and
    every result equals the op run alone."""
    reqs = _requests(400, 4711, lo=1 << 10, hi=1 << 16)
    arr, nj = _jobs(reqs)
    srv = bs.Server(1 << 30, slots=4)
    ids = srv.submit_n(arr, nj)
    assert ids == sorted(ids) and len(set(ids)) == nj
    srv.drain(30000)
    st = srv.stats()
    assert st["completed"] == nj and st["failed"] == 0
    assert st["batches"] <= nj // 20, st
    got = {}
    while len(got) < nj:
        for c in srv.poll():
            assert c.status == 0
            got[c.id] = c
    for k, rid in enumerate(ids):
        q = reqs[k]
        c = got[rid]
        if q["n"]:
            assert torch.equal(bs.Server.result(c, q["f"]).clone(), _alone(q).flatten()), "request %d" % k
        srv.release(rid)
    assert srv.stats()["arena_bytes_in_use"] == 0
    srv.close()


def test_burst_with_an_invalid_job_submits_nothing():
    reqs = _requests(8, 5150, lo=64, hi=4096, fmts=bs.BATCH_FORMATS)
    arr, nj = _jobs(reqs)
    arr[5].a = (arr[5].a or 0) + 4   # misaligned operand
    srv = bs.Server(1 << 26)
    with pytest.raises(bs.BsfpError) as ei:
        srv.submit_n(arr, nj)
    assert ei.value.status == bs.ERR_ALIGN
    assert srv.stats()["submitted"] == 0
    srv.close()
