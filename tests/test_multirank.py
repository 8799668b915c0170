"""The benchmark's multi-rank logic on CPU with two gloo ranks: each rank
draws its own operands (its rank is the generator stream), the job time is
the slowest rank's, and the whole-job throughput counts every rank's
elements.  The data path has no exchange between ranks; only the timing
reduction is a collective."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    ms = 10.0 + 5.0 * r                     # rank 1 is the slower one
    slowest = bench.max_over_ranks(ms, dist, w, "cpu")
    vals = synth.fp_values(5, 7, 4096, synth.SEED_A, stream=r)
    gathered = [torch.zeros(4096, dtype=torch.int64) for _ in range(w)]
    dist.all_gather(gathered, torch.from_numpy(vals.astype(np.int64)))
    same = all(torch.equal(gathered[0], g) for g in gathered[1:])
    out[rank] = (r, w, local, slowest, bench.job_throughput(w, 1000.0, slowest), same)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_data_and_take_the_slowest_time():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert sorted(out.keys()) == [0, 1]
    for rank in (0, 1):
        r, w, local, slowest, thr, same = out[rank]
        assert (r, w, local) == (rank, 2, rank)
        assert slowest == 15.0
        assert thr == pytest.approx(2 * 1000.0 / 15e-3)
        assert not same                      # each rank's operands are its own


def test_reference_arm_works_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(None) == 0    # returns before touching its arguments
