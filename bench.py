#!/usr/bin/env python
"""Benchmark of the bitslice custom-precision FP hot path on one GB300.

Workload (one step): element-wise bs_add and bs_mul, round to nearest even,
on 2^28-element vectors of the 9-bit format 1/4/4 and of the 13-bit format
1/5/7, operands resident on the device in bitslice form -- four kernel
launches, 4 * 2^28 elements.  Operands come from the seeded SplitMix64 recipe
(sign uniform, exponent 98% uniform over the normal range, 1% zero field, 1%
all-ones field, fraction uniform), drawn on the device and packed once before
timing.  Every operand (288-416 MB) is larger than the 129 MB L2, so no flush
is needed between iterations.

Printed: one JSON line with elements/s over the whole job, the roofline of
the dominant kernel (the slower of its HBM bytes at the measured copy
bandwidth and of its circuit's gate count at the measured logic-op issue
rate), the clocks seen during the timed region, an end-to-end figure through
the C ABI from and to pinned host buffers, and the CPU oracle's throughput on
a bounded sample of the same workload.

``--impl reference`` times the CPU oracle itself on the same metric (bounded
samples of the workload per step); only rank 0 works under torchrun.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "custom-FP elements/s and % roofline for bs_add/bs_mul, batched vs plain; p99 latency"
UNIT = "elements/s"
FORMATS = [(4, 4), (5, 7)]
OPS = ["add", "mul"]
N = 1 << 28
RND = 0
WORKLOAD = ("plain single-format at scale: bs_add + bs_mul (RN) on 1/4/4 and 1/5/7, "
            "2^28 elements per vector, operands resident in bitslice form")

# dram__bytes_read.sum + dram__bytes_write.sum of one launch, from ncu captures at 2^26 elements
# scaled x4 to the 2^28-element launch, keyed by (E, M, op, kernel variant): a figure stands only
# for the kernel it was taken on, as it now stands (profiles/traffic_bench_kernels_2p26.md: medians of
# six launches each); a kernel not listed reports null.
NCU_TRAFFIC = {(4, 4, "add", 8): (151.015168e6 + 35.996672e6) * 4,
               (4, 4, "mul", 8): (151.014912e6 + 36.211712e6) * 4,
               (5, 7, "add", 8): (218.130432e6 + 66.021376e6) * 4,
               (5, 7, "mul", 8): (218.155776e6 + 62.862592e6) * 4}


class DeviceTimer:
    """Device time of single calls (CUDA events on the launching stream).
    Before each timed call the L2 is flushed on the same stream: a 256 MB
    buffer is written (which evicts the 129 MB L2), then a second 256 MB
    buffer is read, which writes the first one's dirty lines back to HBM and
    leaves the L2 holding clean lines only.  So no operand is served from the
    previous call's cache, the timed call does not pay for write-backs of the
    flush, and the GPU stays busy while the host enqueues the first event and
    the call, so the host's launch latency is not counted."""

    def __init__(self, torch, stream, flush_bytes: int = 256 << 20):
        self.torch, self.stream = torch, stream
        self.buf = torch.empty(flush_bytes // 4, dtype=torch.int32, device="cuda")
        self.clean = torch.zeros(flush_bytes // 4, dtype=torch.int32, device="cuda")

    def flush(self):
        self.buf.fill_(0)
        self.clean.sum()

    def ms(self, fn, reps: int = 5) -> float:
        torch = self.torch
        fn()
        ts = []
        with torch.cuda.stream(self.stream):
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                self.flush()
                e0.record(self.stream)
                fn()
                e1.record(self.stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))


def apply_tuning() -> int:
    from paper_1602_04716_gb300 import tune
    return tune.apply()


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling (every 200 ms) around the timed region; the
    summary keeps the samples whose timestamps fall inside it (mark_start /
    mark_end), and says so, falling back to all samples if none does."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        self.t_start = self.t_end = None
        self.fh = tempfile.NamedTemporaryFile("w", suffix=".csv", delete=False)
        self.path = self.fh.name
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def mark_start(self):
        self.t_start = time.time()

    def mark_end(self):
        self.t_end = time.time()

    @staticmethod
    def _when(stamp: str):
        import datetime
        try:
            return datetime.datetime.strptime(stamp.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self):
        if self.proc is None:
            self.fh.close()
            os.unlink(self.path)
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        inside = rows
        in_region = False
        if self.t_start is not None and self.t_end is not None:
            sel = [r for r in rows if (self._when(r[0]) or 0) >= self.t_start and (self._when(r[0]) or 0) <= self.t_end]
            if sel:
                inside, in_region = sel, True
        sm = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside), "samples_in_timed_region": in_region}


def lop3_rate(bs, torch) -> float:
    """Chip-wide 32-bit logic-op rate (lane-ops/s) from the LOP3 probe."""
    sms = bs.bsfp_num_sms()
    grid, block, iters = sms * 8, 256, 4000
    sink = torch.empty(grid * block, dtype=torch.int32, device="cuda")
    bs.bsfp_lop3_probe(sink, grid, block, 50)
    torch.cuda.synchronize()
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        bs.bsfp_lop3_probe(sink, grid, block, iters)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return grid * block * iters * bs.PROBE_LOP3_PER_ROUND / (best * 1e-3)


def cpu_baseline(target_s: float = 12.0):
    """The oracle, as it stands, on a bounded sample of the workload: the first
    2^26 elements of each of the four (format, op) vectors, passed over
    repeatedly until about target_s seconds of oracle time have been spent."""
    import oracle
    m = min(N, 1 << 26)
    data = {}
    for E, M in FORMATS:
        data[(E, M)] = (synth.fp_values(E, M, m, synth.SEED_A).astype(np.uint32),
                        synth.fp_values(E, M, m, synth.SEED_B).astype(np.uint32))
    tot, els, passes = 0.0, 0, 0
    while tot < target_s or passes == 0:
        for E, M in FORMATS:
            a, b = data[(E, M)]
            for op in OPS:
                t = time.perf_counter()
                oracle.binop(op, E, M, RND, a, b)
                tot += time.perf_counter() - t
                els += m
        passes += 1
    cores = oracle.num_threads()
    # the same oracle on one core, over the first 2^22 elements of each vector
    m1 = min(m, 1 << 22)
    oracle.set_threads(1)
    try:
        t1, els1 = 0.0, 0
        for E, M in FORMATS:
            a, b = data[(E, M)]
            for op in OPS:
                t = time.perf_counter()
                oracle.binop(op, E, M, RND, a[:m1], b[:m1])
                t1 += time.perf_counter() - t
                els1 += m1
    finally:
        oracle.set_threads(cores)
    return {"value": els / tot, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "first %d elements of each of the 4 (format, op) vectors of the workload (same seeds), "
                      "%d passes, %.1f s of oracle time" % (m, passes, tot),
            "single_core": {"value": els1 / t1, "unit": UNIT, "cores": 1,
                            "sample": "first %d elements of each of the 4 vectors, one pass, %.1f s" % (m1, t1)}}


def run_reference(args):
    rank = dist_env()[0]
    if rank != 0:
        return 0
    import oracle
    m = args.ref_sample
    data = {}
    for E, M in FORMATS:
        data[(E, M)] = (synth.fp_values(E, M, m, synth.SEED_A).astype(np.uint32),
                        synth.fp_values(E, M, m, synth.SEED_B).astype(np.uint32))

    def step():
        for E, M in FORMATS:
            a, b = data[(E, M)]
            for op in OPS:
                oracle.binop(op, E, M, RND, a, b)

    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t) / args.steps
    value = 4 * m / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_elements_per_vector": m, "formats": ["1/4/4", "1/5/7"],
                       "ops": OPS, "rounding": "RN"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "first %d elements of each of the 4 (format, op) vectors per step" % m},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def dist_env():
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, dist, world: int, device) -> float:
    """The largest of the ranks' values (the job ends when its slowest rank
    does); the value itself when there is one rank."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, elements_per_rank_step: float, ms_per_step: float) -> float:
    """Whole-job elements/s: every rank processes its own elements (weak
    scaling, no exchange between ranks)."""
    return world * elements_per_rank_step / (ms_per_step * 1e-3)


def run_gpu(args):
    import torch
    import torch.distributed as dist
    import paper_1602_04716_gb300 as bs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    tuned = apply_tuning()
    n = args.n
    if args.section:
        return run_section(bs, torch, args, rank)

    # ---- operands: drawn on the device, packed once, resident ----
    bufs = {}
    for E, M in FORMATS:
        f = bs.Format(E, M, RND)
        std = bs.empty_standard(f, n)
        planes = []
        for seed in (synth.SEED_A, synth.SEED_B):
            bs.bsfp_synth_fp_values(f, n, seed, rank, 0, std)
            p = bs.empty_bitslice(f, n)
            bs.bsfp_pack(f, std, n, p)
            planes.append(p)
        bufs[(E, M)] = (f, planes[0], planes[1], bs.empty_bitslice(f, n))
        del std
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    kern = [(E, M, op) for E, M in FORMATS for op in OPS]

    def step(evs=None):
        for i, (E, M, op) in enumerate(kern):
            f, a, b, out = bufs[(E, M)]
            if evs is not None:
                evs[i][0].record(stream)
            bs.bsfp_op(op, f, a, b, out, n, stream=stream)
            if evs is not None:
                evs[i][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    L = lop3_rate(bs, torch)
    hbm, hbm_kind = _peaks()

    evs = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in kern]
           for _ in range(args.steps)]
    clocks = Clocks(local) if rank == 0 else None
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = bs.bsfp_launch_count()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if clocks:
        clocks.mark_start()
    t0.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t1.record(stream)
    torch.cuda.synchronize()
    if clocks:
        clocks.mark_end()
    launches = bs.bsfp_launch_count() - launches0
    if world > 1:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    ms_max = max_over_ranks(t0.elapsed_time(t1), dist, world, "cuda")
    ms_step = ms_max / args.steps
    value = job_throughput(world, len(kern) * n, ms_step)

    # ---- per-kernel roofline ----
    kinfo = []
    for i, (E, M, op) in enumerate(kern):
        t = float(np.mean([evs[k][i][0].elapsed_time(evs[k][i][1]) for k in range(args.steps)])) * 1e-3
        f = bufs[(E, M)][0]
        B = 1 + E + M
        G = bs.bsfp_gate_count(f, op)
        nwords = (n + 31) // 32
        bytes_ = 3 * B * n / 8
        r_hbm = hbm * 1e9 / (3 * B / 8)
        r_alu = L * 32 / G
        bound = "hbm" if r_hbm <= r_alu else "alu"
        eps = n / t
        kinfo.append({"kernel": "bs_%s 1/%d/%d" % (op, E, M), "ms": t * 1e3, "elements_per_s": eps,
                      "hbm_gbs": bytes_ / t / 1e9, "logic_tops": G * nwords / t / 1e12, "gates_per_word": G,
                      "wpt": bs.bsfp_variant(f, op), "roofline_elements_per_s": min(r_hbm, r_alu),
                      "bound": bound, "frac": eps / min(r_hbm, r_alu),
                      "hbm_frac": bytes_ / t / 1e9 / hbm, "alu_frac": G * nwords / t / L})
    dom = max(range(len(kern)), key=lambda i: kinfo[i]["ms"])
    d = kinfo[dom]
    E, M, op = kern[dom]
    B = 1 + E + M
    t = d["ms"] * 1e-3
    if d["bound"] == "hbm":
        roof = {"bound": "hbm", "achieved": d["hbm_gbs"], "peak": hbm, "unit": "GB/s",
                "frac": d["hbm_gbs"] / hbm, "peak_source": "%s copy bandwidth (MEASURED_PEAKS.json)" % hbm_kind}
    else:
        roof = {"bound": "alu", "achieved": d["logic_tops"], "peak": L / 1e12, "unit": "Tops/s",
                "frac": d["logic_tops"] * 1e12 / L,
                "peak_source": "measured LOP3 issue rate (bsfp_lop3_probe, this run)"}
    tr = NCU_TRAFFIC.get((E, M, op, d["wpt"])) if n == N else None
    roof.update({"kernel": d["kernel"], "traffic": tr,
                 "algorithmic_bytes": 3 * B * n / 8, "gate_ops": d["gates_per_word"] * ((n + 31) // 32),
                 "hbm_peak_gbs": hbm, "logic_peak_tops": L / 1e12})

    # ---- end to end through the C ABI from pinned host buffers ----
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(bs, torch, n, rank, args)

    batched = None
    if args.batch_jobs > 0:
        batched = run_batched(bs, torch, args, rank, hbm)

    serving = None
    if args.serve_seconds > 0:
        serving = run_serving(bs, torch, args, rank)

    small = run_small_case(bs, torch, rank) if args.sweep_n > 0 else None
    conversions = run_conversions(bs, torch, n, hbm) if args.sweep_n > 0 else None
    integers = run_integers(bs, torch, n, hbm, L) if args.sweep_n > 0 else None

    sweep = None
    if args.sweep_n > 0:
        sweep = run_sweep(bs, torch, args, rank, hbm, L)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "formats": ["1/4/4", "1/5/7"], "ops": OPS, "rounding": "RN",
                           "elements_per_vector": n, "launches_per_step": len(kern),
                           "l2": "no flush: every operand (288-416 MB) exceeds the 129 MB L2",
                           "seeds": [synth.SEED_A, synth.SEED_B], "parallelism": "dp%d" % world,
                           "tuned_shapes_applied": tuned},
                "roofline": roof, "kernels": kinfo, "clocks": clk, "e2e": e2e, "gpu_launches": launches,
                "cpu_baseline": cpu, "batched": batched, "serving": serving,
                "format_sweep": sweep, "small_case": small, "conversions": conversions,
                "integers": integers}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_section(bs, torch, args, rank):
    """One section of the bench on its own (for a profiler capture of its
    kernels, or a quick look): prints one JSON line holding that section."""
    hbm, _ = _peaks()
    n = args.n
    if args.section == "conversions":
        res = run_conversions(bs, torch, n, hbm, reps=args.section_reps)
    elif args.section == "small":
        res = run_small_case(bs, torch, rank)
    elif args.section == "integers":
        res = run_integers(bs, torch, n, hbm, lop3_rate(bs, torch))
    elif args.section == "sweep":
        res = run_sweep(bs, torch, args, rank, hbm, lop3_rate(bs, torch))
    elif args.section == "batched":
        res = run_batched(bs, torch, args, rank, hbm)
    elif args.section == "e2e":
        res = run_e2e(bs, torch, n, rank, args)
    else:
        res = run_serving(bs, torch, args, rank)
    if rank == 0:
        print(json.dumps({"section": args.section, "elements_per_vector": n, args.section: res}), flush=True)
    return 0


BATCH_FORMATS = [(4, 3), (4, 4), (5, 7), (5, 10), (8, 7)]
FTZ_FORMATS = [(4, 3), (4, 4), (5, 7), (5, 10), (8, 7), (8, 23)]   # compiled with flush to zero too
MODE_NAMES = ["RN", "RZ", "RN_FTZ", "RZ_FTZ"]
SWEEP_OPS = ("add", "mul", "fma2", "div")


def batched_workload(bs, torch, njobs, lo, hi, seed, rank=0, formats=BATCH_FORMATS, ops=("add", "mul")):
    """njobs independent vectors: lengths log-uniform in [lo, hi], formats
    uniform over `formats`, ops uniform over `ops`, RN; operands drawn on the
    device and packed.  Returns (ctypes job array, njobs, tensors, elements,
    algorithmic bytes)."""
    lens = synth.log_uniform_lengths(njobs, lo, hi, seed, 2 * rank)
    r = synth.splitmix64(seed, 2 * njobs, 2 * rank + 1)
    std = {}
    specs, keep, elems, nbytes = [], [], 0, 0
    for i in range(njobs):
        E, M = formats[int(r[2 * i] % len(formats))]
        op = ops[int(r[2 * i + 1] % len(ops))]
        n = int(lens[i])
        f = bs.Format(E, M, RND)
        if (E, M) not in std:
            std[(E, M)] = bs.empty_standard(f, hi)
        planes = []
        for k in range(2):
            bs.bsfp_synth_fp_values(f, n, seed + 7919 * i + k, rank, 0, std[(E, M)])
            p = bs.empty_bitslice(f, n)
            bs.bsfp_pack(f, std[(E, M)], n, p)
            planes.append(p)
        out = bs.empty_bitslice(f, n)
        specs.append((f, op, planes[0], planes[1], None, out, n))
        keep += planes + [out]
        elems += n
        nbytes += 3 * (1 + E + M) * n / 8
    torch.cuda.synchronize()
    arr, nj = bs.make_jobs(specs)
    return arr, nj, keep, elems, nbytes


def run_batched(bs, torch, args, rank, hbm):
    """Batched plans -- the persistent kernels (one per op class), the
    streamed kernels (one per format and op class) and the unified streamed
    kernels (one per op class, every format) -- vs per-vector plain
    launches, in a graph and without, on one mixed workload (4,096 vectors,
    lengths log-uniform in [1,024, 4,194,304], formats uniform over the five
    batched formats, add/mul 50/50).  The speedups are those of the faster
    batched plan."""
    arr, nj, keep, elems, nbytes = batched_workload(bs, torch, args.batch_jobs, 1024, 1 << 22, 20160216, rank)
    stream = torch.cuda.current_stream()
    res = {"workload": "%d vectors, lengths log-uniform in [1024, 4194304], formats %s uniform, add/mul 50/50, RN"
                       % (nj, ["1/%d/%d" % fm for fm in BATCH_FORMATS]),
           "elements_per_step": elems, "algorithmic_bytes_per_step": nbytes}

    def timed(fn, steps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = bs.bsfp_launch_count()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, (bs.bsfp_launch_count() - l0) // steps

    variants = {}
    from paper_1602_04716_gb300 import tune
    wpt, bps = (args.batch_wpt, 0) if args.batch_wpt else tune.batch_shape()
    persistent = bs.BatchPlan(arr, nj, bs.BATCH_PERSISTENT, wpt, bps)
    variants["persistent_graph"] = timed(lambda: persistent.run(stream), args.batch_steps)
    streamed = bs.BatchPlan(arr, nj, bs.BATCH_STREAMED, wpt, bps)   # its persistent part takes the tuned shape
    variants["streamed_graph"] = timed(lambda: streamed.run(stream), args.batch_steps)
    unified = bs.BatchPlan(arr, nj, bs.BATCH_UNIFIED, wpt, bps)
    variants["unified_graph"] = timed(lambda: unified.run(stream), args.batch_steps)
    plain_graph = bs.BatchPlan(arr, nj, bs.BATCH_PLAIN)
    variants["plain_graph"] = timed(lambda: plain_graph.run(stream), args.batch_steps)
    variants["plain_launches"] = timed(lambda: bs.bsfp_launch_jobs(arr, nj, stream), args.batch_steps)
    for k, (ms, launches) in variants.items():
        res[k] = {"ms_per_step": ms, "elements_per_s": elems / (ms * 1e-3), "hbm_gbs": nbytes / (ms * 1e-3) / 1e9,
                  "hbm_frac": nbytes / (ms * 1e-3) / 1e9 / hbm, "launches_per_step": launches}
    best = min(("persistent_graph", "streamed_graph", "unified_graph"), key=lambda k: variants[k][0])
    res["best_batched"] = best
    res["speedup_vs_plain_graph"] = variants["plain_graph"][0] / variants[best][0]
    res["speedup_vs_plain_launches"] = variants["plain_launches"][0] / variants[best][0]
    persistent.free()
    streamed.free()
    unified.free()
    plain_graph.free()
    del keep
    return res


def run_serving(bs, torch, args, rank):
    """Serving loop: Poisson arrivals of bs_add/bs_mul requests (lengths
    log-uniform in [256, 2^22], formats uniform over the batched set, RN) on
    device-resident operands, results from a 64 GB budget, through the
    library's server (continuous batching); open-loop replay in native code."""
    pool = args.serve_pool
    arr, nj, keep, _, _ = batched_workload(bs, torch, pool, 256, 1 << 22, 19700101, rank)
    src = [arr[i] for i in range(nj)]
    out = {}
    runs = (("poisson", args.serve_rate, int(args.serve_rate * args.serve_seconds), 64 << 30),
            ("poisson_small_budget", args.serve_rate, int(args.serve_rate * 2), args.serve_small_budget),
            ("saturated", None, args.serve_saturated, 64 << 30))
    for name, rate, nreq, budget in runs:
        pick = synth.splitmix64(424242 + int(rate or 0), nreq, 2 * rank)
        jobs = (bs.bsfp_job * nreq)()
        elems = 0
        for i in range(nreq):
            j = src[int(pick[i] % nj)]
            jobs[i] = bs.bsfp_job(j.f, j.op, j.a, j.b, j.c, None, j.n)
            elems += j.n
        if rate:
            gaps = -np.log1p(-synth.uniform01(nreq, 8675309, 2 * rank)) / rate
            arrival = np.cumsum(gaps * 1e9).astype(np.int64)
        else:
            arrival = np.zeros(nreq, dtype=np.int64)
        srv = bs.Server(budget, slots=args.serve_slots)
        # warm-up: the first second of the same trace (at most 20,000 requests)
        w = min(nreq, int(rate or 20000))
        srv.replay(jobs, w, arrival[:w] - arrival[0], release=True)
        done = srv.replay(jobs, nreq, arrival, release=True, timeout_ms=120000)
        st = srv.stats()
        srv.close()
        sub = np.array([done[i].t_submit_ns for i in range(nreq)], dtype=np.int64)
        fin = np.array([done[i].t_done_ns for i in range(nreq)], dtype=np.int64)
        lat_us = (fin - sub) / 1e3
        span = (fin.max() - sub.min()) / 1e9
        out[name] = {"requests": nreq, "offered_requests_per_s": rate,
                     "achieved_requests_per_s": nreq / span, "elements_per_s": elems / span,
                     "latency_us": {"p50": float(np.percentile(lat_us, 50)), "p99": float(np.percentile(lat_us, 99)),
                                    "p999": float(np.percentile(lat_us, 99.9)), "max": float(lat_us.max())},
                     "budget_bytes": budget, "micro_batches": st["batches"],
                     "peak_inflight_batches": st["peak_inflight_batches"],
                     "arena_peak_bytes": st["arena_peak_bytes"], "failed": st["failed"]}
    out["workload"] = ("Poisson arrivals at %g requests/s for %g s after a 1 s warm-up, results from a 64 GB "
                       "budget (and the same arrivals for 2 s under a %d MB budget, and a saturated run of %d "
                       "requests arriving at once); bs_add/bs_mul 50/50, RN; lengths log-uniform in [256, 4194304]; "
                       "formats %s uniform; operands drawn from %d device-resident pairs; %d slots"
                       % (args.serve_rate, args.serve_seconds, args.serve_small_budget >> 20, args.serve_saturated,
                          ["1/%d/%d" % fm for fm in BATCH_FORMATS], pool, args.serve_slots))
    del keep
    return out


def run_conversions(bs, torch, n, hbm, reps=5):
    """bsfp_from_float (binary32 -> planes, RN), bsfp_to_float (planes ->
    binary32), bsfp_pack and bsfp_unpack for the two formats of the workload
    at n elements: CUDA-event time (median of 5 after a warm-up, DeviceTimer) and
    algorithmic GB/s (4 or the container bytes, + B/8 bytes per element)
    against the measured copy bandwidth."""
    stream = torch.cuda.current_stream()
    timer = DeviceTimer(torch, stream)
    src = torch.empty(n, dtype=torch.float32, device="cuda")
    bs.bsfp_synth_fp_values(bs.Format(8, 23, 0), n, 2024, 0, 0, src)
    back = torch.empty(n, dtype=torch.float32, device="cuda")
    out = {}
    for E, M in FORMATS:
        f = bs.Format(E, M, RND)
        planes = bs.empty_bitslice(f, n)
        std = bs.empty_standard(f, n)
        cb = bs.bsfp_container_bytes(f)
        for name, fn, bpe in (
                ("from_float", lambda: bs.bsfp_from_float(f, src, n, planes, stream=stream), 4),
                ("to_float", lambda: bs.bsfp_to_float(f, planes, n, back, stream=stream), 4),
                ("pack", lambda: bs.bsfp_pack(f, std, n, planes, stream=stream), cb),
                ("unpack", lambda: bs.bsfp_unpack(f, planes, n, std, stream=stream), cb)):
            t = timer.ms(fn, reps=reps) * 1e-3
            gbs = n * (bpe + (1 + E + M) / 8) / t / 1e9
            out["%s 1/%d/%d" % (name, E, M)] = {"ms": t * 1e3, "elements_per_s": n / t, "hbm_gbs": gbs,
                                                "hbm_frac": gbs / hbm}
        del planes, std
    out["workload"] = ("binary32 values of the workload recipe (1/8/23), %d elements, RN; pack/unpack of the "
                       "standard representation beside them" % n)
    return out


def run_integers(bs, torch, n, hbm, L):
    """Integer bitslice vectors (Sec. 3) at the widths the paper names (5, 9,
    13 and 17 bits): add and mul modulo 2^w on n-element vectors of uniform
    w-bit values; CUDA-event time (median of 5, DeviceTimer), GB/s of the algorithmic
    bytes (3w/8 per element) and the roofline fraction."""
    stream = torch.cuda.current_stream()
    timer = DeviceTimer(torch, stream)
    out = {}
    for w in (5, 9, 13, 17):
        # uniform random plane words are uniform random w-bit elements
        words = w * bs.bsfp_plane_stride(n)
        gen = torch.Generator(device="cuda").manual_seed(1602 + w)
        ops_ = [torch.randint(-2 ** 31, 2 ** 31 - 1, (words,), dtype=torch.int32, device="cuda", generator=gen)
                for _ in range(2)]
        res = torch.empty(words, dtype=torch.int32, device="cuda")
        for op in ("add", "mul"):
            t = timer.ms(lambda: bs.bsfp_int_op(op, w, ops_[0], ops_[1], res, n, stream=stream)) * 1e-3
            G = bs.bsfp_int_gate_count(w, op)
            bpe = 3 * w / 8
            roof = min(hbm * 1e9 / bpe, L * 32 / G)
            out["int%d_%s" % (w, op)] = {"ms": t * 1e3, "elements_per_s": n / t, "hbm_gbs": n * bpe / t / 1e9,
                                         "gates_per_word": G, "frac": (n / t) / roof,
                                         "bound": "hbm" if hbm * 1e9 / bpe <= L * 32 / G else "alu"}
        del ops_, res
    out["workload"] = "%d-element vectors of uniformly random w-bit integers, w in 5, 9, 13, 17" % n
    return out


def run_small_case(bs, torch, rank):
    """The 8-bit format 1/4/3 on all 65,536 operand pairs (a = i >> 8,
    b = i & 255): bs_add and bs_mul, RN and RZ, plus the pack/unpack round
    trip, as single launches; too small for a roofline, so latency only.

    Three figures per kernel.  `us`: one launch between CUDA events after an
    L2 flush (DeviceTimer), which carries the fixed device-side cost of any
    launch.  `floor_us`: the same measurement of a one-element fill, the cost
    of an empty launch; `over_floor_us` = `us` - `floor_us` is then the
    kernel's own time.  `back_to_back_us`: 64 launches in a row between two
    events, divided by 64 (warm L2, launch overheads overlapped)."""
    n = 1 << 16
    i = np.arange(n, dtype=np.uint32)
    out = {}
    stream = torch.cuda.current_stream()
    timer = DeviceTimer(torch, stream)
    tiny = torch.empty(1, dtype=torch.int32, device="cuda")
    floor = timer.ms(lambda: tiny.fill_(1), reps=20) * 1e3
    out["floor_us"] = floor

    def back_to_back(fn, k=64):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e3 / k

    def record(name, fn):
        us = timer.ms(fn, reps=20) * 1e3
        out[name] = {"us": us, "over_floor_us": us - floor, "back_to_back_us": back_to_back(fn)}

    for rnd in (0, 1):
        f = bs.Format(4, 3, rnd)
        std = [torch.from_numpy(x.astype(np.uint8)).cuda() for x in (i >> 8, i & 255)]
        planes = [bs.empty_bitslice(f, n) for _ in range(3)]
        back = bs.empty_standard(f, n)
        r = "RZ" if rnd else "RN"
        record("pack", lambda: bs.bsfp_pack(f, std[0], n, planes[0], stream=stream))
        bs.bsfp_pack(f, std[1], n, planes[1], stream=stream)
        for op in ("add", "mul"):
            record("%s_%s" % (op, r), lambda: bs.bsfp_op(op, f, planes[0], planes[1], planes[2], n, stream=stream))
        record("unpack", lambda: bs.bsfp_unpack(f, planes[0], n, back, stream=stream))
        assert torch.equal(back, std[0])
    out["workload"] = ("1/4/3, all 65,536 operand pairs, single launches: CUDA events around one launch after "
                       "an L2 flush (median of 20; host launch latency excluded), the same for a one-element "
                       "fill (floor_us), and 64 back-to-back launches per event pair")
    return out


def run_sweep(bs, torch, args, rank, hbm, L):
    """Format sweep: every 1/E/M with E in 3..8 and M in 2..23, n elements,
    bs_add, bs_mul, fma2 and bs_div under RN and RZ (and both with flush to zero for
    the formats compiled with it), operands from the same value
    recipe.  Per launch: CUDA-event time (median of 3 after one warm-up, L2
    flushed before each, host launch latency excluded: DeviceTimer), HBM
    GB/s of the algorithmic bytes, logic-op rate from the gate count, and the
    fraction of the roofline min(HBM peak / bytes per element, 32 * L / G).
    The RZ/RN ratios of time and gate count per op are the paper's one
    surviving quantitative claim (Sec. 5.2: RZ is markedly cheaper)."""
    n = args.sweep_n
    stream = torch.cuda.current_stream()
    timer = DeviceTimer(torch, stream)
    only = {tuple(int(x) for x in fm.split("/")) for fm in args.sweep_formats.split(",")} if args.sweep_formats \
        else None
    sweep_ops = tuple(op for op in SWEEP_OPS if op in args.sweep_ops.split(","))
    rows = []
    for E in range(3, 9):
        for M in range(2, 24):
            if only is not None and (E, M) not in only:
                continue
            B = 1 + E + M
            f0 = bs.Format(E, M, 0)
            std = bs.empty_standard(f0, n)
            ops_ = []
            for seed in (synth.SEED_A, synth.SEED_B, synth.SEED_C):
                bs.bsfp_synth_fp_values(f0, n, seed, rank, 0, std)
                p = bs.empty_bitslice(f0, n)
                bs.bsfp_pack(f0, std, n, p)
                ops_.append(p)
            out = bs.empty_bitslice(f0, n)
            modes = (0, 1, 2, 3) if (E, M) in FTZ_FORMATS else (0, 1)
            for rnd in modes:
                f = bs.Format(E, M, rnd)
                for op in sweep_ops:
                    t = timer.ms(lambda: bs.bsfp_op(op, f, ops_[0], ops_[1], out, n, c=ops_[2], stream=stream),
                                 reps=3) * 1e-3
                    nin = 3 if op == "fma2" else 2
                    bpe = (nin + 1) * B / 8
                    G = bs.bsfp_gate_count(f, op)
                    r_hbm = hbm * 1e9 / bpe
                    r_alu = L * 32 / G
                    rows.append({"fmt": "1/%d/%d" % (E, M), "rnd": MODE_NAMES[rnd], "op": op, "ms": t * 1e3,
                                 "elements_per_s": n / t, "hbm_gbs": n * bpe / t / 1e9, "gates_per_word": G,
                                 "logic_frac": G * n / 32 / t / L, "bound": "hbm" if r_hbm <= r_alu else "alu",
                                 "frac": (n / t) / min(r_hbm, r_alu)})
            del ops_, out, std
    summary = {"formats": len({r["fmt"] for r in rows}), "elements": n}
    if not rows:
        return summary
    for rnd in ("RN", "RZ"):
        for op in sweep_ops:
            sel = [r for r in rows if r["op"] == op and r["rnd"] == rnd]
            fr = np.array([r["frac"] for r in sel])
            summary["%s_%s" % (op, rnd)] = {"frac_min": float(fr.min()), "frac_median": float(np.median(fr)),
                                            "frac_max": float(fr.max()),
                                            "alu_bound_formats": sum(1 for r in sel if r["bound"] == "alu")}
    for op in sweep_ops:
        rn = {r["fmt"]: r for r in rows if r["op"] == op and r["rnd"] == "RN"}
        rz = {r["fmt"]: r for r in rows if r["op"] == op and r["rnd"] == "RZ"}
        tr = np.array([rz[k]["ms"] / rn[k]["ms"] for k in rn])
        gr = np.array([rz[k]["gates_per_word"] / rn[k]["gates_per_word"] for k in rn])
        summary["rz_over_rn_%s" % op] = {"time_median": float(np.median(tr)), "time_min": float(tr.min()),
                                         "gates_median": float(np.median(gr)), "gates_min": float(gr.min())}
    # flush to zero against gradual underflow, on the formats compiled with it
    for op in sweep_ops:
        pl = {r["fmt"]: r for r in rows if r["op"] == op and r["rnd"] == "RN"}
        fz = {r["fmt"]: r for r in rows if r["op"] == op and r["rnd"] == "RN_FTZ"}
        summary["ftz_over_rn_%s" % op] = {k: {"time": fz[k]["ms"] / pl[k]["ms"],
                                              "gates": fz[k]["gates_per_word"] / pl[k]["gates_per_word"]}
                                          for k in fz}
    if args.sweep_out:
        with open(args.sweep_out, "w") as fh:
            json.dump({"summary": summary, "rows": rows}, fh, indent=1)
        summary["table"] = args.sweep_out
    return summary


def host_link_rates(torch, pinned, reps=3):
    """Plain copy rates of this machine's host link: one page-locked host buffer
    to the device and back, best of `reps` (CUDA events on the current
    stream).  Recorded beside the end-to-end figure, which the link bounds,
    so that the end-to-end numbers of different boxes can be compared."""
    dev = torch.empty_like(pinned, device="cuda")
    nbytes = pinned.numel() * pinned.element_size()
    best = {"h2d": float("inf"), "d2h": float("inf")}
    for _ in range(reps):
        for kind in ("h2d", "d2h"):
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record()
            if kind == "h2d":
                dev.copy_(pinned, non_blocking=True)
            else:
                pinned.copy_(dev, non_blocking=True)
            t1.record()
            t1.synchronize()
            best[kind] = min(best[kind], t0.elapsed_time(t1))
    # both directions at once, on two streams (the pipeline overlaps them)
    dev2 = torch.empty_like(pinned, device="cuda")
    back = torch.empty_like(pinned).pin_memory()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    both = float("inf")
    for _ in range(reps):
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        s1.wait_event(t0)
        s2.wait_event(t0)
        with torch.cuda.stream(s1):
            dev.copy_(pinned, non_blocking=True)
        with torch.cuda.stream(s2):
            back.copy_(dev2, non_blocking=True)
        torch.cuda.current_stream().wait_stream(s1)
        torch.cuda.current_stream().wait_stream(s2)
        t1.record()
        t1.synchronize()
        both = min(both, t0.elapsed_time(t1))
    del dev, dev2, back
    return {"bytes": nbytes, "h2d_gbs": nbytes / best["h2d"] / 1e6, "d2h_gbs": nbytes / best["d2h"] / 1e6,
            "both_directions_gbs": 2 * nbytes / both / 1e6}


def run_e2e(bs, torch, n, rank, args):
    """Per step, for both formats: the two operand vectors in page-locked host
    memory (standard form) through the host-to-host pipeline -- chunked copy
    in, pack, bs_add and bs_mul, unpack, copy out over rotating streams --
    into two result vectors in page-locked host memory.  Both formats are
    submitted back to back (bsfp_pipeline_submit) and the step waits once for
    all four results (bsfp_pipeline_wait)."""
    host_in, host_out = {}, {}
    for E, M in FORMATS:
        f = bs.Format(E, M, RND)
        ins = []
        for seed in (synth.SEED_A, synth.SEED_B):
            d = bs.empty_standard(f, n)
            bs.bsfp_synth_fp_values(f, n, seed, rank, 0, d)
            h = torch.empty(n, dtype=d.dtype, pin_memory=True)
            h.copy_(d)
            ins.append(h)
            del d
        host_in[(E, M)] = ins
        host_out[(E, M)] = [torch.empty(n, dtype=ins[0].dtype, pin_memory=True) for _ in OPS]
    torch.cuda.synchronize()
    pipe = bs.Pipeline(args.e2e_chunk, args.e2e_depth)
    h2d = d2h = 0

    def step():
        nonlocal h2d, d2h
        h2d = d2h = 0
        for E, M in FORMATS:
            f = bs.Format(E, M, RND)
            (ha, hb), outs = host_in[(E, M)], host_out[(E, M)]
            pipe.submit(f, OPS, ha, hb, outs, n)
            h2d += 2 * ha.numel() * ha.element_size()
            d2h += sum(o.numel() * o.element_size() for o in outs)
        pipe.wait()

    for _ in range(max(1, min(args.warmup, 2))):
        step()
    torch.cuda.synchronize()
    k = max(1, args.e2e_steps)
    per_step = []
    t = time.perf_counter()
    for _ in range(k):
        t1 = time.perf_counter()
        step()
        per_step.append((time.perf_counter() - t1) * 1e3)
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t) / k
    pipe.close()
    link = host_link_rates(torch, host_in[FORMATS[-1]][0])
    link_ms = 1e3 * (h2d / (link["h2d_gbs"] * 1e9) + d2h / (link["d2h_gbs"] * 1e9))
    link["serial_copy_ms_per_step"] = link_ms
    link["overlapped_copy_ms_per_step"] = 1e3 * (h2d + d2h) / (link["both_directions_gbs"] * 1e9)
    return {"value": len(FORMATS) * len(OPS) * n / sec, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": sec * 1e3, "steps": k, "step_ms": per_step,
            "median_step_ms": float(np.median(per_step)),
            "host_link": link,
            "path": "pinned host -> bsfp_pipeline_submit per format, one bsfp_pipeline_wait per step (chunks "
                    "of %d over %d streams: H2D, bsfp_pack, bsfp_add + bsfp_mul, bsfp_unpack, D2H) -> pinned host"
                    % (args.e2e_chunk or (1 << 24), args.e2e_depth or 4)}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000,
                    help="timed steps (the default spans about 0.7 s, several clock samples)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["bsfp", "reference"], default="bsfp")
    ap.add_argument("--n", type=int, default=N, help="elements per vector (default 2^28)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20,
                    help="timed end-to-end steps (about 14 ms each); the value is their mean, so one slow step "
                         "on a busy host weighs 1/steps")
    ap.add_argument("--e2e-chunk", type=int, default=0, help="pipeline chunk (elements; 0 = library default)")
    ap.add_argument("--e2e-depth", type=int, default=0, help="pipeline streams (0 = library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-sample", type=int, default=1 << 23,
                    help="reference arm: elements per vector per step")
    ap.add_argument("--batch-jobs", type=int, default=4096,
                    help="vectors in the batched comparison (0 skips it)")
    ap.add_argument("--batch-steps", type=int, default=10)
    ap.add_argument("--batch-wpt", type=int, default=0)
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="Poisson serving run length (0 skips it)")
    ap.add_argument("--serve-small-budget", type=int, default=16 << 20, help="bytes, the back-pressure run")
    ap.add_argument("--serve-rate", type=float, default=20000.0, help="requests/s")
    ap.add_argument("--serve-saturated", type=int, default=20000, help="requests in the saturated run")
    ap.add_argument("--serve-pool", type=int, default=2048, help="device-resident operand pairs")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--sweep-n", type=int, default=1 << 26,
                    help="elements per vector in the format sweep (0 skips it)")
    ap.add_argument("--sweep-out", default=None, help="write the full sweep table (JSON) here")
    ap.add_argument("--sweep-formats", default="",
                    help="comma-separated E/M (e.g. 4/7,6/7): sweep only these formats (default: all)")
    ap.add_argument("--sweep-ops", default=",".join(SWEEP_OPS), help="comma-separated ops of the sweep")
    ap.add_argument("--section", default=None,
                    choices=["conversions", "small", "integers", "sweep", "batched", "serving", "e2e"],
                    help="run only this section of the bench and print it (no main timed loop)")
    ap.add_argument("--section-reps", type=int, default=5, help="timed launches per kernel in --section conversions")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
