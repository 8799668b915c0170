"""Autotuner for the element-wise kernels' launch shape.

For a (format, op) it times every compiled words-per-thread variant at a few
resident-block counts on caller-supplied device operands, with CUDA events on
the launching stream, and keeps the fastest.  Results persist as JSON keyed
by GPU name, format and op, so a later process applies them without timing.
The kernels are straight-line circuits with no data-dependent branches, so
the timing does not depend on operand values.
"""
from __future__ import annotations

import json
import os

from . import bsfp as _b

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")


def _key(f, op) -> str:
    return "%d/%d/%d/%s" % (f.exp_bits, f.man_bits, f.rnd, op)


def gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(0)


def load(path: str = CACHE) -> dict:
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        return json.load(fh)


def save(cache: dict, path: str = CACHE):
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(path: str = CACHE) -> int:
    """Apply every cached shape for this GPU; returns how many were applied."""
    cache = load(path).get(gpu_name(), {})
    n = 0
    for key, v in cache.items():
        e, m, r, op = key.split("/")
        f = _b.Format(int(e), int(m), int(r))
        if v["wpt"] in _b.bsfp_variants_compiled(f, op):
            _b.bsfp_set_variant(f, op, v["wpt"], v["bps"])
            n += 1
    return n


def time_op(op, f, a, b, c, out, n, reps=5) -> float:
    """Median milliseconds of one launch."""
    import torch
    s = torch.cuda.current_stream()
    ts = []
    for _ in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        _b.bsfp_op(op, f, a, b, out, n, c=c)
        e1.record(s)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ts = sorted(ts[1:])
    return ts[len(ts) // 2]


def autotune(op, f, a, b, c, out, n, bps_choices=(0, 1, 2, 3, 4, 6, 8), reps=5, path: str | None = CACHE):
    """Time every (wpt, blocks/SM) shape; set and (optionally) persist the best.
    Returns (best, table) where table maps (wpt, bps) -> ms."""
    table = {}
    for wpt in _b.bsfp_variants_compiled(f, op):
        for bps in bps_choices:
            _b.bsfp_set_variant(f, op, wpt, bps)
            table[(wpt, bps)] = time_op(op, f, a, b, c, out, n, reps)
    best = min(table, key=table.get)
    _b.bsfp_set_variant(f, op, best[0], best[1])
    if path:
        cache = load(path)
        cache.setdefault(gpu_name(), {})[_key(f, op)] = {"wpt": best[0], "bps": best[1], "ms": table[best], "n": n}
        save(cache, path)
    return best, table
