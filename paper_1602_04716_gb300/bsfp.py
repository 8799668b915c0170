"""Thin ctypes binding of libbsfp (include/bsfp.h, include/bsfp_bench.h).

Argument marshalling only: every step of pack, unpack and the arithmetic runs
in the library's CUDA kernels.  Tensors are passed by ``data_ptr()``; torch
supplies device memory and the current stream and nothing else.  A non-zero
status raises ``BsfpError``.  If the library has not been built, every call
fails loudly: there is no other implementation to fall back on.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbsfp.so")

RN, RZ, RN_FTZ, RZ_FTZ = 0, 1, 2, 3
OP_ADD, OP_SUB, OP_MUL, OP_FMA2, OP_DIV = 0, 1, 2, 3, 4
OPS = {"add": OP_ADD, "sub": OP_SUB, "mul": OP_MUL, "fma2": OP_FMA2, "div": OP_DIV}

OK = 0
ERR_FORMAT, ERR_NULL, ERR_ALIGN, ERR_SIZE, ERR_UNSUPPORTED, ERR_CUDA, ERR_BUDGET, ERR_TIMEOUT = range(-1, -9, -1)
VARIANT_STREAMED = 8
PROBE_LOP3_PER_ROUND = 64
MAX_N = 1 << 40


class BsfpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = "%s: %s (%d)" % (where, status_str(status), status)
        if status == ERR_CUDA:
            msg += " [cudaError %d]" % _lib().bsfp_last_cuda_error()
        super().__init__(msg)


class bsfp_format(ctypes.Structure):
    """Format 1/E/M with a rounding mode (RN = 0, RZ = 1)."""
    _fields_ = [("exp_bits", ctypes.c_int32), ("man_bits", ctypes.c_int32), ("rnd", ctypes.c_int32)]

    def __init__(self, exp_bits: int, man_bits: int, rnd: int = RN):
        super().__init__(exp_bits, man_bits, rnd)

    @property
    def bits(self) -> int:
        return 1 + self.exp_bits + self.man_bits

    def __repr__(self):
        return "bsfp_format(1/%d/%d, %s)" % (self.exp_bits, self.man_bits,
                                             ("RN", "RZ", "RN_FTZ", "RZ_FTZ")[self.rnd] if 0 <= self.rnd < 4
                                             else str(self.rnd))


Format = bsfp_format


class bsfp_job(ctypes.Structure):
    """One element-wise op on one vector (a unit of a batch)."""
    _fields_ = [("f", bsfp_format), ("op", ctypes.c_int32), ("a", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("c", ctypes.c_void_p), ("out", ctypes.c_void_p), ("n", ctypes.c_int64)]


class bsfp_batch_options(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("wpt", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32)]


class bsfp_server_options(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("slots", ctypes.c_int32), ("max_batch_jobs", ctypes.c_int32),
                ("max_batch_tiles", ctypes.c_int32), ("wpt", ctypes.c_int32), ("eager_slots", ctypes.c_int32),
                ("min_batch_tiles", ctypes.c_int32), ("batch_wait_us", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class bsfp_completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("out", ctypes.c_void_p), ("n", ctypes.c_int64), ("t_submit_ns", ctypes.c_int64),
                ("t_admit_ns", ctypes.c_int64), ("t_done_ns", ctypes.c_int64)]


class bsfp_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "submitted", "completed", "failed", "pending", "inflight_batches", "batches", "peak_inflight_batches",
        "arena_bytes_in_use", "arena_peak_bytes", "budget_bytes", "launches")]


BATCH_PERSISTENT, BATCH_PLAIN, BATCH_STREAMED, BATCH_UNIFIED = 0, 1, 2, 3
BATCH_FORMATS = [(4, 3), (4, 4), (5, 7), (5, 10), (8, 7)]

_lock = threading.Lock()
_L = None


def _lib():
    global _L
    if _L is not None:
        return _L
    with _lock:
        if _L is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libbsfp.so is not built (%s); run __graft_entry__.build() or "
                                   "python -m paper_1602_04716_gb300.build" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            i32, i64, u32, u64, p = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
            F = bsfp_format
            sig = {
                "bsfp_plane_stride": (i64, [i64]),
                "bsfp_bitslice_bytes": (i64, [F, i64]),
                "bsfp_container_bytes": (i32, [F]),
                "bsfp_pack": (i32, [F, p, i64, p, p]),
                "bsfp_unpack": (i32, [F, p, i64, p, p]),
                "bsfp_add": (i32, [F, p, p, p, i64, p]),
                "bsfp_sub": (i32, [F, p, p, p, i64, p]),
                "bsfp_mul": (i32, [F, p, p, p, i64, p]),
                "bsfp_fma2": (i32, [F, p, p, p, p, i64, p]),
                "bsfp_div": (i32, [F, p, p, p, i64, p]),
                "bsfp_from_float": (i32, [F, i32, p, i64, p, p]),
                "bsfp_int_pack": (i32, [i32, p, i64, p, p]),
                "bsfp_int_unpack": (i32, [i32, p, i64, p, p]),
                "bsfp_int_add": (i32, [i32, p, p, p, i64, p]),
                "bsfp_int_sub": (i32, [i32, p, p, p, i64, p]),
                "bsfp_int_mul": (i32, [i32, p, p, p, i64, p]),
                "bsfp_int_gate_count": (i64, [i32, i32]),
                "bsfp_autotune": (i32, [F, i32, ctypes.c_char_p]),
                "bsfp_autotune_load": (i32, [ctypes.c_char_p]),
                "bsfp_to_float": (i32, [F, p, i64, p, p]),
                "bsfp_status_str": (ctypes.c_char_p, [i32]),
                "bsfp_last_cuda_error": (i32, []),
                "bsfp_gate_count": (i64, [F, i32]),
                "bsfp_variant": (i32, [F, i32]),
                "bsfp_variants_compiled": (i32, [F, i32]),
                "bsfp_set_variant": (i32, [F, i32, i32, i32]),
                "bsfp_launch_count": (i64, []),
                "bsfp_fault_status": (i32, [i32]),
                "bsfp_variant_for": (i32, [F, i32, i64]),
                "bsfp_stream_shape": (i32, [F, i32, ctypes.c_void_p, ctypes.c_void_p]),
                "bsfp_set_stream_min_tiles": (i32, [i32]),
                "bsfp_set_batch_stream_min_tiles": (i32, [i32]),
                "bsfp_stream_selftest": (i32, [F, i32, p, p, p, i64, i64, i64, p]),
                "bsfp_synth_fp_values": (i32, [F, i64, u64, u64, i64, p, p]),
                "bsfp_lop3_probe": (i32, [p, i32, i32, i32, u32, p]),
                "bsfp_num_sms": (i32, []),
                "bsfp_batch_plan_create": (i32, [ctypes.POINTER(bsfp_job), i32, ctypes.POINTER(bsfp_batch_options),
                                                 ctypes.POINTER(p)]),
                "bsfp_batch_run": (i32, [p, p]),
                "bsfp_batch_launches": (i64, [p]),
                "bsfp_batch_free": (None, [p]),
                "bsfp_launch_jobs": (i32, [ctypes.POINTER(bsfp_job), i32, p]),
                "bsfp_batch_run_noalloc": (i32, [ctypes.POINTER(bsfp_job), i32, p]),
                "bsfp_pipeline_create": (i32, [i64, i32, ctypes.POINTER(p)]),
                "bsfp_pipeline_run": (i32, [p, F, i32, ctypes.POINTER(i32), p, p, p, ctypes.POINTER(p), i64]),
                "bsfp_pipeline_submit": (i32, [p, F, i32, ctypes.POINTER(i32), p, p, p, ctypes.POINTER(p), i64]),
                "bsfp_pipeline_wait": (i32, [p]),
                "bsfp_pipeline_free": (None, [p]),
                "bsfp_server_create": (i32, [ctypes.POINTER(bsfp_server_options), ctypes.POINTER(p)]),
                "bsfp_server_submit": (i32, [p, ctypes.POINTER(bsfp_job), ctypes.POINTER(i64)]),
                "bsfp_server_submit_n": (i32, [p, ctypes.POINTER(bsfp_job), i32, ctypes.POINTER(i64),
                                               ctypes.POINTER(i32)]),
                "bsfp_server_poll": (i32, [p, ctypes.POINTER(bsfp_completion), i32]),
                "bsfp_server_release": (i32, [p, i64]),
                "bsfp_server_drain": (i32, [p, i64]),
                "bsfp_server_get_stats": (i32, [p, ctypes.POINTER(bsfp_server_stats)]),
                "bsfp_server_destroy": (None, [p]),
                "bsfp_server_replay": (i32, [p, ctypes.POINTER(bsfp_job), ctypes.POINTER(i64), i32, i32,
                                             ctypes.POINTER(bsfp_completion), i64]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _L = L
    return _L


def lib_path() -> str:
    return LIB_PATH


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(status: int, where: str):
    if status != OK:
        raise BsfpError(status, where)


def _fmt(f) -> bsfp_format:
    if isinstance(f, bsfp_format):
        return f
    e, m, *r = f
    return bsfp_format(e, m, r[0] if r else RN)


# ---------------------------------------------------------------- sizes ---
def bsfp_plane_stride(n: int) -> int:
    return int(_lib().bsfp_plane_stride(n))


def bsfp_bitslice_bytes(f, n: int) -> int:
    return int(_lib().bsfp_bitslice_bytes(_fmt(f), n))


def bsfp_container_bytes(f) -> int:
    return int(_lib().bsfp_container_bytes(_fmt(f)))


# ------------------------------------------------------- pack / unpack ---
def bsfp_pack(f, std_in, n: int, bs_out, stream=None):
    _check(_lib().bsfp_pack(_fmt(f), _ptr(std_in), n, _ptr(bs_out), _stream(stream)), "bsfp_pack")


def bsfp_unpack(f, bs_in, n: int, std_out, stream=None):
    _check(_lib().bsfp_unpack(_fmt(f), _ptr(bs_in), n, _ptr(std_out), _stream(stream)), "bsfp_unpack")


# ------------------------------------------------------------------ ops ---
def bsfp_add(f, a, b, out, n: int, stream=None):
    _check(_lib().bsfp_add(_fmt(f), _ptr(a), _ptr(b), _ptr(out), n, _stream(stream)), "bsfp_add")


def bsfp_sub(f, a, b, out, n: int, stream=None):
    _check(_lib().bsfp_sub(_fmt(f), _ptr(a), _ptr(b), _ptr(out), n, _stream(stream)), "bsfp_sub")


def bsfp_mul(f, a, b, out, n: int, stream=None):
    _check(_lib().bsfp_mul(_fmt(f), _ptr(a), _ptr(b), _ptr(out), n, _stream(stream)), "bsfp_mul")


def bsfp_fma2(f, a, b, c, out, n: int, stream=None):
    _check(_lib().bsfp_fma2(_fmt(f), _ptr(a), _ptr(b), _ptr(c), _ptr(out), n, _stream(stream)), "bsfp_fma2")


def bsfp_div(f, a, b, out, n: int, stream=None):
    _check(_lib().bsfp_div(_fmt(f), _ptr(a), _ptr(b), _ptr(out), n, _stream(stream)), "bsfp_div")


def bsfp_op(op: str, f, a, b, out, n: int, c=None, stream=None):
    """Dispatch by name: add, sub, mul, fma2 or div."""
    if op == "fma2":
        return bsfp_fma2(f, a, b, c, out, n, stream)
    return {"add": bsfp_add, "sub": bsfp_sub, "mul": bsfp_mul, "div": bsfp_div}[op](f, a, b, out, n, stream)


# ---------------------------------------------------------- conversions ---
FLOAT32, BFLOAT16, FLOAT16 = 0, 1, 2


def float_type_of(t) -> int:
    """bsfp_float_type of a torch tensor (float32, bfloat16 or float16)."""
    import torch
    return {torch.float32: FLOAT32, torch.bfloat16: BFLOAT16, torch.float16: FLOAT16}[t.dtype]


def bsfp_from_float(f, src, n: int, bs_out, src_type=None, stream=None):
    """Native floats (a device tensor of float32 / bfloat16 / float16, or a
    pointer with src_type) -> bitslice planes of format f, rounded once."""
    t = float_type_of(src) if src_type is None else src_type
    _check(_lib().bsfp_from_float(_fmt(f), t, _ptr(src), n, _ptr(bs_out), _stream(stream)), "bsfp_from_float")


def bsfp_to_float(f, bs_in, n: int, out, stream=None):
    """Bitslice planes of format f -> float32 (exact)."""
    _check(_lib().bsfp_to_float(_fmt(f), _ptr(bs_in), n, _ptr(out), _stream(stream)), "bsfp_to_float")


# ------------------------------------------------ integer vectors (Sec. 3) ---
INT_OPS = {"add": 0, "sub": 1, "mul": 2}


def bsfp_int_pack(bits: int, std_in, n: int, bs_out, stream=None):
    _check(_lib().bsfp_int_pack(bits, _ptr(std_in), n, _ptr(bs_out), _stream(stream)), "bsfp_int_pack")


def bsfp_int_unpack(bits: int, bs_in, n: int, std_out, stream=None):
    _check(_lib().bsfp_int_unpack(bits, _ptr(bs_in), n, _ptr(std_out), _stream(stream)), "bsfp_int_unpack")


def bsfp_int_op(op: str, bits: int, a, b, out, n: int, stream=None):
    """w-bit integer vectors: op in {add, sub, mul}, modulo 2^bits."""
    fn = {"add": _lib().bsfp_int_add, "sub": _lib().bsfp_int_sub, "mul": _lib().bsfp_int_mul}[op]
    _check(fn(bits, _ptr(a), _ptr(b), _ptr(out), n, _stream(stream)), "bsfp_int_" + op)


def bsfp_int_gate_count(bits: int, op) -> int:
    return int(_lib().bsfp_int_gate_count(bits, INT_OPS.get(op, op)))


def empty_int_bitslice(bits: int, n: int, device="cuda"):
    import torch
    return torch.empty(bits * bsfp_plane_stride(n), dtype=torch.int32, device=device)


# ---------------------------------------------------------- diagnostics ---
def status_str(status: int) -> str:
    return _lib().bsfp_status_str(status).decode()


bsfp_status_str = status_str


def bsfp_last_cuda_error() -> int:
    return int(_lib().bsfp_last_cuda_error())


def bsfp_gate_count(f, op) -> int:
    return int(_lib().bsfp_gate_count(_fmt(f), OPS.get(op, op)))


def bsfp_variant(f, op) -> int:
    return int(_lib().bsfp_variant(_fmt(f), OPS.get(op, op)))


def bsfp_variants_compiled(f, op) -> list:
    """Variants compiled for (f, op): words per thread 1, 2, 4 of the
    grid-stride kernel and VARIANT_STREAMED (8) for the streamed kernel."""
    m = int(_lib().bsfp_variants_compiled(_fmt(f), OPS.get(op, op)))
    return [w for i, w in enumerate((1, 2, 4, VARIANT_STREAMED)) if m > 0 and (m >> i) & 1]


def bsfp_variant_for(f, op, n: int) -> int:
    """The variant a call of (f, op) on n elements launches."""
    return int(_lib().bsfp_variant_for(_fmt(f), OPS.get(op, op), n))


def bsfp_stream_shape(f, op) -> tuple:
    """(tile words, ring stages) of the streamed kernel of (f, op)."""
    tw, st = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(_lib().bsfp_stream_shape(_fmt(f), OPS.get(op, op), ctypes.addressof(tw), ctypes.addressof(st)),
           "bsfp_stream_shape")
    return tw.value, st.value


def bsfp_stream_selftest(f, op, a, b, out, n: int, withhold_tile: int, wait_cycles: int, stream=None):
    """Streamed kernel with one tile's copies withheld and a short wait bound
    (the failure path of its bounded waits)."""
    _check(_lib().bsfp_stream_selftest(_fmt(f), OPS.get(op, op), _ptr(a), _ptr(b), _ptr(out), n, withhold_tile,
                                       wait_cycles, _stream(stream)), "bsfp_stream_selftest")


def bsfp_set_batch_stream_min_tiles(tiles_per_sm: int):
    _check(_lib().bsfp_set_batch_stream_min_tiles(tiles_per_sm), "bsfp_set_batch_stream_min_tiles")


def bsfp_set_stream_min_tiles(tiles_per_sm: int):
    _check(_lib().bsfp_set_stream_min_tiles(tiles_per_sm), "bsfp_set_stream_min_tiles")


def bsfp_fault_status(clear: bool = False) -> int:
    """The current device's fault word (0: none; 1: a streamed kernel gave up
    a bounded wait).  Synchronises the device."""
    v = int(_lib().bsfp_fault_status(1 if clear else 0))
    if v < 0:
        raise BsfpError(ERR_CUDA, "bsfp_fault_status")
    return v


def bsfp_set_variant(f, op, wpt: int, blocks_per_sm: int = 0):
    _check(_lib().bsfp_set_variant(_fmt(f), OPS.get(op, op), wpt, blocks_per_sm), "bsfp_set_variant")


def bsfp_autotune(f, op, cache_path: str | None = None):
    """Native autotuner: time every compiled shape of (f, op) at 2^28 elements,
    apply the fastest, optionally record it in a text cache."""
    _check(_lib().bsfp_autotune(_fmt(f), OPS.get(op, op), cache_path.encode() if cache_path else None),
           "bsfp_autotune")


def bsfp_autotune_load(cache_path: str) -> int:
    return int(_lib().bsfp_autotune_load(cache_path.encode()))


def bsfp_launch_count() -> int:
    return int(_lib().bsfp_launch_count())


# -------------------------------------------------------------- batched ---
def make_jobs(specs):
    """specs: iterable of (format, op, a, b, c, out, n) -> ctypes array of bsfp_job."""
    specs = list(specs)
    arr = (bsfp_job * max(1, len(specs)))()
    for i, (f, op, a, b, c, out, n) in enumerate(specs):
        arr[i] = bsfp_job(_fmt(f), OPS.get(op, op), _ptr(a), _ptr(b), _ptr(c), _ptr(out), n)
    return arr, len(specs)


class BatchPlan:
    """Owns a bsfp_batch_plan; the tensors the jobs point at must outlive it."""

    def __init__(self, jobs, njobs: int, mode: int = BATCH_PERSISTENT, wpt: int = 0, blocks_per_sm: int = 0):
        self._h = ctypes.c_void_p()
        opt = bsfp_batch_options(mode, wpt, blocks_per_sm)
        _check(_lib().bsfp_batch_plan_create(jobs, njobs, ctypes.byref(opt), ctypes.byref(self._h)),
               "bsfp_batch_plan_create")

    def run(self, stream=None):
        _check(_lib().bsfp_batch_run(self._h, _stream(stream)), "bsfp_batch_run")

    @property
    def launches(self) -> int:
        return int(_lib().bsfp_batch_launches(self._h))

    def free(self):
        if self._h:
            _lib().bsfp_batch_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def bsfp_batch_plan_create(jobs, njobs: int, mode: int = BATCH_PERSISTENT, wpt: int = 0,
                           blocks_per_sm: int = 0) -> BatchPlan:
    return BatchPlan(jobs, njobs, mode, wpt, blocks_per_sm)


def bsfp_launch_jobs(jobs, njobs: int, stream=None):
    _check(_lib().bsfp_launch_jobs(jobs, njobs, _stream(stream)), "bsfp_launch_jobs")


NOALLOC_MAX_JOBS, NOALLOC_MAX_TILES = 4096, 1 << 18


def bsfp_batch_run_noalloc(jobs, njobs: int, stream=None):
    """The batched launch with its scratch in the library's fixed device array
    (no allocation); for callers that must not allocate device memory."""
    _check(_lib().bsfp_batch_run_noalloc(jobs, njobs, _stream(stream)), "bsfp_batch_run_noalloc")


# ---------------------------------------------------- host-to-host path ---
PIPE_MAX_OPS = 4


def _host_ptr(x):
    """Address of a host array: a CPU torch tensor or a numpy array."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        assert not x.is_cuda, "host-to-host path: pass host arrays"
        return x.data_ptr()
    return x.ctypes.data


class Pipeline:
    """Owns a bsfp_pipeline: standard arrays in host memory through the GPU
    path and back, in chunks over several streams."""

    def __init__(self, chunk: int = 0, depth: int = 0):
        self._h = ctypes.c_void_p()
        _check(_lib().bsfp_pipeline_create(chunk, depth, ctypes.byref(self._h)), "bsfp_pipeline_create")

    def _call(self, fn, f, ops, a, b, outs, n, c):
        ops = [OPS.get(o, o) for o in ops]
        arr = (ctypes.c_int32 * len(ops))(*ops)
        optr = (ctypes.c_void_p * len(outs))(*[_host_ptr(o) for o in outs])
        _check(getattr(_lib(), fn)(self._h, _fmt(f), len(ops), arr, _host_ptr(a), _host_ptr(b), _host_ptr(c),
                                   optr, n), fn)

    def run(self, f, ops, a, b, outs, n: int, c=None):
        """outs[q] = ops[q](a, b [, c]) on host arrays; returns when done."""
        self._call("bsfp_pipeline_run", f, ops, a, b, outs, n, c)

    def submit(self, f, ops, a, b, outs, n: int, c=None):
        """As run, but returns once the work is enqueued: the arrays must stay
        untouched until wait() returns."""
        self._call("bsfp_pipeline_submit", f, ops, a, b, outs, n, c)

    def wait(self):
        _check(_lib().bsfp_pipeline_wait(self._h), "bsfp_pipeline_wait")

    def close(self):
        if self._h:
            _lib().bsfp_pipeline_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# -------------------------------------------------------------- serving ---
class Server:
    """Owns a bsfp_server (continuous batching of requests on device-resident
    operands).  Operand tensors must outlive the requests that use them."""

    def __init__(self, budget_bytes: int, slots: int = 0, max_batch_jobs: int = 0, max_batch_tiles: int = 0,
                 wpt: int = 0, eager_slots: int = 0, min_batch_tiles: int = 0, batch_wait_us: int = 0):
        self._h = ctypes.c_void_p()
        opt = bsfp_server_options(budget_bytes, slots, max_batch_jobs, max_batch_tiles, wpt, eager_slots,
                                  min_batch_tiles, batch_wait_us, 0)
        _check(_lib().bsfp_server_create(ctypes.byref(opt), ctypes.byref(self._h)), "bsfp_server_create")

    def submit(self, f, op, a, b, n: int, c=None, out=None) -> int:
        job = bsfp_job(_fmt(f), OPS.get(op, op), _ptr(a), _ptr(b), _ptr(c), _ptr(out), n)
        rid = ctypes.c_int64()
        _check(_lib().bsfp_server_submit(self._h, ctypes.byref(job), ctypes.byref(rid)), "bsfp_server_submit")
        return rid.value

    def submit_n(self, jobs, njobs: int) -> list:
        """Submit a ctypes array of bsfp_job in one call; returns the ids."""
        ids = (ctypes.c_int64 * max(1, njobs))()
        bad = ctypes.c_int32(-1)
        _check(_lib().bsfp_server_submit_n(self._h, jobs, njobs, ids, ctypes.byref(bad)), "bsfp_server_submit_n")
        return [ids[i] for i in range(njobs)]

    def poll(self, max_items: int = 256) -> list:
        buf = (bsfp_completion * max_items)()
        k = _lib().bsfp_server_poll(self._h, buf, max_items)
        return [buf[i] for i in range(k)]

    def release(self, rid: int):
        _check(_lib().bsfp_server_release(self._h, rid), "bsfp_server_release")

    def drain(self, timeout_ms: int = 10000):
        _check(_lib().bsfp_server_drain(self._h, timeout_ms), "bsfp_server_drain")

    def stats(self) -> dict:
        st = bsfp_server_stats()
        _check(_lib().bsfp_server_get_stats(self._h, ctypes.byref(st)), "bsfp_server_get_stats")
        return {k: getattr(st, k) for k, _ in bsfp_server_stats._fields_}

    def replay(self, jobs, njobs: int, arrival_ns, release: bool = True, timeout_ms: int = 60000):
        """Open-loop replay; arrival_ns: int64 numpy array.  Returns the
        ctypes array of completions, one per job in submission order."""
        import numpy as np
        arr = np.ascontiguousarray(arrival_ns, dtype=np.int64)
        done = (bsfp_completion * max(1, njobs))()
        _check(_lib().bsfp_server_replay(self._h, jobs, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), njobs,
                                         1 if release else 0, done, timeout_ms), "bsfp_server_replay")
        return done

    @staticmethod
    def result(c: "bsfp_completion", f):
        """The result planes of a finished request as an int32 device tensor
        (a view of server memory: valid until the request is released)."""
        import torch
        words = _fmt(f).bits * bsfp_plane_stride(c.n)
        if words == 0:
            return torch.empty(0, dtype=torch.int32, device="cuda")

        class _View:
            __cuda_array_interface__ = {"shape": (words,), "typestr": "<i4", "data": (c.out, False), "version": 3}
        return torch.as_tensor(_View(), device="cuda")

    def close(self):
        if self._h:
            _lib().bsfp_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------- bench support ---
def bsfp_synth_fp_values(f, n: int, seed: int, stream_id: int, start: int, out, stream=None):
    _check(_lib().bsfp_synth_fp_values(_fmt(f), n, seed, stream_id, start, _ptr(out), _stream(stream)),
           "bsfp_synth_fp_values")


def bsfp_lop3_probe(sink, grid: int, block: int, iters: int, seed: int = 1, stream=None):
    _check(_lib().bsfp_lop3_probe(_ptr(sink), grid, block, iters, seed, _stream(stream)), "bsfp_lop3_probe")


def bsfp_num_sms() -> int:
    return int(_lib().bsfp_num_sms())


# ------------------------------------------------- torch conveniences ---
def container_dtype(f):
    """torch dtype of the standard representation (same bytes as uint8/16/32)."""
    import torch
    cb = bsfp_container_bytes(f)
    return {1: torch.uint8, 2: torch.int16, 4: torch.int32}[cb]


def empty_bitslice(f, n: int, device="cuda"):
    """An uninitialised bitslice operand: B*S int32 words (viewed as uint32)."""
    import torch
    f = _fmt(f)
    return torch.empty(f.bits * bsfp_plane_stride(n), dtype=torch.int32, device=device)


def empty_standard(f, n: int, device="cuda"):
    import torch
    return torch.empty(n, dtype=container_dtype(f), device=device)
