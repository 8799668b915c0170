"""The C ABI without a GPU: the library loads, exports every function the
public headers declare, and its host-side logic (sizes, validation, status
strings, gate counts) behaves as documented.  No call here reaches a kernel
launch: every failing call is rejected by validation first."""
import ctypes
import os
import re

import pytest

import paper_1602_04716_gb300 as bs
from paper_1602_04716_gb300 import bsfp as _binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def _declared():
    names = set()
    for h in os.listdir(INCLUDE):
        if h.endswith(".h"):
            text = open(os.path.join(INCLUDE, h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(bsfp_\w+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_function():
    L = ctypes.CDLL(bs.lib_path())
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_plane_stride_and_sizes():
    assert bs.bsfp_plane_stride(0) == 0
    assert bs.bsfp_plane_stride(1) == 32
    assert bs.bsfp_plane_stride(1024) == 32
    assert bs.bsfp_plane_stride(1025) == 64
    assert bs.bsfp_plane_stride(1 << 28) == 1 << 23
    assert bs.bsfp_plane_stride(-1) == -1
    f = bs.Format(5, 7)
    assert bs.bsfp_bitslice_bytes(f, 1 << 28) == 13 * (1 << 23) * 4
    assert bs.bsfp_container_bytes(bs.Format(4, 3)) == 1
    assert bs.bsfp_container_bytes(bs.Format(4, 4)) == 2
    assert bs.bsfp_container_bytes(bs.Format(5, 10)) == 2
    assert bs.bsfp_container_bytes(bs.Format(8, 23)) == 4
    assert bs.bsfp_container_bytes(bs.Format(9, 7)) == -1


@pytest.mark.parametrize("fmt", [(1, 3, 0), (9, 3, 0), (4, 0, 0), (4, 24, 0), (4, 3, 4), (4, 3, -1)])
def test_bad_format_rejected(fmt):
    f = bs.Format(*fmt)
    L = _binding._lib()
    assert L.bsfp_add(f, 256, 256, 256, 10, None) == bs.ERR_FORMAT
    assert L.bsfp_pack(f, 256, 10, 256, None) == bs.ERR_FORMAT
    assert L.bsfp_bitslice_bytes(f, 10) == -1
    assert L.bsfp_gate_count(f, 0) == -1


def test_validation_order_and_codes():
    L = _binding._lib()
    f = bs.Format(5, 7)
    assert L.bsfp_add(f, 256, 256, 256, -1, None) == bs.ERR_SIZE
    assert L.bsfp_add(f, 256, 256, 256, bs.MAX_N + 1, None) == bs.ERR_SIZE
    assert L.bsfp_add(f, None, 256, 256, 10, None) == bs.ERR_NULL
    assert L.bsfp_fma2(f, 256, 256, None, 256, 10, None) == bs.ERR_NULL
    assert L.bsfp_mul(f, 264, 256, 256, 10, None) == bs.ERR_ALIGN
    assert L.bsfp_sub(f, 256, 256, 260, 10, None) == bs.ERR_ALIGN
    assert L.bsfp_pack(f, 257, 10, 256, None) == bs.ERR_ALIGN       # uint16 container, odd address
    assert L.bsfp_unpack(f, 256, 10, 257, None) == bs.ERR_ALIGN
    assert L.bsfp_unpack(f, 264, 10, 256, None) == bs.ERR_ALIGN
    # n == 0 is valid and launches nothing, whatever the pointers
    for fn in (L.bsfp_add, L.bsfp_sub, L.bsfp_mul):
        assert fn(f, None, None, None, 0, None) == bs.OK
    assert L.bsfp_fma2(f, None, None, None, None, 0, None) == bs.OK
    assert L.bsfp_pack(f, None, 0, None, None) == bs.OK
    assert L.bsfp_unpack(f, None, 0, None, None) == bs.OK


def test_status_strings():
    for code in range(0, -9, -1):
        s = bs.status_str(code)
        assert s and s != "unknown status"
    assert bs.status_str(-100) == "unknown status"


def test_stream_threshold_and_variant_query_arguments():
    L = _binding._lib()
    assert L.bsfp_set_stream_min_tiles(-1) == bs.ERR_SIZE
    assert L.bsfp_set_stream_min_tiles(1025) == bs.ERR_SIZE
    assert L.bsfp_set_stream_min_tiles(2) == bs.OK
    assert L.bsfp_set_batch_stream_min_tiles(-1) == bs.ERR_SIZE
    assert L.bsfp_set_batch_stream_min_tiles((1 << 20) + 1) == bs.ERR_SIZE
    assert L.bsfp_set_batch_stream_min_tiles(8) == bs.OK
    assert bs.bsfp_variant_for(bs.Format(9, 7), "mul", 10) == -1
    assert bs.bsfp_variant_for(bs.Format(5, 7), 9, 10) == -1
    assert bs.bsfp_variant_for(bs.Format(5, 7), "mul", -1) == -1
    f = bs.Format(5, 7)
    bs.bsfp_set_variant(f, "mul", 2, 0)
    assert bs.bsfp_variant_for(f, "mul", 1 << 20) == 2
    # a grid-stride shape set before the streamed variant is its fallback for small calls
    bs.bsfp_set_variant(f, "mul", 4, 3)
    bs.bsfp_set_variant(f, "mul", bs.VARIANT_STREAMED)
    assert bs.bsfp_variant(f, "mul") == bs.VARIANT_STREAMED
    assert bs.bsfp_variant_for(f, "mul", 1) == 4
    assert bs.bsfp_variant_for(f, "mul", 1 << 32) == bs.VARIANT_STREAMED
    bs.bsfp_set_variant(f, "mul", 0, 0)   # back to the default, fallback included
    bs.bsfp_set_variant(f, "mul", bs.VARIANT_STREAMED)
    assert bs.bsfp_variant_for(f, "mul", 1) == bs.bsfp_variants_compiled(f, "mul")[1]   # default: 2 words/thread
    bs.bsfp_set_variant(f, "mul", 0, 0)


def test_variants_and_overrides():
    f = bs.Format(5, 7)
    assert bs.bsfp_variants_compiled(f, "add") == [1, 2, 4, bs.VARIANT_STREAMED]
    assert bs.bsfp_variants_compiled(f, "mul") == [1, 2, 4, bs.VARIANT_STREAMED]
    assert bs.bsfp_variants_compiled(f, "fma2") == [1, 2, bs.VARIANT_STREAMED]
    assert bs.bsfp_variants_compiled(bs.Format(4, 4), "fma2") == [1, 2, 4]   # 9 planes: below the fma2 band
    assert bs.bsfp_variants_compiled(bs.Format(8, 23), "mul") == [1, 2]
    assert bs.bsfp_variant(f, "add") in (1, 2, 4, bs.VARIANT_STREAMED)
    g = bs.Format(6, 9)
    # a format outside the tuned set: its default words per thread, and (16 planes) the streamed mul,
    # which its mul calls take by default
    assert bs.bsfp_variants_compiled(g, "mul") == [2, bs.VARIANT_STREAMED]
    assert bs.bsfp_variant(g, "mul") == bs.VARIANT_STREAMED
    assert len(bs.bsfp_variants_compiled(g, "add")) == 1
    assert bs.bsfp_variants_compiled(bs.Format(3, 5), "mul") == [2]   # 9 planes: below the streamed band
    # division: streamed for 8..24 planes and 3 fraction bits or more, the default for the formats
    # outside the tuned set from 4 fraction bits on
    assert bs.bsfp_variants_compiled(f, "div") == [1, 2, 4, bs.VARIANT_STREAMED]
    assert bs.bsfp_variants_compiled(g, "div") == [2, bs.VARIANT_STREAMED]
    assert bs.bsfp_variant(g, "div") == bs.VARIANT_STREAMED
    assert bs.bsfp_variants_compiled(bs.Format(3, 5), "div") == [2, bs.VARIANT_STREAMED]
    assert bs.bsfp_variants_compiled(bs.Format(7, 10), "div") == [2, bs.VARIANT_STREAMED]   # 18 planes
    assert bs.bsfp_variants_compiled(bs.Format(8, 16), "div") == [1]   # 25 planes: above the band
    assert bs.bsfp_variants_compiled(bs.Format(3, 2), "div") == [2]    # 6 planes: below it
    assert bs.bsfp_variants_compiled(bs.Format(6, 2), "div") == [2]    # 2 fraction bits: HBM-bound, none
    # fma2: streamed for 10..19 planes and 4 fraction bits or more, the default for the formats outside
    # the tuned set
    assert bs.bsfp_variants_compiled(g, "fma2") == [1, bs.VARIANT_STREAMED]
    assert bs.bsfp_variant(g, "fma2") == bs.VARIANT_STREAMED
    assert bs.bsfp_variants_compiled(bs.Format(3, 6), "fma2") == [2, bs.VARIANT_STREAMED]
    assert bs.bsfp_variants_compiled(bs.Format(8, 10), "fma2") == [1, bs.VARIANT_STREAMED]
    assert bs.bsfp_variants_compiled(bs.Format(3, 5), "fma2") == [2]   # 9 planes: below the band
    assert bs.bsfp_variants_compiled(bs.Format(8, 11), "fma2") == [1]  # 20 planes: above it
    assert bs.bsfp_variants_compiled(bs.Format(8, 3), "fma2") == [2]   # 3 fraction bits: HBM-bound, none
    assert bs.bsfp_variants_compiled(bs.Format(6, 3), "div") == [2, bs.VARIANT_STREAMED]
    assert bs.bsfp_variant(bs.Format(6, 3), "div") in (2, bs.VARIANT_STREAMED)   # 3 bits: the tuner's choice
    with pytest.raises(bs.BsfpError):
        bs.bsfp_set_variant(g, "mul", 4)
    bs.bsfp_set_variant(f, "mul", 1, 3)
    assert bs.bsfp_variant(f, "mul") == 1
    bs.bsfp_set_variant(f, "mul", bs.VARIANT_STREAMED, 0)
    assert bs.bsfp_variant(f, "mul") == bs.VARIANT_STREAMED
    with pytest.raises(bs.BsfpError):
        bs.bsfp_set_variant(bs.Format(4, 4), "fma2", bs.VARIANT_STREAMED)
    for bad in (3, 5, 16):
        with pytest.raises(bs.BsfpError):
            bs.bsfp_set_variant(f, "mul", bad)
    bs.bsfp_set_variant(f, "mul", 2, 0)
    assert bs.bsfp_variant(f, "mul") == 2
    # every format in range is compiled for every op
    for e in range(2, 9):
        for m in range(1, 24):
            for op in range(4):
                assert bs.bsfp_variants_compiled(bs.Format(e, m), op), (e, m, op)


def test_gate_counts_follow_table1_classes():
    """Sec. 4, Table 1: add/sub is O(n log n) in the significand width and mul
    O(n^2).  Over M = 7 -> 23 at E = 8 the multiplier must grow much faster
    than the adder, and sub costs the same as add (one folded inversion)."""
    g = lambda e, m, op, r=0: bs.bsfp_gate_count(bs.Format(e, m, r), op)
    add7, add23 = g(8, 7, "add"), g(8, 23, "add")
    mul7, mul23 = g(8, 7, "mul"), g(8, 23, "mul")
    assert add23 / add7 < 3.0
    assert mul23 / mul7 > 4.0
    assert g(5, 7, "sub") == g(5, 7, "add")
    assert g(5, 7, "fma2") <= g(5, 7, "add") + g(5, 7, "mul")
    # RZ drops the round-up logic, so it never costs more than RN (Sec. 5.2)
    for e, m in [(4, 3), (5, 10), (8, 23)]:
        for op in ("add", "mul"):
            assert g(e, m, op, 1) <= g(e, m, op, 0)


def test_server_options_validated_before_any_cuda_call():
    L = _binding._lib()
    h = ctypes.c_void_p()
    for bad in [(0, 4, 1024, 1 << 16, 2), (1 << 20, 17, 0, 0, 0), (1 << 20, 0, 5000, 0, 0),
                (1 << 20, 0, 0, 64, 0), (1 << 20, 0, 0, 0, 3), (-1, 0, 0, 0, 0)]:
        opt = _binding.bsfp_server_options(*bad)
        assert L.bsfp_server_create(ctypes.byref(opt), ctypes.byref(h)) == bs.ERR_SIZE
        assert not h.value
    assert L.bsfp_server_create(None, None) == bs.ERR_NULL
    rid = ctypes.c_int64()
    assert L.bsfp_server_submit(None, None, ctypes.byref(rid)) == bs.ERR_NULL
    assert L.bsfp_server_poll(None, None, 4) == 0
    assert L.bsfp_server_release(None, 1) == bs.ERR_NULL
    assert L.bsfp_server_drain(None, 1) == bs.ERR_NULL
    L.bsfp_server_destroy(None)


def test_noalloc_sizes_rejected_before_any_cuda_call():
    L = _binding._lib()
    jobs = (bs.bsfp_job * 1)()
    assert L.bsfp_batch_run_noalloc(jobs, bs.NOALLOC_MAX_JOBS + 1, None) == bs.ERR_SIZE
    assert L.bsfp_batch_run_noalloc(jobs, -1, None) == bs.ERR_SIZE
    assert L.bsfp_batch_run_noalloc(jobs, 0, None) == bs.OK


def test_pipeline_arguments_validated_before_any_cuda_call():
    L = _binding._lib()
    h = ctypes.c_void_p()
    for chunk, depth in ((1000, 2), (-1024, 2), (1 << 31, 2), (4096, 17), (4096, -1)):
        assert L.bsfp_pipeline_create(chunk, depth, ctypes.byref(h)) == bs.ERR_SIZE
        assert not h.value
    assert L.bsfp_pipeline_create(4096, 2, None) == bs.ERR_NULL
    ops = (ctypes.c_int32 * 1)(0)
    outs = (ctypes.c_void_p * 1)(256)
    assert L.bsfp_pipeline_run(None, bs.Format(4, 3), 1, ops, 256, 256, None, outs, 10) == bs.ERR_NULL
    assert L.bsfp_pipeline_submit(None, bs.Format(4, 3), 1, ops, 256, 256, None, outs, 10) == bs.ERR_NULL
    assert L.bsfp_pipeline_wait(None) == bs.ERR_NULL
    L.bsfp_pipeline_free(None)


def test_flush_to_zero_only_for_the_compiled_formats():
    """RN/RZ with flush to zero (modes 2, 3) have kernels for the tuned
    formats only; any other format is refused before anything runs."""
    L = _binding._lib()
    for rnd in (bs.RN_FTZ, bs.RZ_FTZ):
        assert L.bsfp_add(bs.Format(6, 9, rnd), 256, 256, 256, 10, None) == bs.ERR_UNSUPPORTED
        assert L.bsfp_variants_compiled(bs.Format(6, 9, rnd), 2) == 0
        assert L.bsfp_variants_compiled(bs.Format(5, 7, rnd), 2) > 0
        assert bs.bsfp_gate_count(bs.Format(5, 7, rnd), "mul") < bs.bsfp_gate_count(bs.Format(5, 7, rnd & 1), "mul")


def test_conversion_arguments_validated_before_any_cuda_call():
    L = _binding._lib()
    f = bs.Format(5, 7)
    assert L.bsfp_from_float(f, 3, 256, 10, 256, None) == bs.ERR_UNSUPPORTED
    assert L.bsfp_from_float(bs.Format(9, 7), 0, 256, 10, 256, None) == bs.ERR_FORMAT
    assert L.bsfp_from_float(f, 0, None, 10, 256, None) == bs.ERR_NULL
    assert L.bsfp_from_float(f, 0, 258, 10, 256, None) == bs.ERR_ALIGN
    assert L.bsfp_from_float(f, 1, 258, 10, 260, None) == bs.ERR_ALIGN
    assert L.bsfp_from_float(bs.Format(6, 9, bs.RN_FTZ), 0, 256, 10, 256, None) == bs.ERR_UNSUPPORTED
    assert L.bsfp_from_float(f, 0, 256, -1, 256, None) == bs.ERR_SIZE
    assert L.bsfp_from_float(f, 0, 256, 0, 256, None) == bs.OK
    assert L.bsfp_to_float(f, 256, 10, 258, None) == bs.ERR_ALIGN
    assert L.bsfp_to_float(bs.Format(6, 9, bs.RZ_FTZ), 256, 10, 256, None) == bs.ERR_UNSUPPORTED


def test_integer_vectors_validated_before_any_cuda_call():
    L = _binding._lib()
    for fn in (L.bsfp_int_add, L.bsfp_int_sub, L.bsfp_int_mul):
        assert fn(0, 256, 256, 256, 10, None) == bs.ERR_FORMAT
        assert fn(33, 256, 256, 256, 10, None) == bs.ERR_FORMAT
        assert fn(5, 256, 256, 256, -1, None) == bs.ERR_SIZE
        assert fn(5, None, 256, 256, 10, None) == bs.ERR_NULL
        assert fn(5, 264, 256, 256, 10, None) == bs.ERR_ALIGN
        assert fn(5, 256, 256, 256, 0, None) == bs.OK
    assert L.bsfp_int_pack(9, 257, 10, 256, None) == bs.ERR_ALIGN
    assert L.bsfp_int_unpack(40, 256, 10, 256, None) == bs.ERR_FORMAT
    # gates per word: the Fig. 2 adder is two 3-input gates per slice but the first
    assert [bs.bsfp_int_gate_count(w, "add") for w in (1, 5, 13)] == [1, 9, 25]
    assert bs.bsfp_int_gate_count(33, "add") == -1


def test_autotune_arguments_and_cache_loading(tmp_path):
    L = _binding._lib()
    assert L.bsfp_autotune(bs.Format(9, 7), 0, None) == bs.ERR_FORMAT
    assert L.bsfp_autotune(bs.Format(5, 7), 9, None) == bs.ERR_UNSUPPORTED
    assert L.bsfp_autotune(bs.Format(6, 9, bs.RN_FTZ), 2, None) == bs.ERR_UNSUPPORTED
    assert bs.bsfp_autotune_load(str(tmp_path / "missing")) == -1
    cache = tmp_path / "shapes.txt"
    # E M rounding op wpt blocks/SM ms: two valid shapes, one not compiled (wpt 4 for 1/6/9), a comment
    cache.write_text("# test\n5 7 0 2 2 3 0.1\n4 4 1 0 1 0 0.2\n6 9 0 2 4 0 0.3\n")
    assert bs.bsfp_autotune_load(str(cache)) == 2
    assert bs.bsfp_variant(bs.Format(5, 7, 0), "mul") == 2
    assert bs.bsfp_variant(bs.Format(4, 4, 1), "add") == 1
    bs.bsfp_set_variant(bs.Format(5, 7, 0), "mul", 0, 0)
    bs.bsfp_set_variant(bs.Format(4, 4, 1), "add", 0, 0)


def test_batch_plan_options_validated_before_any_cuda_call():
    """Plan modes are PERSISTENT (0), PLAIN (1), STREAMED (2) and UNIFIED (3);
    anything else, or a bad shape, is refused before a job is looked at."""
    L = _binding._lib()
    h = ctypes.c_void_p()
    for mode, wpt, bps in ((4, 0, 0), (-1, 0, 0), (bs.BATCH_STREAMED, 3, 0), (bs.BATCH_STREAMED, 0, 65),
                           (bs.BATCH_UNIFIED, 3, 0)):
        opt = bs.bsfp_batch_options(mode, wpt, bps)
        assert L.bsfp_batch_plan_create(None, 0, ctypes.byref(opt), ctypes.byref(h)) == bs.ERR_SIZE
    assert L.bsfp_batch_plan_create(None, -1, None, ctypes.byref(h)) == bs.ERR_SIZE
    assert L.bsfp_batch_plan_create(None, 1, None, ctypes.byref(h)) == bs.ERR_NULL


def test_tuning_cache_matches_the_build():
    """Every per-format entry of the committed tuning cache names a variant
    compiled for its (format, op), with a blocks-per-SM choice the tuner
    offers; tune.apply() silently skips any other entry, so drift between the
    cache and the build would otherwise show only as slower launches.  Each
    GPU's cache covers every generated format in all four modes and op
    classes."""
    from paper_1602_04716_gb300 import build, tune
    cache = tune.load()
    assert cache, "no tuning cache committed"
    for gpu, entries in cache.items():
        keys = [k for k in entries if k.count("/") == 3]
        for key in keys:
            v = entries[key]
            e, m, r, op = key.split("/")
            f = bs.Format(int(e), int(m), int(r))
            assert v["wpt"] in bs.bsfp_variants_compiled(f, op), (gpu, key, v)
            assert v["bps"] in (0, 1, 2, 3, 4, 6, 8), (gpu, key, v)
            assert v["ms"] > 0 and v["n"] > 0, (gpu, key, v)
        want = {"%d/%d/%d/%s" % (E, M, r, op) for E, M in build.GEN_FORMATS for r in range(4)
                for op in ("add", "mul", "fma2", "div")}
        assert want <= set(keys), (gpu, sorted(want - set(keys))[:8])


def test_stream_shape_query():
    """Tiles and ring stages of the streamed kernels, as compiled (no device
    needed); formats and op classes without one are refused."""
    assert bs.bsfp_stream_shape(bs.Format(5, 7), "add") == (32 * 11 * 2, 3)
    assert bs.bsfp_stream_shape(bs.Format(5, 7), "sub") == (32 * 11 * 2, 3)
    assert bs.bsfp_stream_shape(bs.Format(5, 7), "mul") == (32 * 15 * 2, 2)
    assert bs.bsfp_stream_shape(bs.Format(4, 4, bs.RZ), "mul") == (32 * 11 * 2, 4)
    assert bs.bsfp_stream_shape(bs.Format(8, 7), "mul") == (32 * 14 * 2, 2)
    assert bs.bsfp_stream_shape(bs.Format(5, 7), "div") == (32 * 15 * 2, 2)
    assert bs.bsfp_stream_shape(bs.Format(3, 5, bs.RZ), "div") == (32 * 15 * 2, 2)
    assert bs.bsfp_stream_shape(bs.Format(7, 9), "div") == (32 * 12 * 2, 2)
    assert bs.bsfp_stream_shape(bs.Format(8, 10, bs.RZ), "div") == (32 * 11 * 2, 2)
    assert bs.bsfp_stream_shape(bs.Format(8, 13), "div") == (32 * 8 * 2, 2)
    assert bs.bsfp_stream_shape(bs.Format(5, 7), "fma2") == (32 * 11 * 2, 2)
    assert bs.bsfp_stream_shape(bs.Format(8, 7, bs.RZ_FTZ), "fma2") == (32 * 12 * 2, 2)
    assert bs.bsfp_stream_shape(bs.Format(6, 9), "fma2") == (32 * 12 * 2, 2)
    assert bs.bsfp_stream_shape(bs.Format(8, 10), "fma2") == (32 * 11 * 2, 2)
    for f, op in ((bs.Format(4, 4), "fma2"), (bs.Format(8, 11), "fma2"), (bs.Format(3, 5), "add"),
                  (bs.Format(8, 23), "mul"), (bs.Format(8, 23), "div"), (bs.Format(3, 5, bs.RN_FTZ), "div")):
        with pytest.raises(bs.BsfpError) as ei:
            bs.bsfp_stream_shape(f, op)
        assert ei.value.status == bs.ERR_UNSUPPORTED


@pytest.mark.parametrize("field,value", [("slots", 17), ("eager_slots", 5), ("eager_slots", -1),
                                         ("min_batch_tiles", -2), ("batch_wait_us", -2),
                                         ("batch_wait_us", 2000000), ("reserved", 1), ("wpt", 3)])
def test_server_options_are_checked_before_anything_is_allocated(field, value):
    L = _binding._lib()
    opt = _binding.bsfp_server_options(1 << 20, 4, 0, 0, 0, 0, 0, 0, 0)
    setattr(opt, field, value)
    h = ctypes.c_void_p()
    assert L.bsfp_server_create(ctypes.byref(opt), ctypes.byref(h)) == bs.ERR_SIZE
    assert not h.value


def test_server_bulk_submit_arguments():
    L = _binding._lib()
    assert L.bsfp_server_submit_n(None, None, 1, None, None) == bs.ERR_NULL


def test_stream_shapes_fit_and_load_the_schedulers_evenly():
    """Every compiled streamed kernel (all formats, ops and modes): a tile is
    a whole number of consumer warps' columns (64 each), the ring of NIN
    planes x tile x stages fits the 227 KB one block may use, and the
    consumer count is one that spreads evenly over the SM's four schedulers
    (warp index mod 4): never 9 or 10, which measured 7-13% slower than 8
    on the logic-bound multipliers."""
    seen = set()
    for E in range(2, 9):
        for M in range(1, 24):
            if 1 + E + M > 32:
                continue
            B = 1 + E + M
            for rnd in range(4):
                f = bs.Format(E, M, rnd)
                for op in ("add", "mul", "fma2", "div"):
                    try:
                        if bs.VARIANT_STREAMED not in bs.bsfp_variants_compiled(f, op):
                            continue
                    except bs.BsfpError:
                        continue
                    tw, stages = bs.bsfp_stream_shape(f, op)
                    assert tw % 64 == 0 and stages >= 2, (E, M, rnd, op, tw, stages)
                    nc = tw // 64
                    nin = 3 * B if (op == "fma2" and B <= 13) else 2 * B
                    assert nin * tw * 4 * stages + 256 <= 232448, (E, M, rnd, op, tw, stages)
                    assert nc not in (9, 10) and 8 <= nc <= 15, (E, M, rnd, op, nc)
                    seen.add((op, nc, stages))
    # every op class has a streamed kernel somewhere, in several shapes
    assert {op for op, _, _ in seen} == {"add", "mul", "fma2", "div"}
    assert len(seen) >= 8
