/*
 * api.cu -- the C ABI of libbsfp (declared in include/bsfp.h): argument
 * validation, the (format, op) dispatch table, launch shapes and the
 * autotuner's overrides.
 *
 * The paper's library generator (Sec. 5.1) turned a configuration file of
 * exponent bits, mantissa bits and rounding mode into a header plus a shared
 * library specialised to that format.  Here every format 1/E/M with
 * 2 <= E <= 8, 1 <= M <= 23 is compiled ahead of time as C++ template
 * instances, and the format becomes a run-time argument that selects the
 * instance from a table.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "binop.cuh"
#include "bsfp.h"
#include "convert.cuh"
#include "internal.h"
#include "tma.cuh"

namespace bsfp {

BinopEntry g_binop_table[TAB_E][TAB_M][TAB_R][OPC_ALL];
ConvEntry g_conv_table[9][24][4];
typedef cudaError_t (*int_launch_fn)(const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t S, int64_t nwords,
                                     uint32_t tailmask, int grid, cudaStream_t s);
int_launch_fn g_int_table[33][3];

/* Each exponent width is compiled as two translation units, M in [1, 11]
 * and [12, 23], and its division as two more; each fills its part of the
 * table. */
#define BSFP_DECL_REG(E) void register_e##E##_m1(); void register_e##E##_m12(); \
    void register_div_e##E##_m1(); void register_div_e##E##_m12();
BSFP_DECL_REG(2) BSFP_DECL_REG(3) BSFP_DECL_REG(4) BSFP_DECL_REG(5) BSFP_DECL_REG(6) BSFP_DECL_REG(7)
BSFP_DECL_REG(8)
#undef BSFP_DECL_REG
void register_conv_e2(); void register_conv_e3(); void register_conv_e4(); void register_conv_e5();
void register_conv_e6(); void register_conv_e7(); void register_conv_e8();
void register_int_w1(); void register_int_w17();
/* streamed kernels, one translation unit per format (stream_inst.cu) */
void register_stream_e4_m3(); void register_stream_e4_m4(); void register_stream_e5_m7();
void register_stream_e5_m10(); void register_stream_e8_m7();
/* streamed mul (12..24 planes), fma2 (10..19) and division (8..24) of the
 * other formats, one unit per exponent width and op class
 * (stream_band_inst.cu) */
void register_stream_mul_e2(); void register_stream_mul_e3(); void register_stream_mul_e4();
void register_stream_mul_e5(); void register_stream_mul_e6(); void register_stream_mul_e7();
void register_stream_mul_e8();
void register_stream_div_e2(); void register_stream_div_e3(); void register_stream_div_e4();
void register_stream_div_e5(); void register_stream_div_e6(); void register_stream_div_e7();
void register_stream_div_e8();
void register_stream_fma2_e2(); void register_stream_fma2_e3(); void register_stream_fma2_e4();
void register_stream_fma2_e5(); void register_stream_fma2_e6(); void register_stream_fma2_e7();
void register_stream_fma2_e8();

cudaError_t launch_pack(int cb, const void* in, int64_t n, int B, uint32_t* out, int64_t S, cudaStream_t st);
cudaError_t launch_unpack(int cb, const uint32_t* in, int64_t S, int B, void* out, int64_t n, cudaStream_t st);

static std::once_flag g_init_once;
static void init_tables() {
    register_e2_m1(); register_e2_m12();
    register_e3_m1(); register_e3_m12();
    register_e4_m1(); register_e4_m12();
    register_e5_m1(); register_e5_m12();
    register_e6_m1(); register_e6_m12();
    register_e7_m1(); register_e7_m12();
    register_e8_m1(); register_e8_m12();
    register_div_e2_m1(); register_div_e2_m12();
    register_div_e3_m1(); register_div_e3_m12();
    register_div_e4_m1(); register_div_e4_m12();
    register_div_e5_m1(); register_div_e5_m12();
    register_div_e6_m1(); register_div_e6_m12();
    register_div_e7_m1(); register_div_e7_m12();
    register_div_e8_m1(); register_div_e8_m12();
    register_conv_e2(); register_conv_e3(); register_conv_e4(); register_conv_e5();
    register_conv_e6(); register_conv_e7(); register_conv_e8();
    register_int_w1(); register_int_w17();
    /* after the grid-stride kernels: these extend their entries */
    register_stream_e4_m3(); register_stream_e4_m4(); register_stream_e5_m7();
    register_stream_e5_m10(); register_stream_e8_m7();
    register_stream_mul_e2(); register_stream_mul_e3(); register_stream_mul_e4(); register_stream_mul_e5();
    register_stream_mul_e6(); register_stream_mul_e7(); register_stream_mul_e8();
    register_stream_div_e2(); register_stream_div_e3(); register_stream_div_e4(); register_stream_div_e5();
    register_stream_div_e6(); register_stream_div_e7(); register_stream_div_e8();
    register_stream_fma2_e2(); register_stream_fma2_e3(); register_stream_fma2_e4(); register_stream_fma2_e5();
    register_stream_fma2_e6(); register_stream_fma2_e7(); register_stream_fma2_e8();
}

/* The streamed kernel is taken only when every SM gets at least this many
 * tiles: with fewer, its ring never fills and the grid-stride kernel is
 * faster (bsfp_set_stream_min_tiles). */
static std::atomic<int32_t> g_stream_min_tiles{2};

/* Devices on which a streamed kernel has opted in to its shared memory, one
 * bit per device, per (E, M, rounding, op class). */
static std::atomic<uint64_t> g_stream_ready[TAB_E][TAB_M][TAB_R][OPC_ALL];

/* The fault word the streamed kernels set when a wait runs out of time, per
 * device (its address is looked up once per device). */
static __device__ int g_fault_word;
static std::atomic<int*> g_fault_addr[64];

static int current_device() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return -1;
    }
    return dev;
}

static int* fault_word(int dev) {
    if (dev < 0 || dev >= 64) return nullptr;
    int* p = g_fault_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        void* a = nullptr;
        if (cudaGetSymbolAddress(&a, g_fault_word) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        p = static_cast<int*>(a);
        g_fault_addr[dev].store(p, std::memory_order_release);
    }
    return p;
}

/* Launch shape per (E, M, rounding, op class): words per thread and resident
 * blocks per SM (0 = the occupancy maximum). */
struct Shape {
    int8_t wpt;
    int16_t bps;
    /* the grid-stride shape the streamed variant gives way to for calls too
     * small for it: the last grid-stride shape set (0 = the default) */
    int8_t fb_wpt;
    int16_t fb_bps;
};

/* Variant and blocks/SM of a call on S plane words under shape sh. */
static void pick_shape(const Shape& sh, const BinopEntry* e, int64_t S, int* wpt, int* bps);
/* The shapes, each packed into one atomic word: a launch reads its shape
 * with one load and takes no lock; writers (bsfp_set_variant) serialise on
 * g_shape_mu for their read-modify-write. */
static std::atomic<uint64_t> g_shape[TAB_E][TAB_M][TAB_R][OPC_ALL];
static std::atomic<int> g_occ[TAB_E][TAB_M][TAB_R][OPC_ALL][5];   /* cached occupancy per wpt */
static std::mutex g_shape_mu;

static uint64_t pack_shape(const Shape& s) {
    return (uint64_t)(uint8_t)s.wpt | ((uint64_t)(uint16_t)s.bps << 8) | ((uint64_t)(uint8_t)s.fb_wpt << 24) |
           ((uint64_t)(uint16_t)s.fb_bps << 32);
}
static Shape unpack_shape(uint64_t v) {
    Shape s;
    s.wpt = (int8_t)(uint8_t)(v & 0xFFu);
    s.bps = (int16_t)(uint16_t)((v >> 8) & 0xFFFFu);
    s.fb_wpt = (int8_t)(uint8_t)((v >> 24) & 0xFFu);
    s.fb_bps = (int16_t)(uint16_t)((v >> 32) & 0xFFFFu);
    return s;
}
static Shape load_shape(const bsfp_format& f, int opc) {
    return unpack_shape(g_shape[f.exp_bits][f.man_bits][f.rnd][opc].load(std::memory_order_acquire));
}

static std::atomic<int64_t> g_launches{0};
static thread_local int32_t g_last_cuda = 0;

/* Record a CUDA failure for bsfp_last_cuda_error and clear the runtime's
 * per-thread last-error slot: a refused cudaMalloc, say, must not surface
 * later as the "launch error" of an unrelated kernel (ours or the caller's)
 * checked with cudaGetLastError. */
static bsfp_status cuda_fail(cudaError_t e) {
    g_last_cuda = (int32_t)e;
    (void)cudaGetLastError();
    return BSFP_ERR_CUDA;
}

bool format_ok(const bsfp_format& f) {
    return f.exp_bits >= 2 && f.exp_bits <= 8 && f.man_bits >= 1 && f.man_bits <= 23 &&
           1 + f.exp_bits + f.man_bits <= 32 && f.rnd >= BSFP_RN && f.rnd <= BSFP_RZ_FTZ;
}

static int bits_of(const bsfp_format& f) { return 1 + f.exp_bits + f.man_bits; }

bool aligned(const void* p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

int opclass(int op) {
    switch (op) {
        case BSFP_OP_ADD:
        case BSFP_OP_SUB: return OPC_ADDSUB;
        case BSFP_OP_MUL: return OPC_MUL;
        case BSFP_OP_FMA2: return OPC_FMA2;
        case BSFP_OP_DIV: return OPC_DIV;
    }
    return -1;
}

static const BinopEntry* entry_for(const bsfp_format& f, int opc) {
    std::call_once(g_init_once, init_tables);
    const BinopEntry* e = &g_binop_table[f.exp_bits][f.man_bits][f.rnd][opc];
    return e->launch ? e : nullptr;
}

static int occupancy(const bsfp_format& f, int opc, const BinopEntry* e, int wpt) {
    std::atomic<int>& o = g_occ[f.exp_bits][f.man_bits][f.rnd][opc][wpt];
    int v = o.load(std::memory_order_relaxed);
    if (v == 0) {   /* looked up once; racing first calls store the same value */
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, e->kernel(wpt), 128, 0) != cudaSuccess || v < 1) {
            (void)cudaGetLastError();
            v = 1;
        }
        o.store(v, std::memory_order_relaxed);
    }
    return v;
}

/* Validate one element-wise op and work out its launch: kernel entry, args,
 * words per thread and grid.  Returns BSFP_OK with *skip set when n == 0.
 * force_streamed: take the streamed kernel whatever the shape table and the
 * call's size (the caller has checked that it is compiled). */
static bsfp_status prepare_binop_impl(const bsfp_format& f, int op, const uint32_t* a, const uint32_t* b,
                                      const uint32_t* c, uint32_t* out, int64_t n, PreparedOp* po,
                                      bool force_streamed);

bsfp_status prepare_binop(const bsfp_format& f, int op, const uint32_t* a, const uint32_t* b, const uint32_t* c,
                          uint32_t* out, int64_t n, PreparedOp* po) {
    return prepare_binop_impl(f, op, a, b, c, out, n, po, false);
}

bsfp_status validate_binop(const bsfp_format& f, int op, const uint32_t* a, const uint32_t* b, const uint32_t* c,
                           const uint32_t* out, int64_t n, int* opc_out) {
    if (!format_ok(f)) return BSFP_ERR_FORMAT;
    const int opc = opclass(op);
    if (opc < 0) return BSFP_ERR_UNSUPPORTED;
    if (n < 0 || n > BSFP_MAX_N) return BSFP_ERR_SIZE;
    *opc_out = opc;
    if (n == 0) return BSFP_OK;
    if (!a || !b || !out || (opc == OPC_FMA2 && !c)) return BSFP_ERR_NULL;
    if (!aligned(a, 16) || !aligned(b, 16) || !aligned(out, 16) || (opc == OPC_FMA2 && !aligned(c, 16)))
        return BSFP_ERR_ALIGN;
    return entry_for(f, opc) ? BSFP_OK : BSFP_ERR_UNSUPPORTED;
}

static bsfp_status prepare_binop_impl(const bsfp_format& f, int op, const uint32_t* a, const uint32_t* b,
                                      const uint32_t* c, uint32_t* out, int64_t n, PreparedOp* po,
                                      bool force_streamed) {
    po->skip = false;
    if (!format_ok(f)) return BSFP_ERR_FORMAT;
    const int opc = opclass(op);
    if (opc < 0) return BSFP_ERR_UNSUPPORTED;
    if (n < 0 || n > BSFP_MAX_N) return BSFP_ERR_SIZE;
    if (n == 0) {
        po->skip = true;
        return BSFP_OK;
    }
    if (!a || !b || !out || (opc == OPC_FMA2 && !c)) return BSFP_ERR_NULL;
    if (!aligned(a, 16) || !aligned(b, 16) || !aligned(out, 16) || (opc == OPC_FMA2 && !aligned(c, 16)))
        return BSFP_ERR_ALIGN;
    const BinopEntry* e = entry_for(f, opc);
    if (!e) return BSFP_ERR_UNSUPPORTED;

    BinopArgs& p = po->args;
    p.a = a;
    p.b = b;
    p.c = c;
    p.out = out;
    p.S = bsfp_plane_stride(n);
    p.nwords = (n + 31) / 32;
    p.tailmask = (n % 32) ? ((1u << (n % 32)) - 1u) : ~0u;
    p.negb = (op == BSFP_OP_SUB) ? ~0u : 0u;
    p.wait_cycles = STREAM_WAIT_CYCLES;
    p.withhold_tile = -1;
    po->entry = e;
    po->opc = opc;

    const int dev = current_device();
    p.fault = fault_word(dev);
    int wpt, bps;
    if (force_streamed) {
        wpt = VARIANT_STREAMED;
        bps = 1;
    } else {
        pick_shape(load_shape(f, opc), e, p.S, &wpt, &bps);
        if (wpt != VARIANT_STREAMED) {
            const int occ = occupancy(f, opc, e, wpt);
            bps = (bps > 0 && bps < occ) ? bps : occ;
        }
    }
    if (wpt == VARIANT_STREAMED) {
        /* one block per SM (the ring takes its shared memory), one tile of
         * stream_tw word columns per block at a time */
        std::atomic<uint64_t>& ready = g_stream_ready[f.exp_bits][f.man_bits][f.rnd][opc];
        const uint64_t bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
        if (!bit || !(ready.load(std::memory_order_acquire) & bit)) {
            const cudaError_t err = e->stream_prepare();
            if (err != cudaSuccess) return cuda_fail(err);
            ready.fetch_or(bit, std::memory_order_acq_rel);
        }
        const int64_t tiles = (p.S + e->stream_tw - 1) / e->stream_tw;
        const int64_t sms = device_num_sms();
        po->wpt = wpt;
        po->grid = (int)(tiles < sms ? tiles : sms);
        return BSFP_OK;
    }
    const int64_t chunks = p.S / wpt;
    const int64_t need = (chunks + 127) / 128;
    const int64_t cap = (int64_t)device_num_sms() * bps;
    po->wpt = wpt;
    po->grid = (int)(need < cap ? need : cap);
    return BSFP_OK;
}

static void pick_shape(const Shape& sh, const BinopEntry* e, int64_t S, int* wpt, int* bps) {
    *wpt = (sh.wpt && (e->wpt_mask & (unsigned)sh.wpt)) ? sh.wpt : (e->preferred ? e->preferred : e->default_wpt);
    *bps = sh.bps;
    if (*wpt == VARIANT_STREAMED) {
        const int64_t tiles = (S + e->stream_tw - 1) / e->stream_tw;
        if (tiles >= (int64_t)g_stream_min_tiles.load(std::memory_order_relaxed) * device_num_sms()) {
            *bps = 1;
            return;
        }
        /* too small to fill the ring: the fallback grid-stride shape */
        const bool fb = sh.fb_wpt && (e->wpt_mask & (unsigned)sh.fb_wpt);
        *wpt = fb ? sh.fb_wpt : e->default_wpt;
        *bps = fb ? sh.fb_bps : 0;
    }
}

bsfp_status launch_prepared(const PreparedOp& po, cudaStream_t s) {
    if (po.skip) return BSFP_OK;
    const cudaError_t err = (po.wpt == VARIANT_STREAMED) ? po.entry->stream_launch(po.args, po.grid, s)
                                                         : po.entry->launch(po.args, po.wpt, po.grid, s);
    if (err != cudaSuccess) return cuda_fail(err);
    return BSFP_OK;
}

void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int* current_fault_word() { return fault_word(current_device()); }

bsfp_status run_op_by_code(const bsfp_format& f, int op, const uint32_t* a, const uint32_t* b, const uint32_t* c,
                           uint32_t* out, int64_t n, cudaStream_t s) {
    PreparedOp po;
    const bsfp_status st = prepare_binop(f, op, a, b, c, out, n, &po);
    if (st != BSFP_OK || po.skip) return st;
    const bsfp_status r = launch_prepared(po, s);
    if (r == BSFP_OK) count_launches(1);
    return r;
}

bsfp_status set_cuda_error(cudaError_t e) { return cuda_fail(e); }

/* Run one element-wise op. */
static bsfp_status run_binop(const bsfp_format& f, int op, const uint32_t* a, const uint32_t* b, const uint32_t* c,
                             uint32_t* out, int64_t n, cudaStream_t s) {
    PreparedOp po;
    const bsfp_status st = prepare_binop(f, op, a, b, c, out, n, &po);
    if (st != BSFP_OK || po.skip) return st;
    const bsfp_status r = launch_prepared(po, s);
    if (r == BSFP_OK) count_launches(1);
    return r;
}

}  // namespace bsfp

using namespace bsfp;

extern "C" {

int64_t bsfp_plane_stride(int64_t n) {
    if (n < 0) return -1;
    const int64_t words = (n + 31) / 32;
    return (words + 31) / 32 * 32;
}

int64_t bsfp_bitslice_bytes(bsfp_format f, int64_t n) {
    if (!format_ok(f) || n < 0 || n > BSFP_MAX_N) return -1;
    return (int64_t)bits_of(f) * bsfp_plane_stride(n) * 4;
}

int32_t bsfp_container_bytes(bsfp_format f) {
    if (!format_ok(f)) return -1;
    const int B = bits_of(f);
    return B <= 8 ? 1 : (B <= 16 ? 2 : 4);
}

bsfp_status bsfp_pack(bsfp_format f, const void* std_in, int64_t n, uint32_t* bs_out, bsfp_stream_t s) {
    if (!format_ok(f)) return BSFP_ERR_FORMAT;
    if (n < 0 || n > BSFP_MAX_N) return BSFP_ERR_SIZE;
    if (n == 0) return BSFP_OK;
    if (!std_in || !bs_out) return BSFP_ERR_NULL;
    const int cb = bsfp_container_bytes(f);
    if (!aligned(std_in, (uintptr_t)cb) || !aligned(bs_out, 16)) return BSFP_ERR_ALIGN;
    const cudaError_t e = launch_pack(cb, std_in, n, bits_of(f), bs_out, bsfp_plane_stride(n), (cudaStream_t)s);
    if (e != cudaSuccess) return cuda_fail(e);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return BSFP_OK;
}

bsfp_status bsfp_unpack(bsfp_format f, const uint32_t* bs_in, int64_t n, void* std_out, bsfp_stream_t s) {
    if (!format_ok(f)) return BSFP_ERR_FORMAT;
    if (n < 0 || n > BSFP_MAX_N) return BSFP_ERR_SIZE;
    if (n == 0) return BSFP_OK;
    if (!bs_in || !std_out) return BSFP_ERR_NULL;
    const int cb = bsfp_container_bytes(f);
    if (!aligned(bs_in, 16) || !aligned(std_out, (uintptr_t)cb)) return BSFP_ERR_ALIGN;
    const cudaError_t e = launch_unpack(cb, bs_in, bsfp_plane_stride(n), bits_of(f), std_out, n, (cudaStream_t)s);
    if (e != cudaSuccess) return cuda_fail(e);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return BSFP_OK;
}

bsfp_status bsfp_add(bsfp_format f, const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t n, bsfp_stream_t s) {
    return run_binop(f, BSFP_OP_ADD, a, b, nullptr, out, n, (cudaStream_t)s);
}

bsfp_status bsfp_sub(bsfp_format f, const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t n, bsfp_stream_t s) {
    return run_binop(f, BSFP_OP_SUB, a, b, nullptr, out, n, (cudaStream_t)s);
}

bsfp_status bsfp_mul(bsfp_format f, const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t n, bsfp_stream_t s) {
    return run_binop(f, BSFP_OP_MUL, a, b, nullptr, out, n, (cudaStream_t)s);
}

bsfp_status bsfp_fma2(bsfp_format f, const uint32_t* a, const uint32_t* b, const uint32_t* c, uint32_t* out,
                      int64_t n, bsfp_stream_t s) {
    return run_binop(f, BSFP_OP_FMA2, a, b, c, out, n, (cudaStream_t)s);
}

bsfp_status bsfp_div(bsfp_format f, const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t n, bsfp_stream_t s) {
    return run_binop(f, BSFP_OP_DIV, a, b, nullptr, out, n, (cudaStream_t)s);
}

/* Grid of the conversions: the word-column tiles over 4-warp blocks, at most
 * 8 blocks per SM. */
static int conv_grid(int64_t tiles) {
    const int64_t want = (tiles + CV_WARPS - 1) / CV_WARPS;
    const int64_t cap = (int64_t)device_num_sms() * 8;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

bsfp_status bsfp_from_float(bsfp_format f, int32_t type, const void* in, int64_t n, uint32_t* bs_out,
                            bsfp_stream_t s) {
    if (!format_ok(f)) return BSFP_ERR_FORMAT;
    if (type < BSFP_FLOAT32 || type > BSFP_FLOAT16) return BSFP_ERR_UNSUPPORTED;
    if (n < 0 || n > BSFP_MAX_N) return BSFP_ERR_SIZE;
    if (n == 0) return BSFP_OK;
    if (!in || !bs_out) return BSFP_ERR_NULL;
    if (!aligned(in, type == BSFP_FLOAT32 ? 4 : 2) || !aligned(bs_out, 16)) return BSFP_ERR_ALIGN;
    std::call_once(g_init_once, init_tables);
    const ConvEntry& e = g_conv_table[f.exp_bits][f.man_bits][f.rnd];
    if (!e.from) return BSFP_ERR_UNSUPPORTED;
    const int64_t S = bsfp_plane_stride(n);
    const cudaError_t err = e.from(in, type, n, bs_out, S, conv_grid(S / 32), (cudaStream_t)s);
    if (err != cudaSuccess) return cuda_fail(err);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return BSFP_OK;
}

bsfp_status bsfp_to_float(bsfp_format f, const uint32_t* bs_in, int64_t n, float* out, bsfp_stream_t s) {
    if (!format_ok(f)) return BSFP_ERR_FORMAT;
    if (n < 0 || n > BSFP_MAX_N) return BSFP_ERR_SIZE;
    if (n == 0) return BSFP_OK;
    if (!bs_in || !out) return BSFP_ERR_NULL;
    if (!aligned(bs_in, 16) || !aligned(out, 4)) return BSFP_ERR_ALIGN;
    std::call_once(g_init_once, init_tables);
    const ConvEntry& e = g_conv_table[f.exp_bits][f.man_bits][f.rnd];
    if (!e.to) return BSFP_ERR_UNSUPPORTED;
    const int64_t S = bsfp_plane_stride(n);
    const cudaError_t err =
        e.to(bs_in, S, n, reinterpret_cast<uint32_t*>(out), conv_grid((n + 1023) / 1024), (cudaStream_t)s);
    if (err != cudaSuccess) return cuda_fail(err);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return BSFP_OK;
}

/* ------------------------------------------------ integer vectors (Sec. 3) */
static int int_container_bytes(int w) { return w <= 8 ? 1 : (w <= 16 ? 2 : 4); }

bsfp_status bsfp_int_pack(int32_t bits, const void* std_in, int64_t n, uint32_t* bs_out, bsfp_stream_t s) {
    if (bits < 1 || bits > 32) return BSFP_ERR_FORMAT;
    if (n < 0 || n > BSFP_MAX_N) return BSFP_ERR_SIZE;
    if (n == 0) return BSFP_OK;
    if (!std_in || !bs_out) return BSFP_ERR_NULL;
    const int cb = int_container_bytes(bits);
    if (!aligned(std_in, (uintptr_t)cb) || !aligned(bs_out, 16)) return BSFP_ERR_ALIGN;
    const cudaError_t e = launch_pack(cb, std_in, n, bits, bs_out, bsfp_plane_stride(n), (cudaStream_t)s);
    if (e != cudaSuccess) return cuda_fail(e);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return BSFP_OK;
}

bsfp_status bsfp_int_unpack(int32_t bits, const uint32_t* bs_in, int64_t n, void* std_out, bsfp_stream_t s) {
    if (bits < 1 || bits > 32) return BSFP_ERR_FORMAT;
    if (n < 0 || n > BSFP_MAX_N) return BSFP_ERR_SIZE;
    if (n == 0) return BSFP_OK;
    if (!bs_in || !std_out) return BSFP_ERR_NULL;
    const int cb = int_container_bytes(bits);
    if (!aligned(bs_in, 16) || !aligned(std_out, (uintptr_t)cb)) return BSFP_ERR_ALIGN;
    const cudaError_t e = launch_unpack(cb, bs_in, bsfp_plane_stride(n), bits, std_out, n, (cudaStream_t)s);
    if (e != cudaSuccess) return cuda_fail(e);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return BSFP_OK;
}

static bsfp_status run_int(int32_t bits, int op, const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t n,
                           bsfp_stream_t s) {
    if (bits < 1 || bits > 32) return BSFP_ERR_FORMAT;
    if (n < 0 || n > BSFP_MAX_N) return BSFP_ERR_SIZE;
    if (n == 0) return BSFP_OK;
    if (!a || !b || !out) return BSFP_ERR_NULL;
    if (!aligned(a, 16) || !aligned(b, 16) || !aligned(out, 16)) return BSFP_ERR_ALIGN;
    std::call_once(g_init_once, init_tables);
    const int_launch_fn fn = g_int_table[bits][op];
    if (!fn) return BSFP_ERR_UNSUPPORTED;
    const int64_t S = bsfp_plane_stride(n);
    const int wpt = bits <= 16 ? 4 : 2;
    const int64_t need = (S / wpt + 127) / 128;
    const int64_t cap = (int64_t)device_num_sms() * 8;
    const cudaError_t e = fn(a, b, out, S, (n + 31) / 32, (n % 32) ? ((1u << (n % 32)) - 1u) : ~0u,
                             (int)(need < cap ? need : cap), (cudaStream_t)s);
    if (e != cudaSuccess) return cuda_fail(e);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return BSFP_OK;
}

bsfp_status bsfp_int_add(int32_t bits, const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t n,
                         bsfp_stream_t s) {
    return run_int(bits, IOP_ADD, a, b, out, n, s);
}

bsfp_status bsfp_int_sub(int32_t bits, const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t n,
                         bsfp_stream_t s) {
    return run_int(bits, IOP_SUB, a, b, out, n, s);
}

bsfp_status bsfp_int_mul(int32_t bits, const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t n,
                         bsfp_stream_t s) {
    return run_int(bits, IOP_MUL, a, b, out, n, s);
}

long bsfp_int_gate_count_impl(int bits, int op);

int64_t bsfp_int_gate_count(int32_t bits, int32_t op) { return bsfp_int_gate_count_impl(bits, op); }

const char* bsfp_status_str(int32_t status) {
    switch (status) {
        case BSFP_OK: return "ok";
        case BSFP_ERR_FORMAT: return "format out of range (need 2<=E<=8, 1<=M<=23, rounding RN or RZ)";
        case BSFP_ERR_NULL: return "null pointer";
        case BSFP_ERR_ALIGN: return "misaligned pointer (bitslice: 16 bytes; standard: container size)";
        case BSFP_ERR_SIZE: return "size out of range";
        case BSFP_ERR_UNSUPPORTED: return "not compiled into the library";
        case BSFP_ERR_CUDA: return "CUDA error";
        case BSFP_ERR_BUDGET: return "over the memory budget";
        case BSFP_ERR_TIMEOUT: return "timed out";
    }
    return "unknown status";
}

int32_t bsfp_last_cuda_error(void) { return g_last_cuda; }

long bsfp_gate_count_e2(int, int, int);
long bsfp_gate_count_e3(int, int, int);
long bsfp_gate_count_e4(int, int, int);
long bsfp_gate_count_e5(int, int, int);
long bsfp_gate_count_e6(int, int, int);
long bsfp_gate_count_e7(int, int, int);
long bsfp_gate_count_e8(int, int, int);

int64_t bsfp_gate_count(bsfp_format f, int32_t op) {
    if (!format_ok(f) || op < 0 || op > 4) return -1;
    const int m = f.man_bits, r = f.rnd;
    switch (f.exp_bits) {
        case 2: return bsfp_gate_count_e2(m, r, op);
        case 3: return bsfp_gate_count_e3(m, r, op);
        case 4: return bsfp_gate_count_e4(m, r, op);
        case 5: return bsfp_gate_count_e5(m, r, op);
        case 6: return bsfp_gate_count_e6(m, r, op);
        case 7: return bsfp_gate_count_e7(m, r, op);
        case 8: return bsfp_gate_count_e8(m, r, op);
    }
    return -1;
}

int32_t bsfp_variants_compiled(bsfp_format f, int32_t op) {
    if (!format_ok(f) || opclass(op) < 0) return -1;
    const BinopEntry* e = entry_for(f, opclass(op));
    return e ? (int32_t)e->wpt_mask : 0;
}

bsfp_status bsfp_stream_selftest(bsfp_format f, int32_t op, const uint32_t* a, const uint32_t* b, uint32_t* out,
                                 int64_t n, int64_t withhold_tile, int64_t wait_cycles, cudaStream_t s) {
    if (wait_cycles < (1ll << 16) || wait_cycles > (1ll << 34)) return BSFP_ERR_SIZE;
    if (!format_ok(f)) return BSFP_ERR_FORMAT;
    const int opc = opclass(op);
    if (opc != OPC_ADDSUB && opc != OPC_MUL) return BSFP_ERR_UNSUPPORTED;
    if (n <= 0) return BSFP_ERR_SIZE;
    const BinopEntry* e = entry_for(f, opc);
    if (!e || !(e->wpt_mask & (unsigned)VARIANT_STREAMED)) return BSFP_ERR_UNSUPPORTED;
    /* the streamed kernel whatever the shape settings and size */
    PreparedOp po;
    bsfp_status st = prepare_binop_impl(f, op, a, b, nullptr, out, n, &po, true);
    if (st != BSFP_OK) return st;
    const int64_t tiles = (po.args.S + e->stream_tw - 1) / e->stream_tw;
    if (po.wpt != VARIANT_STREAMED || withhold_tile < -1 || withhold_tile >= tiles) return BSFP_ERR_SIZE;
    po.args.withhold_tile = withhold_tile;
    po.args.wait_cycles = wait_cycles;
    st = launch_prepared(po, s);
    if (st == BSFP_OK) count_launches(1);
    return st;
}

bsfp_status bsfp_set_stream_min_tiles(int32_t tiles_per_sm) {
    if (tiles_per_sm < 0 || tiles_per_sm > 1024) return BSFP_ERR_SIZE;
    g_stream_min_tiles.store(tiles_per_sm, std::memory_order_relaxed);
    return BSFP_OK;
}

int32_t bsfp_variant_for(bsfp_format f, int32_t op, int64_t n) {
    if (!format_ok(f) || opclass(op) < 0 || n < 0 || n > BSFP_MAX_N) return -1;
    const int opc = opclass(op);
    const BinopEntry* e = entry_for(f, opc);
    if (!e) return 0;
    int wpt, bps;
    pick_shape(load_shape(f, opc), e, bsfp_plane_stride(n), &wpt, &bps);
    return wpt;
}

bsfp_status bsfp_stream_shape(bsfp_format f, int32_t op, int32_t* tile_words, int32_t* stages) {
    if (!format_ok(f)) return BSFP_ERR_FORMAT;
    if (opclass(op) < 0) return BSFP_ERR_UNSUPPORTED;
    if (!tile_words || !stages) return BSFP_ERR_NULL;
    const BinopEntry* e = entry_for(f, opclass(op));
    if (!e || !(e->wpt_mask & (unsigned)VARIANT_STREAMED)) return BSFP_ERR_UNSUPPORTED;
    *tile_words = e->stream_tw;
    *stages = e->stream_nst;
    return BSFP_OK;
}

int32_t bsfp_variant(bsfp_format f, int32_t op) {
    if (!format_ok(f) || opclass(op) < 0) return -1;
    const int opc = opclass(op);
    const BinopEntry* e = entry_for(f, opc);
    if (!e) return 0;
    const Shape sh = load_shape(f, opc);
    return (sh.wpt && (e->wpt_mask & (unsigned)sh.wpt)) ? sh.wpt : (e->preferred ? e->preferred : e->default_wpt);
}

bsfp_status bsfp_set_variant(bsfp_format f, int32_t op, int32_t wpt, int32_t blocks_per_sm) {
    if (!format_ok(f)) return BSFP_ERR_FORMAT;
    const int opc = opclass(op);
    if (opc < 0 || blocks_per_sm < 0 || blocks_per_sm > 64) return BSFP_ERR_SIZE;
    if (wpt != 0 && wpt != 1 && wpt != 2 && wpt != 4 && wpt != VARIANT_STREAMED) return BSFP_ERR_SIZE;
    const BinopEntry* e = entry_for(f, opc);
    if (!e || (wpt != 0 && !(e->wpt_mask & (unsigned)wpt))) return BSFP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_shape_mu);
    std::atomic<uint64_t>& slot = g_shape[f.exp_bits][f.man_bits][f.rnd][opc];
    Shape sh = unpack_shape(slot.load(std::memory_order_relaxed));
    sh.wpt = (int8_t)wpt;
    sh.bps = (int16_t)blocks_per_sm;
    if (wpt != VARIANT_STREAMED) {   /* a grid-stride shape (or the default) is also the fallback */
        sh.fb_wpt = (int8_t)wpt;
        sh.fb_bps = (int16_t)blocks_per_sm;
    }
    slot.store(pack_shape(sh), std::memory_order_release);
    return BSFP_OK;
}

int64_t bsfp_launch_count(void) { return g_launches.load(); }

int32_t bsfp_fault_status(int32_t clear) {
    int* p = fault_word(current_device());
    if (!p) return -1;
    int v = 0;
    cudaError_t err = cudaDeviceSynchronize();
    if (err == cudaSuccess) err = cudaMemcpy(&v, p, sizeof v, cudaMemcpyDeviceToHost);
    if (err == cudaSuccess && clear && v) {
        const int zero = 0;
        err = cudaMemcpy(p, &zero, sizeof zero, cudaMemcpyHostToDevice);
    }
    if (err != cudaSuccess) {
        cuda_fail(err);
        return -1;
    }
    return v;
}

}  // extern "C"
