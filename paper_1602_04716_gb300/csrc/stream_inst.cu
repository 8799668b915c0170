/*
 * stream_inst.cu -- instantiates the streamed kernels (stream.cuh) for one
 * format, compiled once per format with -DBSFP_SE=E -DBSFP_SM=M, and adds
 * them to that format's dispatch-table entries (add/sub and mul with their
 * job-list form, and division and fma2 where the format lies in their
 * bands, every rounding mode) as variant VARIANT_STREAMED.  Which variant a call takes
 * stays the autotuner's choice for these formats.  Registered after the
 * grid-stride kernels, whose entries it extends.
 */
#include "stream.cuh"

#if !defined(BSFP_SE) || !defined(BSFP_SM)
#error "compile with -DBSFP_SE=<exponent bits> -DBSFP_SM=<mantissa bits>"
#endif

namespace bsfp {

static_assert(stream_format(BSFP_SE, BSFP_SM), "format without a streamed kernel");

template <int E, int M, int R, int OPC>
static void add_stream(BinopEntry& e) {
    e.stream_launch = stream_launch<E, M, R, OPC>;
    e.stream_prepare = stream_prepare<E, M, R, OPC>;
    e.stream_tw = StreamShape<E, M, OPC>::TW;
    e.stream_nst = StreamShape<E, M, OPC>::NST;
    e.stream_batch_launch = stream_batch_launch<E, M, R, OPC>;
    e.stream_batch_prepare = stream_batch_prepare<E, M, R, OPC>;
    e.wpt_mask |= (unsigned)VARIANT_STREAMED;
}

/* division and fma2 run their streamed kernel only as single calls: no
 * job-list form */
template <int E, int M, int R, int OPC>
static void add_stream_single(BinopEntry& e) {
    e.stream_launch = stream_launch<E, M, R, OPC>;
    e.stream_prepare = stream_prepare<E, M, R, OPC>;
    e.stream_tw = StreamShape<E, M, OPC>::TW;
    e.stream_nst = StreamShape<E, M, OPC>::NST;
    e.wpt_mask |= (unsigned)VARIANT_STREAMED;
}

template <int E, int M, int R>
static void fill_stream_mode() {
    add_stream<E, M, R, OPC_ADDSUB>(g_binop_table[E][M][R][OPC_ADDSUB]);
    add_stream<E, M, R, OPC_MUL>(g_binop_table[E][M][R][OPC_MUL]);
    if constexpr (stream_div_format(E, M)) add_stream_single<E, M, R, OPC_DIV>(g_binop_table[E][M][R][OPC_DIV]);
    if constexpr (stream_fma2_format(E, M)) add_stream_single<E, M, R, OPC_FMA2>(g_binop_table[E][M][R][OPC_FMA2]);
}

#define BSFP_SCAT2(a, b) a##b
#define BSFP_SCAT(a, b) BSFP_SCAT2(a, b)

/* register_stream_e<E>_m<M>: called once by the dispatcher */
void BSFP_SCAT(BSFP_SCAT(BSFP_SCAT(register_stream_e, BSFP_SE), _m), BSFP_SM)() {
    fill_stream_mode<BSFP_SE, BSFP_SM, 0>();   /* RN */
    fill_stream_mode<BSFP_SE, BSFP_SM, 1>();   /* RZ */
    fill_stream_mode<BSFP_SE, BSFP_SM, 2>();   /* RN, flush to zero */
    fill_stream_mode<BSFP_SE, BSFP_SM, 3>();   /* RZ, flush to zero */
}

}  // namespace bsfp
