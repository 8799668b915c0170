/*
 * stream_mul_inst.cu -- the streamed kernel (stream.cuh) for mul under RN
 * and RZ of every format of 12 to 24 planes outside the tuned set, compiled
 * once per exponent width with -DBSFP_SE=E.  For formats of at most 16
 * planes it becomes the variant their mul calls take by default
 * (BinopEntry::preferred): measured over the sweep it beat the grid-stride
 * kernel in nearly every one of them.  For 17 to 24 planes it won for some
 * formats and lost for others (its 8 consumer warps have the registers of
 * the wide multipliers but hide less latency), so there the grid-stride
 * kernel stays the default and the autotuner picks per format and mode.
 * Calls too small to fill the ring fall back to the grid-stride default as
 * usual.  Registered after the grid-stride kernels, whose entries it
 * extends.
 */
#include "stream.cuh"

#ifndef BSFP_SE
#error "compile with -DBSFP_SE=<exponent bits>"
#endif

namespace bsfp {

template <int E, int M, int R>
static void add_stream_mul(BinopEntry& e) {
    e.stream_launch = stream_launch<E, M, R, OPC_MUL>;
    e.stream_prepare = stream_prepare<E, M, R, OPC_MUL>;
    e.stream_tw = StreamShape<E, M, OPC_MUL>::TW;
    e.stream_nst = StreamShape<E, M, OPC_MUL>::NST;
    e.wpt_mask |= (unsigned)VARIANT_STREAMED;
    if constexpr (1 + E + M <= 16) e.preferred = VARIANT_STREAMED;
}

template <int E, int M>
static void fill_stream_mul() {
    if constexpr (M <= 23 && stream_mul_format(E, M)) {
        add_stream_mul<E, M, 0>(g_binop_table[E][M][0][OPC_MUL]);
        add_stream_mul<E, M, 1>(g_binop_table[E][M][1][OPC_MUL]);
    }
    if constexpr (M < 23) fill_stream_mul<E, M + 1>();
}

#define BSFP_SMCAT2(a, b) a##b
#define BSFP_SMCAT(a, b) BSFP_SMCAT2(a, b)

/* register_stream_mul_e<E>: called once by the dispatcher */
void BSFP_SMCAT(register_stream_mul_e, BSFP_SE)() { fill_stream_mul<BSFP_SE, 1>(); }

}  // namespace bsfp
