/*
 * stream_band_inst.cu -- the streamed kernel (stream.cuh) for one op class
 * under RN and RZ of the formats outside the tuned set that fall in that
 * class's band, compiled once per exponent width and op class with
 * -DBSFP_SE=E -DBSFP_SOPC=<1 mul, 2 fma2, 3 div>.
 *
 *   mul, 12 to 24 planes: for formats of at most 20 planes it becomes the
 *     variant a mul call takes by default (BinopEntry::preferred): measured
 *     over the sweep it beat the grid-stride kernel in nearly every one of
 *     those up to 16 planes, and with 11 consumer warps it was 4-10% faster
 *     on six multipliers of 17-20 planes.  For 21 to 24 planes (8 consumer
 *     warps, all the ring holds) it won for some formats and lost for
 *     others, so there the grid-stride kernel stays the default and the
 *     autotuner picks per format and mode.
 *   div, 8 to 24 planes and at least 3 fraction bits: the default from 4
 *     fraction bits on, where over the sweep (2^26 elements) it was faster
 *     than the grid-stride kernel in all but two of the 82 format-modes of
 *     8-17 planes (median 4.5%, up to 11%; the other two within 0.3%), and
 *     on seven dividers of 18-22 planes by 1-6%.  With 3 fraction
 *     bits it won under RN and lost under RZ by up to 5%, so there the
 *     autotuner picks; with 2 it lost everywhere and is not compiled.
 *   fma2, 10 to 19 planes and at least 4 fraction bits: the default
 *     throughout (9-14% faster than the grid-stride kernel on nine formats
 *     of 11 to 17 planes; over the sweep, with 2 or 3 fraction bits, where
 *     fma2 is HBM-bound, it was up to 11% slower).
 *
 * Calls too small to fill the ring fall back to the grid-stride default as
 * usual.  Registered after the grid-stride kernels, whose entries it
 * extends.
 */
#include "stream.cuh"

#if !defined(BSFP_SE) || !defined(BSFP_SOPC)
#error "compile with -DBSFP_SE=<exponent bits> -DBSFP_SOPC=<op class>"
#endif

namespace bsfp {

static_assert(BSFP_SOPC == OPC_MUL || BSFP_SOPC == OPC_FMA2 || BSFP_SOPC == OPC_DIV, "op classes with a streamed band");

template <int E, int M, int R, int OPC>
static void add_stream_band(BinopEntry& e) {
    e.stream_launch = stream_launch<E, M, R, OPC>;
    e.stream_prepare = stream_prepare<E, M, R, OPC>;
    e.stream_tw = StreamShape<E, M, OPC>::TW;
    e.stream_nst = StreamShape<E, M, OPC>::NST;
    e.wpt_mask |= (unsigned)VARIANT_STREAMED;
    if constexpr (OPC == OPC_DIV ? M >= 4 : (OPC == OPC_FMA2 || 1 + E + M <= 20)) e.preferred = VARIANT_STREAMED;
}

template <int E, int M, int OPC>
static void fill_stream_band() {
    if constexpr (M <= 23 && !tuned_format(E, M) && stream_band_format(E, M, OPC)) {
        add_stream_band<E, M, 0, OPC>(g_binop_table[E][M][0][OPC]);
        add_stream_band<E, M, 1, OPC>(g_binop_table[E][M][1][OPC]);
    }
    if constexpr (M < 23) fill_stream_band<E, M + 1, OPC>();
}

#define BSFP_SBCAT2(a, b) a##b
#define BSFP_SBCAT(a, b) BSFP_SBCAT2(a, b)

/* register_stream_{mul,fma2,div}_e<E>: called once by the dispatcher */
#if BSFP_SOPC == 1
void BSFP_SBCAT(register_stream_mul_e, BSFP_SE)() { fill_stream_band<BSFP_SE, 1, OPC_MUL>(); }
#elif BSFP_SOPC == 2
void BSFP_SBCAT(register_stream_fma2_e, BSFP_SE)() { fill_stream_band<BSFP_SE, 1, OPC_FMA2>(); }
#else
void BSFP_SBCAT(register_stream_div_e, BSFP_SE)() { fill_stream_band<BSFP_SE, 1, OPC_DIV>(); }
#endif

}  // namespace bsfp
