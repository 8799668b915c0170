/*
 * conv_inst.cu -- instantiates the fused float conversions for one exponent
 * width (compiled once per E in [2, 8] with -DBSFP_E=E): every M, both
 * roundings, and the flush-to-zero modes for the formats compiled with them.
 */
#include "binop.cuh"
#include "convert.cuh"

#ifndef BSFP_E
#error "compile with -DBSFP_E=<exponent bits>"
#endif

namespace bsfp {

template <int E, int M, int R>
static void fill_conv_mode() {
    /* the widening direction depends on flush to zero only */
    g_conv_table[E][M][R] = ConvEntry{launch_from_float<E, M, R>, launch_to_float<E, M, R & 2>};
}

template <int E, int M>
static void fill_conv() {
    if constexpr (1 + E + M <= 32) {
        fill_conv_mode<E, M, 0>();
        fill_conv_mode<E, M, 1>();
        if constexpr (tuned_format(E, M)) {
            fill_conv_mode<E, M, 2>();
            fill_conv_mode<E, M, 3>();
        }
    }
    if constexpr (M < 23) fill_conv<E, M + 1>();
}

#define BSFP_CCAT2(a, b) a##b
#define BSFP_CCAT(a, b) BSFP_CCAT2(a, b)

void BSFP_CCAT(register_conv_e, BSFP_E)() { fill_conv<BSFP_E, 1>(); }

}  // namespace bsfp
