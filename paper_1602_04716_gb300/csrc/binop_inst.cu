/*
 * binop_inst.cu -- instantiates the element-wise kernels for one exponent
 * width.  The build compiles this file once per E in [2, 8] with -DBSFP_E=E,
 * so the 7 translation units build in parallel; each fills its slice of the
 * dispatch table for M in [BSFP_M_LO, BSFP_M_HI], both rounding modes and the
 * three kernel classes (add/sub, mul, fma2).  This replaces the paper's
 * library generator (Sec. 5.1), which emitted code per configured format.
 */
#include "binop.cuh"

#ifndef BSFP_E
#error "compile with -DBSFP_E=<exponent bits>"
#endif
#ifndef BSFP_M_LO
#define BSFP_M_LO 1
#endif
#ifndef BSFP_M_HI
#define BSFP_M_HI 23
#endif

namespace bsfp {

template <int E, int M>
static void fill_format() {
    if constexpr (M >= BSFP_M_LO && M <= BSFP_M_HI && 1 + E + M <= 32) {
        g_binop_table[E][M][0][OPC_ADDSUB] = make_entry<E, M, false, OPC_ADDSUB>();
        g_binop_table[E][M][1][OPC_ADDSUB] = make_entry<E, M, true, OPC_ADDSUB>();
        g_binop_table[E][M][0][OPC_MUL] = make_entry<E, M, false, OPC_MUL>();
        g_binop_table[E][M][1][OPC_MUL] = make_entry<E, M, true, OPC_MUL>();
        g_binop_table[E][M][0][OPC_FMA2] = make_entry<E, M, false, OPC_FMA2>();
        g_binop_table[E][M][1][OPC_FMA2] = make_entry<E, M, true, OPC_FMA2>();
    }
    if constexpr (M < BSFP_M_HI) fill_format<E, M + 1>();
}

#define BSFP_CAT2(a, b) a##b
#define BSFP_CAT(a, b) BSFP_CAT2(a, b)
#define BSFP_CAT3(a, b, c) BSFP_CAT(BSFP_CAT(a, b), c)

/* register_e<E>_m<LO>: called once by the dispatcher */
void BSFP_CAT3(BSFP_CAT(register_e, BSFP_E), _m, BSFP_M_LO)() { fill_format<BSFP_E, BSFP_M_LO>(); }

}  // namespace bsfp
