/*
 * binop_inst.cu -- instantiates the element-wise kernels for one exponent
 * width.  The build compiles this file once per E in [2, 8] with -DBSFP_E=E,
 * so the 7 translation units build in parallel; each fills its slice of the
 * dispatch table for M in [BSFP_M_LO, BSFP_M_HI], both rounding modes (and
 * their flush-to-zero forms for the tuned formats) and the four kernel
 * classes (add/sub, mul, fma2, div).  This replaces the paper's
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

/* Op classes this unit instantiates: all four, or only division
 * (-DBSFP_DIV_UNIT, a unit of its own so that the printed division circuits
 * compile in parallel with the others), or all but division
 * (-DBSFP_NO_DIV, the units that a division unit pairs with). */
#if defined(BSFP_DIV_UNIT)
constexpr bool unit_has(int opc) { return opc == OPC_DIV; }
#elif defined(BSFP_NO_DIV)
constexpr bool unit_has(int opc) { return opc != OPC_DIV; }
#else
constexpr bool unit_has(int) { return true; }
#endif

template <int E, int M, int R>
static void fill_mode() {
    if constexpr (unit_has(OPC_ADDSUB)) g_binop_table[E][M][R][OPC_ADDSUB] = make_entry<E, M, R, OPC_ADDSUB>();
    if constexpr (unit_has(OPC_MUL)) g_binop_table[E][M][R][OPC_MUL] = make_entry<E, M, R, OPC_MUL>();
    if constexpr (unit_has(OPC_FMA2)) g_binop_table[E][M][R][OPC_FMA2] = make_entry<E, M, R, OPC_FMA2>();
    if constexpr (unit_has(OPC_DIV)) g_binop_table[E][M][R][OPC_DIV] = make_entry<E, M, R, OPC_DIV>();
}

template <int E, int M>
static void fill_format() {
    if constexpr (M >= BSFP_M_LO && M <= BSFP_M_HI && 1 + E + M <= 32) {
        fill_mode<E, M, 0>();   /* RN */
        fill_mode<E, M, 1>();   /* RZ */
        /* the flush-to-zero modes are compiled for the tuned formats only */
        if constexpr (tuned_format(E, M)) {
            fill_mode<E, M, 2>();
            fill_mode<E, M, 3>();
        }
    }
    if constexpr (M < BSFP_M_HI) fill_format<E, M + 1>();
}

#define BSFP_CAT2(a, b) a##b
#define BSFP_CAT(a, b) BSFP_CAT2(a, b)
#define BSFP_CAT3(a, b, c) BSFP_CAT(BSFP_CAT(a, b), c)

/* register_e<E>_m<LO> (register_div_e<E>_m<LO> for a division unit):
 * called once by the dispatcher */
#if defined(BSFP_DIV_UNIT)
void BSFP_CAT3(BSFP_CAT(register_div_e, BSFP_E), _m, BSFP_M_LO)() { fill_format<BSFP_E, BSFP_M_LO>(); }
#else
void BSFP_CAT3(BSFP_CAT(register_e, BSFP_E), _m, BSFP_M_LO)() { fill_format<BSFP_E, BSFP_M_LO>(); }
#endif

}  // namespace bsfp
