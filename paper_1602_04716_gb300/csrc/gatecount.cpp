/*
 * gatecount.cpp -- counts the logic gates of the bitslice circuits.
 *
 * The circuits of circuit.cuh are recorded as netlists of 3-input gates (one
 * LOP3 each on sm_103a) by netlist.h, with inversions absorbed, constants and
 * repeated inputs folded, identical gates shared and dead gates dropped.  The
 * result G(op, E, M, rounding) is the number of 3-input logic instructions per 32-element word of the circuit as
 * built -- the "work" term of the logic-throughput roofline.  Table 1 of the
 * paper gives the asymptotic classes (add O(n log n), mul O(n^2)); this file
 * gives the exact constants.
 *
 * Host code only; it computes no arithmetic results.  Compiled once per
 * exponent width E with -DBSFP_E=E.
 */
#include "netlist.h"

namespace bsfp {
namespace gc {
namespace {

template <int E, int M, int R, int OP> static long count_one() {
    constexpr int B = 1 + E + M;
    Graph g, mg;
    GW r[B], mr[B];
    record<E, M, R, OP>(g, r);
    lut3_map(g, r, B, mg, mr);
    return count_live(mg, mr, B);
}

template <int E, int M, int OP> static long count_op(int rnd) {
    switch (rnd) {
        case 0: return count_one<E, M, 0, OP>();
        case 1: return count_one<E, M, 1, OP>();
        case 2: return count_one<E, M, 2, OP>();
        case 3: return count_one<E, M, 3, OP>();
    }
    return -1;
}

/* rnd: rounding mode (bit 0 toward zero, bit 1 flush to zero) */
template <int E, int M> static long count_fmt(int rnd, int op) {
    if constexpr (E + M + 1 > 32) {
        return -1;
    } else {
        switch (op) {
            case 0: return count_op<E, M, OP_ADD>(rnd);
            case 1: return count_op<E, M, OP_SUB>(rnd);
            case 2: return count_op<E, M, OP_MUL>(rnd);
            case 3: return count_op<E, M, OP_FMA2>(rnd);
            case 4: return count_op<E, M, OP_DIV>(rnd);
        }
        return -1;
    }
}

template <int E, int M> static long count_m(int m, int rnd, int op) {
    if (m == M) return count_fmt<E, M>(rnd, op);
    if constexpr (M < 23) return count_m<E, M + 1>(m, rnd, op);
    return -1;
}

}  // namespace
}  // namespace gc
}  // namespace bsfp

/* One translation unit per exponent width (-DBSFP_E=E), so that the
 * 23 x 8 instantiations of each E compile in parallel with the others. */
#ifndef BSFP_E
#error "compile with -DBSFP_E=<exponent bits>"
#endif
#define BSFP_GC_CAT2(a, b) a##b
#define BSFP_GC_CAT(a, b) BSFP_GC_CAT2(a, b)

extern "C" long BSFP_GC_CAT(bsfp_gate_count_e, BSFP_E)(int man_bits, int rnd, int op) {
    if (man_bits < 1 || man_bits > 23 || op < 0 || op > 4 || rnd < 0 || rnd > 3) return -1;
    return bsfp::gc::count_m<BSFP_E, 1>(man_bits, rnd, op);
}

#if BSFP_E == 2
/* Gates per word of the w-bit integer ops (compiled once, with the E = 2 unit). */
namespace bsfp {
namespace gc {
namespace {
template <int w> static long count_int(int bits, int op) {
    if (bits == w) {
        Graph g;
        GW r[w];
        if (op == 0) record_int<w, IOP_ADD>(g, r);
        else if (op == 1) record_int<w, IOP_SUB>(g, r);
        else record_int<w, IOP_MUL>(g, r);
        return count_live(g, r, w);
    }
    if constexpr (w < 32) return count_int<w + 1>(bits, op);
    return -1;
}
}  // namespace
}  // namespace gc
}  // namespace bsfp

extern "C" long bsfp_int_gate_count_impl(int bits, int op) {
    if (bits < 1 || bits > 32 || op < 0 || op > 2) return -1;
    return bsfp::gc::count_int<1>(bits, op);
}
#endif
