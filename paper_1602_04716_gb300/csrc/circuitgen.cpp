/*
 * circuitgen.cpp -- build-time tool: prints the netlists of chosen circuits
 * as straight-line code with one 3-input logic instruction per gate.
 *
 * The circuits are written once, as the templates of circuit.cuh.  Recorded
 * by netlist.h they become netlists in which every gate is a function of at
 * most three words with its truth table, inversions absorbed, constants
 * folded, identical gates shared and dead gates dropped, and then re-covered
 * by 3-input functions (lut3_map in netlist.h), which merges a gate into its
 * user wherever the two read at most three values -- G gates in all.
 * Left to the compiler, the same templates become more instructions than
 * that, because it re-derives its own 3-input groupings from the and/or/xor
 * expressions (a majority gate that shares x^y with the neighbouring sum, for
 * example, costs two instructions instead of one).  Printing the netlist
 * gate by gate as BSFP_LOP3(truth table, x, y, z) fixes the instruction count
 * at G.  This plays the part of the paper's generator (Sec. 5.1: a
 * configuration of formats in, generated code for them out).
 *
 * Usage: circuitgen OUT.cuh    (formats from -DBSFP_GEN_FORMATS="X(E, M) ...",
 *                               -DBSFP_GEN_ADDMUL="Y(E, M) ..." and/or
 *                               -DBSFP_GEN_DIV="Z(E, M) ...")
 *
 * For each X format and rounding mode R (bit 0 toward zero, bit 1 flush to
 * zero) it prints GenCircuit<E, M, R, OPC>
 * specialisations for the op classes add (b's sign flip is applied by the
 * caller), mul, fma2 and div, with eval(a, b, c, r) over the B slices of each
 * operand.  For each Y format it prints add and mul under RN and RZ only (the
 * kernels compose fma2 from those two), and for each Z format div under RN
 * and RZ.  The printed file is included inside
 * namespace bsfp by gen_circuit.cuh, which defines BSFP_LOP3 and
 * BSFP_GEN_FN.
 */
#include <stdio.h>

#include <string>

#include "netlist.h"

#if !defined(BSFP_GEN_FORMATS) && !defined(BSFP_GEN_ADDMUL) && !defined(BSFP_GEN_DIV)
#error "compile with -DBSFP_GEN_FORMATS=\"X(E, M) ...\", -DBSFP_GEN_ADDMUL=\"Y(E, M) ...\" or -DBSFP_GEN_DIV=\"Z(E, M) ...\""
#endif
#ifndef BSFP_GEN_FORMATS
#define BSFP_GEN_FORMATS
#endif
#ifndef BSFP_GEN_ADDMUL
#define BSFP_GEN_ADDMUL
#endif
#ifndef BSFP_GEN_DIV
#define BSFP_GEN_DIV
#endif

namespace bsfp {
namespace gc {
namespace {

/* Name of a value: constant, operand slice a/b/c[i], or gate g<id>. */
std::string value_name(int32_t ref, int B) {
    const int32_t id = ref >> 1;
    const bool inv = ref & 1;
    std::string s;
    if (id == 0) return inv ? "0xFFFFFFFFu" : "0u";
    if (id <= B) {
        s = "a[" + std::to_string(id - 1) + "]";
    } else if (id <= 2 * B) {
        s = "b[" + std::to_string(id - 1 - B) + "]";
    } else if (id <= 3 * B) {
        s = "c[" + std::to_string(id - 1 - 2 * B) + "]";
    } else {
        s = "g" + std::to_string(id);
    }
    return inv ? "~" + s : s;
}

template <int E, int M, int R, int OP>
void emit(FILE* f, int opc) {
    constexpr int B = 1 + E + M;
    Graph rec;
    GW rr[B];
    record<E, M, R, OP>(rec, rr);
    Graph g;
    GW r[B];
    lut3_map(rec, rr, B, g, r);
    const std::vector<char> live = live_set(g, r, B);
    long n = 0;
    for (char m : live) n += m;
    fprintf(f, "template <> struct GenCircuit<%d, %d, %d, %d> {\n", E, M, R, opc);
    fprintf(f, "    static constexpr bool available = true;\n");
    fprintf(f, "    static constexpr int gates = %ld;\n", n);
    fprintf(f, "    BSFP_GEN_FN static void eval(const uint32_t* a, const uint32_t* b, const uint32_t* c, uint32_t* r) {\n");
    fprintf(f, "        (void)a; (void)b; (void)c;\n");
    const int first = g.ninputs + 1;
    for (size_t idx = 0; idx < g.lut.size(); ++idx) {
        if (!live[idx]) continue;
        const int32_t id = first + (int32_t)idx;
        std::string x[3];
        for (int k = 0; k < 3; ++k) x[k] = g.in[k][idx] >= 0 ? value_name(g.in[k][idx], B) : std::string();
        /* an unused slot is a don't-care of the truth table: repeat slot a */
        for (int k = 1; k < 3; ++k)
            if (x[k].empty()) x[k] = x[0];
        fprintf(f, "        const uint32_t g%d = BSFP_LOP3(0x%02X, %s, %s, %s);\n", id, (unsigned)g.lut[idx],
                x[0].c_str(), x[1].c_str(), x[2].c_str());
    }
    for (int i = 0; i < B; ++i) fprintf(f, "        r[%d] = %s;\n", i, value_name(r[i].ref, B).c_str());
    fprintf(f, "    }\n};\n");
}

template <int E, int M, int R>
void emit_mode(FILE* f) {
    /* op classes: 0 = add/sub, 1 = mul, 2 = fma2, 3 = div (OpClass of binop.cuh) */
    emit<E, M, R, OP_ADD>(f, 0);
    emit<E, M, R, OP_MUL>(f, 1);
    emit<E, M, R, OP_FMA2>(f, 2);
    emit<E, M, R, OP_DIV>(f, 3);
}

/* every rounding mode: RN, RZ, and both with flush to zero */
template <int E, int M>
void emit_format(FILE* f) {
    emit_mode<E, M, 0>(f);
    emit_mode<E, M, 1>(f);
    emit_mode<E, M, 2>(f);
    emit_mode<E, M, 3>(f);
}

/* add and mul, RN and RZ */
template <int E, int M>
void emit_addmul(FILE* f) {
    emit<E, M, 0, OP_ADD>(f, 0);
    emit<E, M, 0, OP_MUL>(f, 1);
    emit<E, M, 1, OP_ADD>(f, 0);
    emit<E, M, 1, OP_MUL>(f, 1);
}

/* div, RN and RZ */
template <int E, int M>
void emit_div(FILE* f) {
    emit<E, M, 0, OP_DIV>(f, 3);
    emit<E, M, 1, OP_DIV>(f, 3);
}

}  // namespace
}  // namespace gc
}  // namespace bsfp

int main(int argc, char** argv) {
    if (argc != 2) {
        fprintf(stderr, "usage: %s OUT.cuh\n", argv[0]);
        return 2;
    }
    FILE* f = fopen(argv[1], "w");
    if (!f) {
        perror(argv[1]);
        return 1;
    }
    fprintf(f, "/* Generated by circuitgen from the circuits of circuit.cuh; do not edit. */\n");
    fprintf(f, "#define BSFP_GEN_HAVE_FORMATS 1\n");
#define X(E, M) bsfp::gc::emit_format<E, M>(f);
    BSFP_GEN_FORMATS
#undef X
#define Y(E, M) bsfp::gc::emit_addmul<E, M>(f);
    BSFP_GEN_ADDMUL
#undef Y
#define Z(E, M) bsfp::gc::emit_div<E, M>(f);
    BSFP_GEN_DIV
#undef Z
    if (fclose(f) != 0) {
        perror(argv[1]);
        return 1;
    }
    return 0;
}
