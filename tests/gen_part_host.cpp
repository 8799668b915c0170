/* Test harness: evaluates on the host the netlists circuitgen prints for the
 * formats outside the tuned set -- the add/mul header or the division header
 * of one exponent width and fraction range -- so that they can be compared
 * with the oracle on a CPU.  Compiled by the tests with -DBSFP_E=<E>,
 * -DBSFP_M_LO/-DBSFP_M_HI and -DBSFP_GEN_PART="<header>".  Test
 * infrastructure only; nothing in the library calls it. */
#include <stdint.h>

#include "gen_circuit.cuh"

using namespace bsfp;

template <int E, int M, int R, int OPC>
static int run(bool neg_b, const uint32_t* a, const uint32_t* b, uint32_t* out, long nwords, long S) {
    constexpr int B = 1 + E + M;
    if constexpr (B > 32 || !GenCircuit<E, M, R, OPC>::available) {
        return -1;
    } else {
        for (long w = 0; w < nwords; ++w) {
            uint32_t x[B], y[B], z[B], r[B];
            for (int i = 0; i < B; ++i) {
                x[i] = a[i * S + w];
                y[i] = b[i * S + w];
                z[i] = 0u;
            }
            if (neg_b) y[B - 1] = ~y[B - 1];
            GenCircuit<E, M, R, OPC>::eval(x, y, z, r);
            for (int i = 0; i < B; ++i) out[i * S + w] = r[i];
        }
        return 0;
    }
}

/* op: 0 add, 1 sub, 2 mul, 4 div (op classes 0, 0, 1, 3) */
template <int E, int M>
static int dispatch(int rnd, int op, const uint32_t* a, const uint32_t* b, uint32_t* out, long nwords, long S) {
    if (rnd == 0) {
        switch (op) {
            case 0: return run<E, M, 0, 0>(false, a, b, out, nwords, S);
            case 1: return run<E, M, 0, 0>(true, a, b, out, nwords, S);
            case 2: return run<E, M, 0, 1>(false, a, b, out, nwords, S);
            case 4: return run<E, M, 0, 3>(false, a, b, out, nwords, S);
        }
    } else if (rnd == 1) {
        switch (op) {
            case 0: return run<E, M, 1, 0>(false, a, b, out, nwords, S);
            case 1: return run<E, M, 1, 0>(true, a, b, out, nwords, S);
            case 2: return run<E, M, 1, 1>(false, a, b, out, nwords, S);
            case 4: return run<E, M, 1, 3>(false, a, b, out, nwords, S);
        }
    }
    return -1;
}

template <int M>
static int by_m(int m, int rnd, int op, const uint32_t* a, const uint32_t* b, uint32_t* out, long nwords, long S) {
    if (m == M) return dispatch<BSFP_E, M>(rnd, op, a, b, out, nwords, S);
    if constexpr (M < BSFP_M_HI) return by_m<M + 1>(m, rnd, op, a, b, out, nwords, S);
    return -1;
}

extern "C" int host_gen_part(int m, int rnd, int op, const uint32_t* a, const uint32_t* b, uint32_t* out, long nwords,
                             long S) {
    return by_m<BSFP_M_LO>(m, rnd, op, a, b, out, nwords, S);
}
