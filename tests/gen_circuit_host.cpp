/* Test harness: evaluates the generated netlists of gen_circuits.cuh (the
 * gate-by-gate circuits the CUDA kernels run for the listed formats) on the
 * host with 32-bit words, so that they can be compared with the oracle on a
 * CPU.  Test infrastructure only; nothing in the library calls it.  Built by
 * tests/test_circuit_host.py with g++ after the build has generated the
 * header. */
#include <stdint.h>

#include "gen_circuit.cuh"

using namespace bsfp;

template <int E, int M, int R, int OPC>
static int run(bool neg_b, const uint32_t* a, const uint32_t* b, const uint32_t* c, uint32_t* out, long nwords,
               long S) {
    constexpr int B = 1 + E + M;
    if constexpr (!GenCircuit<E, M, R, OPC>::available) {
        return -1;
    } else {
        for (long w = 0; w < nwords; ++w) {
            uint32_t x[B], y[B], z[B], r[B];
            for (int i = 0; i < B; ++i) {
                x[i] = a[i * S + w];
                y[i] = b[i * S + w];
                z[i] = c[i * S + w];
            }
            if (neg_b) y[B - 1] = ~y[B - 1];
            GenCircuit<E, M, R, OPC>::eval(x, y, z, r);
            for (int i = 0; i < B; ++i) out[i * S + w] = r[i];
        }
        return 0;
    }
}

template <int E, int M, int R>
static int dispatch_opc(int op, const uint32_t* a, const uint32_t* b, const uint32_t* c, uint32_t* out, long nwords,
                        long S) {
    /* op: 0 add, 1 sub, 2 mul, 3 fma2, 4 div -> op classes 0 (add/sub), 1, 2, 3 */
    switch (op) {
        case 0: return run<E, M, R, 0>(false, a, b, c, out, nwords, S);
        case 1: return run<E, M, R, 0>(true, a, b, c, out, nwords, S);
        case 2: return run<E, M, R, 1>(false, a, b, c, out, nwords, S);
        case 3: return run<E, M, R, 2>(false, a, b, c, out, nwords, S);
        case 4: return run<E, M, R, 3>(false, a, b, c, out, nwords, S);
    }
    return -1;
}

/* rnd: rounding mode (bit 0 toward zero, bit 1 flush to zero) */
template <int E, int M>
static int dispatch_fmt(int rnd, int op, const uint32_t* a, const uint32_t* b, const uint32_t* c, uint32_t* out,
                        long nwords, long S) {
    switch (rnd) {
        case 0: return dispatch_opc<E, M, 0>(op, a, b, c, out, nwords, S);
        case 1: return dispatch_opc<E, M, 1>(op, a, b, c, out, nwords, S);
        case 2: return dispatch_opc<E, M, 2>(op, a, b, c, out, nwords, S);
        case 3: return dispatch_opc<E, M, 3>(op, a, b, c, out, nwords, S);
    }
    return -1;
}

#define FMT(E, M) \
    if (e == E && m == M) return dispatch_fmt<E, M>(rnd, op, a, b, c, out, nwords, S);

extern "C" int host_gen_circuit(int e, int m, int rnd, int op, const uint32_t* a, const uint32_t* b,
                                const uint32_t* c, uint32_t* out, long nwords, long S) {
    FMT(4, 3) FMT(4, 4) FMT(5, 7) FMT(5, 10) FMT(8, 7) FMT(8, 23)
    return -1;
}
