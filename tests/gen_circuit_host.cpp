/* Test harness: evaluates the generated netlists of gen_circuits.cuh (the
 * gate-by-gate circuits the CUDA kernels run for the listed formats) on the
 * host with 32-bit words, so that they can be compared with the oracle on a
 * CPU.  Test infrastructure only; nothing in the library calls it.  Built by
 * tests/test_circuit_host.py with g++ after the build has generated the
 * header. */
#include <stdint.h>

#include "gen_circuit.cuh"

using namespace bsfp;

template <int E, int M, bool RZ, int OPC>
static int run(bool neg_b, const uint32_t* a, const uint32_t* b, const uint32_t* c, uint32_t* out, long nwords,
               long S) {
    constexpr int B = 1 + E + M;
    if constexpr (!GenCircuit<E, M, RZ, OPC>::available) {
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
            GenCircuit<E, M, RZ, OPC>::eval(x, y, z, r);
            for (int i = 0; i < B; ++i) out[i * S + w] = r[i];
        }
        return 0;
    }
}

template <int E, int M>
static int dispatch_fmt(int rz, int op, const uint32_t* a, const uint32_t* b, const uint32_t* c, uint32_t* out,
                        long nwords, long S) {
    /* op: 0 add, 1 sub, 2 mul, 3 fma2 -> op classes 0 (add/sub), 1, 2 */
    const bool neg = op == 1;
    switch ((op == 0 || op == 1 ? 0 : op - 1) * 2 + (rz ? 1 : 0)) {
        case 0: return run<E, M, false, 0>(neg, a, b, c, out, nwords, S);
        case 1: return run<E, M, true, 0>(neg, a, b, c, out, nwords, S);
        case 2: return run<E, M, false, 1>(neg, a, b, c, out, nwords, S);
        case 3: return run<E, M, true, 1>(neg, a, b, c, out, nwords, S);
        case 4: return run<E, M, false, 2>(neg, a, b, c, out, nwords, S);
        case 5: return run<E, M, true, 2>(neg, a, b, c, out, nwords, S);
    }
    return -1;
}

#define FMT(E, M) \
    if (e == E && m == M) return dispatch_fmt<E, M>(rz, op, a, b, c, out, nwords, S);

extern "C" int host_gen_circuit(int e, int m, int rz, int op, const uint32_t* a, const uint32_t* b,
                                const uint32_t* c, uint32_t* out, long nwords, long S) {
    FMT(4, 3) FMT(4, 4) FMT(5, 7) FMT(5, 10) FMT(8, 7) FMT(8, 23)
    return -1;
}
