/* Test harness: evaluates the bitslice circuits of the CUDA library's
 * circuit.cuh on the host with 32-bit words, so that the circuit logic can be
 * compared with the oracle on a CPU (the GPU parity tests run the same
 * templates inside the kernels).  Test infrastructure only; nothing in the
 * library calls it.  Built by tests/_helpers.py with g++. */
#include <stdint.h>

#include "circuit.cuh"

using namespace bsfp;

template <int E, int M, int R, int OP>
static void run(const uint32_t* a, const uint32_t* b, const uint32_t* c, uint32_t* out, long nwords, long S) {
    constexpr int B = 1 + E + M;
    for (long w = 0; w < nwords; ++w) {
        uint32_t x[B], y[B], z[B], r[B];
        for (int i = 0; i < B; ++i) {
            x[i] = a[i * S + w];
            y[i] = b[i * S + w];
            z[i] = c[i * S + w];
        }
        fp_op<E, M, R, OP>(x, y, z, r);
        for (int i = 0; i < B; ++i) out[i * S + w] = r[i];
    }
}

template <int E, int M, int OP>
static int dispatch_mode(int rnd, const uint32_t* a, const uint32_t* b, const uint32_t* c, uint32_t* out, long nwords,
                         long S) {
    switch (rnd) {
        case 0: run<E, M, 0, OP>(a, b, c, out, nwords, S); return 0;
        case 1: run<E, M, 1, OP>(a, b, c, out, nwords, S); return 0;
        case 2: run<E, M, 2, OP>(a, b, c, out, nwords, S); return 0;
        case 3: run<E, M, 3, OP>(a, b, c, out, nwords, S); return 0;
    }
    return -1;
}

/* rnd: rounding mode (bit 0 toward zero, bit 1 flush to zero) */
template <int E, int M>
static int dispatch_fmt(int rnd, int op, const uint32_t* a, const uint32_t* b, const uint32_t* c, uint32_t* out,
                        long nwords, long S) {
    switch (op) {
        case 0: return dispatch_mode<E, M, OP_ADD>(rnd, a, b, c, out, nwords, S);
        case 1: return dispatch_mode<E, M, OP_SUB>(rnd, a, b, c, out, nwords, S);
        case 2: return dispatch_mode<E, M, OP_MUL>(rnd, a, b, c, out, nwords, S);
        case 3: return dispatch_mode<E, M, OP_FMA2>(rnd, a, b, c, out, nwords, S);
        case 4: return dispatch_mode<E, M, OP_DIV>(rnd, a, b, c, out, nwords, S);
    }
    return -1;
}

template <int E, int M, int R>
static void run_conv(int dir, const uint32_t* a, uint32_t* out, long nwords, long S) {
    constexpr int B = 1 + E + M;
    for (long w = 0; w < nwords; ++w) {
        uint32_t x[32], r[32];
        if (dir == 0) {   /* binary32 (32 planes) -> 1/E/M */
            for (int i = 0; i < 32; ++i) x[i] = a[i * S + w];
            from_f32<E, M, mode_rz(R), mode_ftz(R)>(x, r);
            for (int i = 0; i < B; ++i) out[i * S + w] = r[i];
        } else {          /* 1/E/M -> binary32 */
            for (int i = 0; i < B; ++i) x[i] = a[i * S + w];
            to_f32<E, M, mode_ftz(R)>(x, r);
            for (int i = 0; i < 32; ++i) out[i * S + w] = r[i];
        }
    }
}

template <int E, int M>
static int dispatch_conv(int rnd, int dir, const uint32_t* a, uint32_t* out, long nwords, long S) {
    switch (rnd) {
        case 0: run_conv<E, M, 0>(dir, a, out, nwords, S); return 0;
        case 1: run_conv<E, M, 1>(dir, a, out, nwords, S); return 0;
        case 2: run_conv<E, M, 2>(dir, a, out, nwords, S); return 0;
        case 3: run_conv<E, M, 3>(dir, a, out, nwords, S); return 0;
    }
    return -1;
}

#define FMT(E, M) \
    if (e == E && m == M) return dispatch_fmt<E, M>(rnd, op, a, b, c, out, nwords, S);

extern "C" int host_circuit(int e, int m, int rnd, int op, const uint32_t* a, const uint32_t* b, const uint32_t* c,
                            uint32_t* out, long nwords, long S) {
    /* the formats the CPU tests exercise */
    FMT(2, 1) FMT(2, 3) FMT(3, 2) FMT(3, 3) FMT(2, 5) FMT(3, 4) FMT(4, 3) FMT(5, 2) FMT(4, 4) FMT(5, 4)
    FMT(4, 5) FMT(5, 7) FMT(5, 10) FMT(8, 7) FMT(8, 23) FMT(3, 23) FMT(8, 2) FMT(6, 9) FMT(7, 13)
    FMT(2, 23) FMT(8, 1) FMT(3, 12)
    return -1;
}

#define FMTC(E, M) \
    if (e == E && m == M) return dispatch_conv<E, M>(rnd, dir, a, out, nwords, S);

/* dir 0: binary32 planes in (32 x S), 1/E/M planes out; dir 1: the reverse */
extern "C" int host_convert(int e, int m, int rnd, int dir, const uint32_t* a, uint32_t* out, long nwords, long S) {
    FMTC(2, 1) FMTC(3, 2) FMTC(4, 3) FMTC(5, 2) FMTC(3, 4) FMTC(4, 4) FMTC(5, 7) FMTC(5, 10) FMTC(8, 7)
    FMTC(8, 23) FMTC(6, 9) FMTC(7, 13) FMTC(3, 23) FMTC(2, 23) FMTC(8, 1)
    return -1;
}

template <int w>
static int run_int(int op, const uint32_t* a, const uint32_t* b, uint32_t* out, long nwords, long S) {
    if constexpr (w > 32) {
        return -1;
    } else {
        for (long k = 0; k < nwords; ++k) {
            uint32_t x[w], y[w], r[w];
            for (int i = 0; i < w; ++i) {
                x[i] = a[i * S + k];
                y[i] = b[i * S + k];
            }
            if (op == 0) int_op<w, IOP_ADD>(x, y, r);
            else if (op == 1) int_op<w, IOP_SUB>(x, y, r);
            else int_op<w, IOP_MUL>(x, y, r);
            for (int i = 0; i < w; ++i) out[i * S + k] = r[i];
        }
        return 0;
    }
}

template <int w>
static int dispatch_int(int bits, int op, const uint32_t* a, const uint32_t* b, uint32_t* out, long nwords, long S) {
    if (bits == w) return run_int<w>(op, a, b, out, nwords, S);
    if constexpr (w < 32) return dispatch_int<w + 1>(bits, op, a, b, out, nwords, S);
    return -1;
}

/* w-bit integer vectors: op 0 add, 1 sub, 2 mul */
extern "C" int host_int(int bits, int op, const uint32_t* a, const uint32_t* b, uint32_t* out, long nwords, long S) {
    return dispatch_int<1>(bits, op, a, b, out, nwords, S);
}
