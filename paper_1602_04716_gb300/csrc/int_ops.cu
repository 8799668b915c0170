/*
 * int_ops.cu -- the integer bitslice vectors of Sec. 3: w-bit unsigned (or
 * two's-complement) integers, 1 <= w <= 32, in the same plane-major layout
 * as the floats (B = w planes), added, subtracted and multiplied modulo 2^w
 * by the circuits of circuit.cuh (the Fig. 2 ripple adder; a carry-save
 * array kept to the low w columns).  The kernel is the element-wise kernel
 * of binop.cuh in miniature: each thread loads WPT words of every input
 * plane with one vector load, runs the circuit per word in registers and
 * stores the w result planes; the partly filled last column keeps its valid
 * lanes and padding columns are written as zero.
 *
 * Compiled twice, for w in [BSFP_W_LO, BSFP_W_HI] (1..16 and 17..32).
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "binop.cuh"
#include "circuit.cuh"

#ifndef BSFP_W_LO
#define BSFP_W_LO 1
#define BSFP_W_HI 32
#endif

namespace bsfp {

typedef cudaError_t (*int_launch_fn)(const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t S, int64_t nwords,
                                     uint32_t tailmask, int grid, cudaStream_t s);

template <int w, int OP, int WPT>
__global__ void __launch_bounds__(128) int_kernel(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b,
                                                  uint32_t* __restrict__ out, int64_t S, int64_t nwords,
                                                  uint32_t tailmask) {
    const int64_t nchunks = S / WPT;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < nchunks; ch += stride) {
        const int64_t w0 = ch * WPT;
        uint32_t xa[w][WPT], xb[w][WPT], r[w][WPT];
#pragma unroll
        for (int i = 0; i < w; ++i) vload<WPT>(a + i * S + w0, xa[i]);
#pragma unroll
        for (int i = 0; i < w; ++i) vload<WPT>(b + i * S + w0, xb[i]);
#pragma unroll
        for (int k = 0; k < WPT; ++k) {
            uint32_t x[w], y[w], o[w];
#pragma unroll
            for (int i = 0; i < w; ++i) {
                x[i] = xa[i][k];
                y[i] = xb[i][k];
            }
            int_op<w, OP>(x, y, o);
#pragma unroll
            for (int i = 0; i < w; ++i) r[i][k] = o[i];
        }
        if (w0 + WPT >= nwords) {
#pragma unroll
            for (int k = 0; k < WPT; ++k) {
                const int64_t wd = w0 + k;
                const uint32_t m = (wd + 1 < nwords) ? ~0u : (wd + 1 == nwords ? tailmask : 0u);
#pragma unroll
                for (int i = 0; i < w; ++i) r[i][k] &= m;
            }
        }
#pragma unroll
        for (int i = 0; i < w; ++i) vstore<WPT>(out + i * S + w0, r[i]);
    }
}

template <int w, int OP>
static cudaError_t int_launch(const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t S, int64_t nwords,
                              uint32_t tailmask, int grid, cudaStream_t s) {
    constexpr int WPT = (w <= 16) ? 4 : 2;
    int_kernel<w, OP, WPT><<<grid, 128, 0, s>>>(a, b, out, S, nwords, tailmask);
    return cudaGetLastError();
}

extern int_launch_fn g_int_table[33][3];

template <int w>
static void fill_int() {
    if constexpr (w >= BSFP_W_LO && w <= BSFP_W_HI) {
        g_int_table[w][IOP_ADD] = int_launch<w, IOP_ADD>;
        g_int_table[w][IOP_SUB] = int_launch<w, IOP_SUB>;
        g_int_table[w][IOP_MUL] = int_launch<w, IOP_MUL>;
    }
    if constexpr (w < BSFP_W_HI) fill_int<w + 1>();
}

#define BSFP_ICAT2(a, b) a##b
#define BSFP_ICAT(a, b) BSFP_ICAT2(a, b)
void BSFP_ICAT(register_int_w, BSFP_W_LO)() { fill_int<BSFP_W_LO>(); }

}  // namespace bsfp
