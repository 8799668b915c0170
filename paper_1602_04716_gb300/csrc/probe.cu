/*
 * probe.cu -- the logic-issue probe declared in bsfp_bench.h.
 *
 * Each thread runs 8 independent chains; a chain is three words updated in
 * turn through XOR3, majority and select -- the three gate shapes the
 * circuits use most -- so that no update cancels the one before it.  Eight
 * chains give each warp enough independent instructions to keep the logic
 * pipe busy; the result is stored so that nothing is dead.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "bsfp_bench.h"

namespace bsfp {

template <unsigned L>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm volatile("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(L));
    return d;
}

__global__ void lop3_probe_kernel(uint32_t* sink, int iters, uint32_t seed) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t x[8], y[8], z[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        x[k] = seed ^ (t * 0x9E3779B9u) ^ (k * 0x85EBCA6Bu);
        y[k] = x[k] * 0xC2B2AE35u + k;
        z[k] = y[k] ^ (x[k] >> 7);
    }
    for (int it = 0; it < iters; ++it) {
        /* 8 chains x 8 updates = 64 LOP3 per round */
#pragma unroll
        for (int r = 0; r < 8; r += 3) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                x[k] = lop3<0x96>(x[k], y[k], z[k]);
                if (r + 1 < 8) y[k] = lop3<0xE8>(y[k], z[k], x[k]);
                if (r + 2 < 8) z[k] = lop3<0xCA>(z[k], x[k], y[k]);
            }
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc ^= x[k] ^ y[k] ^ z[k];
    sink[t] = acc;
}

}  // namespace bsfp

extern "C" bsfp_status bsfp_lop3_probe(uint32_t* sink, int32_t grid, int32_t block, int32_t iters, uint32_t seed,
                                       bsfp_stream_t s) {
    if (!sink) return BSFP_ERR_NULL;
    if (((uintptr_t)sink & 3u) != 0) return BSFP_ERR_ALIGN;
    if (grid < 1 || block < 32 || block > 1024 || (block & 31) || iters < 0) return BSFP_ERR_SIZE;
    bsfp::lop3_probe_kernel<<<grid, block, 0, (cudaStream_t)s>>>(sink, iters, seed);
    return cudaGetLastError() == cudaSuccess ? BSFP_OK : BSFP_ERR_CUDA;
}

extern "C" int32_t bsfp_num_sms(void) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}
