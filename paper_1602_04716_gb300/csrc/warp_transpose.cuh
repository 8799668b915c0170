/*
 * warp_transpose.cuh -- the 32x32 bit-matrix transpose of one warp, shared by
 * pack/unpack (transpose.cu) and the fused conversions (convert.cuh).
 */
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bsfp {

/* Transpose the 32x32 bit matrix held one row per lane: afterwards lane c
 * holds, in bit l, bit c of lane l's input row. */
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
    /* stages 16 and 8 move whole bytes: one byte permute each picks the kept
     * bytes of x and the partner's bytes, in place of rotate + merge.
     * Lower rows (lane bit clear) keep their low half / even bytes and take
     * the partner's low half / even bytes one position up; upper rows the
     * reverse.  Byte selectors index {x: 0-3, y: 4-7}. */
    {
        const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, 16);
        x = __byte_perm(x, y, (lane & 16) ? 0x3276u : 0x5410u);
    }
    {
        const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, 8);
        x = __byte_perm(x, y, (lane & 8) ? 0x3715u : 0x6240u);
    }
#pragma unroll
    for (int k = 4; k >= 1; k >>= 1) {
        const uint32_t lowmask = (k == 4) ? 0x0F0F0F0Fu : (k == 2) ? 0x33333333u : 0x55555555u;
        const bool upper = (lane & k) != 0;
        const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, k);
        /* rows without bit k take the partner's low columns moved up by k;
         * rows with bit k take the partner's high columns moved down by k */
        const uint32_t r = __funnelshift_l(y, y, upper ? 32 - k : k);
        const uint32_t keep = upper ? ~lowmask : lowmask;
        x = (x & keep) | (r & ~keep);
    }
    return x;
}

}  // namespace bsfp
