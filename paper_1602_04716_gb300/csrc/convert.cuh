/*
 * convert.cuh -- fused conversions between native floats and bitslice
 * operands of a format 1/E/M (not the paper's operations: the step before
 * and after them when the data are ordinary floats).
 *
 * from_float: a warp owns 1024 elements (32 word columns).  For each of the
 * 32 element groups it loads 32 consecutive floats (binary32, or bfloat16 /
 * binary16 widened exactly to binary32 bit patterns), transposes the 32x32
 * bit matrix across the warp and stores the 32 slices of the group into
 * padded shared memory; then lane c holds the 32 binary32 slices of column
 * c, runs the narrowing circuit from_f32 (circuit.cuh) on whole words and
 * stores the B output planes, each a coalesced 128-byte row per warp.
 *
 * to_float: the reverse -- each lane loads the B planes of its column, runs
 * the exact widening circuit to_f32, the 32 result slices go through shared
 * memory and the warp transpose back to 32 binary32 values per group,
 * stored as coalesced rows.
 *
 * Elements past n are read as +0 (they become zero padding); outputs past n
 * are not written.
 */
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "circuit.cuh"
#include "warp_transpose.cuh"

namespace bsfp {

constexpr int CV_WARPS = 4;    /* warps per block */
constexpr int CV_ROW = 33;     /* padded shared-memory row (words) */

/* source element types of from_float (bsfp_float_type in bsfp.h) */
enum : int { SRC_F32 = 0, SRC_BF16 = 1, SRC_F16 = 2 };

__device__ __forceinline__ uint32_t load_as_f32_bits(const void* in, int src, int64_t i) {
    if (src == SRC_F32) return __ldcs(static_cast<const uint32_t*>(in) + i);
    if (src == SRC_BF16) return (uint32_t)__ldcs(static_cast<const unsigned short*>(in) + i) << 16;
    const unsigned short h = __ldcs(static_cast<const unsigned short*>(in) + i);
    return __float_as_uint(__half2float(__ushort_as_half(h)));
}

template <int E, int M, int R>
__global__ void __launch_bounds__(32 * CV_WARPS) from_float_kernel(const void* __restrict__ in, int src, int64_t n,
                                                                   uint32_t* __restrict__ out, int64_t S) {
    constexpr int B = 1 + E + M;
    __shared__ uint32_t sm[CV_WARPS][32 * CV_ROW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* s = sm[warp];
    const int64_t ntiles = S / 32;
    for (int64_t tile = (int64_t)blockIdx.x * CV_WARPS + warp; tile < ntiles;
         tile += (int64_t)gridDim.x * CV_WARPS) {
        const int64_t e0 = tile * 1024;
        /* all 32 loads of the tile first, so that they are in flight together */
        uint32_t v[32];
#pragma unroll
        for (int t = 0; t < 32; ++t) {
            const int64_t i = e0 + (int64_t)t * 32 + lane;
            v[t] = (i < n) ? load_as_f32_bits(in, src, i) : 0u;
        }
#pragma unroll
        for (int t = 0; t < 32; ++t) s[lane * CV_ROW + t] = warp_transpose32(v[t], lane);   /* lane b: slice b */
        __syncwarp();
        uint32_t x[32], r[B];
#pragma unroll
        for (int b = 0; b < 32; ++b) x[b] = s[b * CV_ROW + lane];
        from_f32<E, M, mode_rz(R), mode_ftz(R)>(x, r);
#pragma unroll
        for (int b = 0; b < B; ++b) __stcs(out + b * S + tile * 32 + lane, r[b]);
        __syncwarp();
    }
}

template <int E, int M, int R>
__global__ void __launch_bounds__(32 * CV_WARPS) to_float_kernel(const uint32_t* __restrict__ in, int64_t S, int64_t n,
                                                                 uint32_t* __restrict__ out) {
    constexpr int B = 1 + E + M;
    __shared__ uint32_t sm[CV_WARPS][32 * CV_ROW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* s = sm[warp];
    const int64_t ntiles = (n + 1023) / 1024;
    for (int64_t tile = (int64_t)blockIdx.x * CV_WARPS + warp; tile < ntiles;
         tile += (int64_t)gridDim.x * CV_WARPS) {
        uint32_t x[B], r[32];
#pragma unroll
        for (int b = 0; b < B; ++b) x[b] = __ldcs(in + b * S + tile * 32 + lane);
        to_f32<E, M, mode_ftz(R)>(x, r);
#pragma unroll
        for (int b = 0; b < 32; ++b) s[b * CV_ROW + lane] = r[b];
        __syncwarp();
        const int64_t e0 = tile * 1024;
#pragma unroll 4
        for (int t = 0; t < 32; ++t) {
            /* lane b takes slice b of group t; after the transpose lane j
             * holds element j of the group */
            const uint32_t v = warp_transpose32(s[lane * CV_ROW + t], lane);
            const int64_t i = e0 + (int64_t)t * 32 + lane;
            if (i < n) __stcs(out + i, v);
        }
        __syncwarp();
    }
}

typedef cudaError_t (*from_float_fn)(const void* in, int src, int64_t n, uint32_t* out, int64_t S, int grid,
                                     cudaStream_t s);
typedef cudaError_t (*to_float_fn)(const uint32_t* in, int64_t S, int64_t n, uint32_t* out, int grid, cudaStream_t s);

struct ConvEntry {
    from_float_fn from;
    to_float_fn to;
};

template <int E, int M, int R>
cudaError_t launch_from_float(const void* in, int src, int64_t n, uint32_t* out, int64_t S, int grid, cudaStream_t s) {
    from_float_kernel<E, M, R><<<grid, 32 * CV_WARPS, 0, s>>>(in, src, n, out, S);
    return cudaGetLastError();
}

template <int E, int M, int R>
cudaError_t launch_to_float(const uint32_t* in, int64_t S, int64_t n, uint32_t* out, int grid, cudaStream_t s) {
    to_float_kernel<E, M, R><<<grid, 32 * CV_WARPS, 0, s>>>(in, S, n, out);
    return cudaGetLastError();
}

/* filled by the per-exponent translation units (conv_inst.cu) */
extern ConvEntry g_conv_table[9][24][4];

}  // namespace bsfp
