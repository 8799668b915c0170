/*
 * convert.cuh -- fused conversions between native floats and bitslice
 * operands of a format 1/E/M (not the paper's operations: the step before
 * and after them when the data are ordinary floats).
 *
 * A warp owns a tile of 32 word columns (1024 elements) and each lane one
 * column, as in pack/unpack (transpose.cu, bit_transpose.cuh).
 *
 * from_float: the tile's source values go to the warp's staging area in
 * shared memory (coalesced 16-byte loads); each lane reads its column's 32
 * values and transposes them in registers into 32 binary32 slices -- bfloat16
 * sources transpose as 16-bit rows into slices 16..31 (slices 0..15 are
 * zero), binary16 sources are widened exactly to binary32 value by value
 * first -- then runs the narrowing circuit from_f32 (circuit.cuh) on whole
 * words and stores the B output planes, a coalesced 128-byte row per warp.
 *
 * to_float: the reverse -- each lane loads the B planes of its column, runs
 * the exact widening circuit to_f32, transposes the 32 result slices into 32
 * binary32 values in registers, and the warp stores the tile from the
 * staging area with coalesced 16-byte stores.
 *
 * The staged column sits in the lane's registers rotated by rho elements
 * (bit_transpose.cuh); the element-wise circuits do not care, and each plane
 * word is rotated back (or into place) by one funnel rotate.  Elements past n
 * are read as +0 (they become zero padding); outputs past n are not written.
 */
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bit_transpose.cuh"
#include "circuit.cuh"

namespace bsfp {

constexpr int CV_WARPS = 4;    /* warps per block */

/* source element types of from_float (bsfp_float_type in bsfp.h) */
enum : int { SRC_F32 = 0, SRC_BF16 = 1, SRC_F16 = 2 };

/* The tile's 1024 source values (CB bytes each) into the staging area. */
template <int CB>
__device__ __forceinline__ void cv_stage_in(uint8_t* s, const void* in, int64_t e0, int64_t n, bool vec, int lane) {
    if (vec && e0 + 1024 <= n) {
        const uint4* src = reinterpret_cast<const uint4*>(static_cast<const uint8_t*>(in) + e0 * CB);
        uint4 v[2 * CB];
#pragma unroll
        for (int k = 0; k < 2 * CB; ++k) v[k] = __ldcs(src + lane + 32 * k);
#pragma unroll
        for (int k = 0; k < 2 * CB; ++k) reinterpret_cast<uint4*>(s)[lane + 32 * k] = v[k];
    } else if constexpr (CB == 4) {
        const uint32_t* src = static_cast<const uint32_t*>(in);
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            const int64_t i = e0 + lane + 32 * k;
            reinterpret_cast<uint32_t*>(s)[lane + 32 * k] = (i < n) ? __ldcs(src + i) : 0u;
        }
    } else {
        const unsigned short* src = static_cast<const unsigned short*>(in);
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            const int64_t i = e0 + lane + 32 * k;
            reinterpret_cast<unsigned short*>(s)[lane + 32 * k] = (i < n) ? __ldcs(src + i) : (unsigned short)0;
        }
    }
}

template <int E, int M, int R>
__global__ void __launch_bounds__(32 * CV_WARPS) from_float_kernel(const void* __restrict__ in, int src, int64_t n,
                                                                   uint32_t* __restrict__ out, int64_t S, bool vec) {
    constexpr int B = 1 + E + M;
    __shared__ __align__(16) uint8_t sm[CV_WARPS][4096];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t* s = sm[warp];
    const int64_t ntiles = S / 32;
    for (int64_t tile = (int64_t)blockIdx.x * CV_WARPS + warp; tile < ntiles;
         tile += (int64_t)gridDim.x * CV_WARPS) {
        const int64_t e0 = tile * 1024;
        uint32_t x[32];
        int rho;
        if (src == SRC_F32) {
            cv_stage_in<4>(s, in, e0, n, vec, lane);
            __syncwarp();
            stage_read_column<4>(s, lane, x);
            transpose32(x);
            rho = stage_rho<4>(lane);
        } else {
            cv_stage_in<2>(s, in, e0, n, vec, lane);
            __syncwarp();
            uint32_t w[16];
            stage_read_column<2>(s, lane, w);
            if (src == SRC_BF16) {
                /* a bfloat16 is the top half of its binary32: slices 16..31
                 * are the transposed 16-bit rows, slices 0..15 zero */
                gather16(w, x + 16);
                transpose16x2(x + 16);
#pragma unroll
                for (int b = 0; b < 16; ++b) x[b] = 0u;
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const unsigned short h = (unsigned short)((j & 1) ? (w[j >> 1] >> 16) : (w[j >> 1] & 0xFFFFu));
                    x[j] = __float_as_uint(__half2float(__ushort_as_half(h)));
                }
                transpose32(x);
            }
            rho = stage_rho<2>(lane);
        }
        __syncwarp();   /* the next tile may overwrite the staging area */
        uint32_t r[B];
        from_f32<E, M, mode_rz(R), mode_ftz(R)>(x, r);
        uint32_t* o = out + tile * 32 + lane;
#pragma unroll
        for (int b = 0; b < B; ++b) __stcs(o + b * S, rotl32(r[b], rho));
    }
}

template <int E, int M, int R>
__global__ void __launch_bounds__(32 * CV_WARPS) to_float_kernel(const uint32_t* __restrict__ in, int64_t S, int64_t n,
                                                                 uint32_t* __restrict__ out, bool vec) {
    constexpr int B = 1 + E + M;
    __shared__ __align__(16) uint8_t sm[CV_WARPS][4096];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t* s = sm[warp];
    const int rho = stage_rho<4>(lane);
    const int64_t ntiles = (n + 1023) / 1024;
    for (int64_t tile = (int64_t)blockIdx.x * CV_WARPS + warp; tile < ntiles;
         tile += (int64_t)gridDim.x * CV_WARPS) {
        uint32_t x[B], r[32];
        const uint32_t* src = in + tile * 32 + lane;
#pragma unroll
        for (int b = 0; b < B; ++b) x[b] = rotr32(__ldcs(src + b * S), rho);
        to_f32<E, M, mode_ftz(R)>(x, r);
        transpose32(r);
        stage_write_column<4>(s, lane, r);
        __syncwarp();
        const int64_t e0 = tile * 1024;
        if (vec && e0 + 1024 <= n) {
            uint4* dst = reinterpret_cast<uint4*>(out + e0);
#pragma unroll
            for (int k = 0; k < 8; ++k) __stcs(dst + lane + 32 * k, reinterpret_cast<const uint4*>(s)[lane + 32 * k]);
        } else {
#pragma unroll 8
            for (int k = 0; k < 32; ++k) {
                const int64_t i = e0 + lane + 32 * k;
                if (i < n) out[i] = reinterpret_cast<const uint32_t*>(s)[lane + 32 * k];
            }
        }
        __syncwarp();   /* the next tile may overwrite the staging area */
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
    from_float_kernel<E, M, R><<<grid, 32 * CV_WARPS, 0, s>>>(in, src, n, out, S, ((uintptr_t)in & 15u) == 0);
    return cudaGetLastError();
}

template <int E, int M, int R>
cudaError_t launch_to_float(const uint32_t* in, int64_t S, int64_t n, uint32_t* out, int grid, cudaStream_t s) {
    to_float_kernel<E, M, R><<<grid, 32 * CV_WARPS, 0, s>>>(in, S, n, out, ((uintptr_t)out & 15u) == 0);
    return cudaGetLastError();
}

/* filled by the per-exponent translation units (conv_inst.cu) */
extern ConvEntry g_conv_table[9][24][4];

}  // namespace bsfp
