/*
 * transpose.cu -- pack and unpack between the standard representation and
 * the bitslice layout (the "helper operations for transforming data in the
 * standard format" of Sec. 4; layout of Sec. 2, Fig. 1).
 *
 * Standard representation: element i is the B-bit encoding right-aligned in a
 * container of CB = 1, 2 or 4 bytes (B <= 8, <= 16, <= 32), array index i.
 * Bitslice: bit b of element i is bit (i mod 32) of word b*S + i/32.
 *
 * Both directions are the same 32x32 bit-matrix transpose, done by a warp
 * with one row per lane in five butterfly stages (shfl.xor + funnel rotate +
 * one 3-input merge per stage).  A warp owns a tile of 32 word columns
 * (1024 elements).  For containers narrower than 32 bits one transpose
 * serves 32/(8*CB) element groups at once: lane j's row holds element j of
 * 4/CB consecutive 32-element groups, one per CB-byte lane of the row, and
 * the transposed rows are the planes of those groups side by side.
 *
 *  pack:   coalesced container loads -> transpose -> shared memory
 *          [plane][column] -> coalesced 128-byte plane-row stores.
 *  unpack: coalesced 128-byte plane-row loads -> shared memory -> transpose
 *          -> coalesced container stores.
 *
 * Elements past n are packed as zero and every padding word of the planes is
 * written, so a packed operand always has zero padding.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "warp_transpose.cuh"

namespace bsfp {

constexpr int TP_WARPS = 8;              /* warps per block */
constexpr int TP_ROW = 33;               /* padded shared-memory row (words) */

template <int CB> struct Container;
template <> struct Container<1> { using T = uint8_t; };
template <> struct Container<2> { using T = uint16_t; };
template <> struct Container<4> { using T = uint32_t; };

template <int CB>
__global__ void __launch_bounds__(32 * TP_WARPS) pack_kernel(const void* __restrict__ in_, int64_t n, int B,
                                                             uint32_t* __restrict__ out, int64_t S) {
    using T = typename Container<CB>::T;
    constexpr int GP = 4 / CB;           /* element groups per transpose */
    constexpr int BITS = 8 * CB;
    __shared__ uint32_t sm[TP_WARPS][32 * TP_ROW];
    const T* in = static_cast<const T*>(in_);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* s = sm[warp];
    const int64_t ntiles = S / 32;
    for (int64_t tile = (int64_t)blockIdx.x * TP_WARPS + warp; tile < ntiles; tile += (int64_t)gridDim.x * TP_WARPS) {
        const int64_t e0 = tile * 1024;
        /* all loads of the tile first, so that they are in flight together */
        uint32_t rows[32 / GP];
#pragma unroll
        for (int t = 0; t < 32 / GP; ++t) {
            uint32_t row = 0;
#pragma unroll
            for (int q = 0; q < GP; ++q) {
                const int64_t i = e0 + (int64_t)(t * GP + q) * 32 + lane;
                const uint32_t v = (i < n) ? (uint32_t)__ldcs(in + i) : 0u;
                row |= v << (BITS * q);
            }
            rows[t] = row;
        }
#pragma unroll
        for (int t = 0; t < 32 / GP; ++t) {
            const uint32_t col = warp_transpose32(rows[t], lane);
            /* lane = BITS*q + b now holds plane b of group t*GP+q */
            const int b = lane % BITS, g = t * GP + lane / BITS;
            if (b < B) s[b * TP_ROW + g] = col;
        }
        __syncwarp();
        for (int b = 0; b < B; ++b) out[b * S + tile * 32 + lane] = s[b * TP_ROW + lane];
        __syncwarp();
    }
}

template <int CB>
__global__ void __launch_bounds__(32 * TP_WARPS) unpack_kernel(const uint32_t* __restrict__ in, int64_t S, int B,
                                                               void* __restrict__ out_, int64_t n) {
    using T = typename Container<CB>::T;
    constexpr int GP = 4 / CB;
    constexpr int BITS = 8 * CB;
    constexpr uint32_t VMASK = (CB == 4) ? 0xFFFFFFFFu : ((1u << BITS) - 1u);
    __shared__ uint32_t sm[TP_WARPS][32 * TP_ROW];
    T* out = static_cast<T*>(out_);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* s = sm[warp];
    const int64_t ntiles = (n + 1023) / 1024;
    for (int64_t tile = (int64_t)blockIdx.x * TP_WARPS + warp; tile < ntiles; tile += (int64_t)gridDim.x * TP_WARPS) {
        for (int b = 0; b < B; ++b) s[b * TP_ROW + lane] = __ldcs(in + b * S + tile * 32 + lane);
        __syncwarp();
        const int64_t e0 = tile * 1024;
#pragma unroll 4
        for (int t = 0; t < 32 / GP; ++t) {
            const int b = lane % BITS, g = t * GP + lane / BITS;
            const uint32_t row = (b < B) ? s[b * TP_ROW + g] : 0u;
            const uint32_t x = warp_transpose32(row, lane);
            /* lane j: bits BITS*q .. hold element j of group t*GP+q */
#pragma unroll
            for (int q = 0; q < GP; ++q) {
                const int64_t i = e0 + (int64_t)(t * GP + q) * 32 + lane;
                if (i < n) out[i] = (T)((x >> (BITS * q)) & VMASK);
            }
        }
        __syncwarp();
    }
}

static int g_num_sms = 0;

static int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

/* Grid: enough blocks to cover the tiles, at most 8 resident blocks per SM. */
static int tp_grid(int64_t ntiles) {
    const int64_t want = (ntiles + TP_WARPS - 1) / TP_WARPS;
    const int64_t cap = (int64_t)num_sms() * 8;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

cudaError_t launch_pack(int cb, const void* in, int64_t n, int B, uint32_t* out, int64_t S, cudaStream_t st) {
    const int grid = tp_grid(S / 32);
    switch (cb) {
        case 1: pack_kernel<1><<<grid, 32 * TP_WARPS, 0, st>>>(in, n, B, out, S); break;
        case 2: pack_kernel<2><<<grid, 32 * TP_WARPS, 0, st>>>(in, n, B, out, S); break;
        case 4: pack_kernel<4><<<grid, 32 * TP_WARPS, 0, st>>>(in, n, B, out, S); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_unpack(int cb, const uint32_t* in, int64_t S, int B, void* out, int64_t n, cudaStream_t st) {
    const int grid = tp_grid((n + 1023) / 1024);
    switch (cb) {
        case 1: unpack_kernel<1><<<grid, 32 * TP_WARPS, 0, st>>>(in, S, B, out, n); break;
        case 2: unpack_kernel<2><<<grid, 32 * TP_WARPS, 0, st>>>(in, S, B, out, n); break;
        case 4: unpack_kernel<4><<<grid, 32 * TP_WARPS, 0, st>>>(in, S, B, out, n); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int device_num_sms() { return num_sms(); }

}  // namespace bsfp
