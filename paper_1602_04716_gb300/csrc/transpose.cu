/*
 * transpose.cu -- pack and unpack between the standard representation and
 * the bitslice layout (the "helper operations for transforming data in the
 * standard format" of Sec. 4; layout of Sec. 2, Fig. 1).
 *
 * Standard representation: element i is the B-bit encoding right-aligned in a
 * container of CB = 1, 2 or 4 bytes (B <= 8, <= 16, <= 32), array index i.
 * Bitslice: bit b of element i is bit (i mod 32) of word b*S + i/32.
 *
 * A warp owns a tile of 32 word columns (1024 elements) and each lane one
 * column.  Both directions go through the warp's 1024*CB-byte staging area in
 * shared memory and the in-register transposes of bit_transpose.cuh:
 *
 *  pack:   coalesced 16-byte loads of the tile -> shared memory -> each lane
 *          reads its column (32 elements), transposes it in registers and
 *          stores its B plane words; the warp's stores are 128-byte rows.
 *          The next tile's loads are issued before the current one is
 *          staged.
 *  unpack: each lane loads its column's B plane words (128-byte rows per
 *          warp), transposes them into 32 elements, writes them to shared
 *          memory -> coalesced 16-byte stores of the tile.  The next tile's
 *          plane words are loaded before the current one is transposed.
 *
 * There is no cross-lane shuffle: a column's transpose is 64 (CB = 1), 128
 * (CB = 2) or 256 (CB = 4) logic instructions of one thread.  Tiles whose
 * standard array is not 16-byte aligned, and the last, partly filled tile,
 * move their elements one container at a time instead (coalesced, bounded by
 * n).  Elements past n are packed as zero and every padding word of the
 * planes is written, so a packed operand always has zero padding.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "bit_transpose.cuh"

namespace bsfp {

constexpr int TP_WARPS = 8;   /* warps per block */

template <int CB> struct Container;
template <> struct Container<1> { using T = uint8_t; };
template <> struct Container<2> { using T = uint16_t; };
template <> struct Container<4> { using T = uint32_t; };

/* The tile's 1024 containers from the standard array into the staging area:
 * whole 16-byte chunks when the tile is full and the array 16-byte aligned,
 * else container by container with zeros past n. */
template <int CB>
__device__ __forceinline__ void stage_load_tile(uint8_t* s, const void* in, int64_t e0, int64_t n, bool vec, int lane) {
    using T = typename Container<CB>::T;
    if (vec && e0 + 1024 <= n) {
        const uint4* src = reinterpret_cast<const uint4*>(static_cast<const uint8_t*>(in) + e0 * CB);
        uint4 v[2 * CB];
#pragma unroll
        for (int k = 0; k < 2 * CB; ++k) v[k] = __ldcs(src + lane + 32 * k);
#pragma unroll
        for (int k = 0; k < 2 * CB; ++k) reinterpret_cast<uint4*>(s)[lane + 32 * k] = v[k];
    } else {
        const T* src = static_cast<const T*>(in);
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            const int64_t i = e0 + lane + 32 * k;
            reinterpret_cast<T*>(s)[lane + 32 * k] = (i < n) ? __ldcs(src + i) : (T)0;
        }
    }
}

/* The staged tile out to the standard array, the first min(1024, n - e0)
 * containers only. */
template <int CB>
__device__ __forceinline__ void stage_store_tile(const uint8_t* s, void* out, int64_t e0, int64_t n, bool vec,
                                                 int lane) {
    using T = typename Container<CB>::T;
    if (vec && e0 + 1024 <= n) {
        uint4* dst = reinterpret_cast<uint4*>(static_cast<uint8_t*>(out) + e0 * CB);
#pragma unroll
        for (int k = 0; k < 2 * CB; ++k) __stcs(dst + lane + 32 * k, reinterpret_cast<const uint4*>(s)[lane + 32 * k]);
    } else {
        T* dst = static_cast<T*>(out);
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            const int64_t i = e0 + lane + 32 * k;
            if (i < n) dst[i] = reinterpret_cast<const T*>(s)[lane + 32 * k];
        }
    }
}

/* The container width of B-bit elements. */
__host__ __device__ constexpr int container_of(int B) { return B <= 8 ? 1 : (B <= 16 ? 2 : 4); }

/* A full, 16-byte aligned tile's 2*CB chunks of the lane. */
template <int CB>
__device__ __forceinline__ void load_chunks(const void* in, int64_t e0, int lane, uint4* v) {
    const uint4* src = reinterpret_cast<const uint4*>(static_cast<const uint8_t*>(in) + e0 * CB);
#pragma unroll
    for (int k = 0; k < 2 * CB; ++k) v[k] = __ldcs(src + lane + 32 * k);
}

/* Whether a transpose kernel loads the next tile ahead: for 2- and 1-byte
 * containers.  Measured at 2^28 elements on 2-byte ones: 1-3% faster for
 * 1/4/4 and 1/5/7, pack and unpack.  For 4-byte containers (twice the
 * registers) it lost as often as it won (1/8/15, 1/8/23: +-2-3%), so they
 * keep one tile in flight per warp. */
__host__ __device__ constexpr bool tp_prefetch(int CB) { return CB <= 2; }

/* Full, aligned tiles: each warp loads the next tile's chunks before it
 * transposes and stores the current one, so that two tiles' loads are in
 * flight per warp (tp_prefetch).  Other tiles (the ragged last one, the
 * padding, an unaligned array) are staged element by element when their
 * turn comes. */
template <int B>
__global__ void __launch_bounds__(32 * TP_WARPS) pack_kernel(const void* __restrict__ in, int64_t n,
                                                             uint32_t* __restrict__ out, int64_t S, bool vec) {
    constexpr int CB = container_of(B);
    constexpr bool PF = tp_prefetch(CB);
    __shared__ __align__(16) uint8_t sm[TP_WARPS][1024 * CB];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t* s = sm[warp];
    const int rho = stage_rho<CB>(lane);
    const int64_t ntiles = S / 32;
    const int64_t stride = (int64_t)gridDim.x * TP_WARPS;
    int64_t tile = (int64_t)blockIdx.x * TP_WARPS + warp;
    bool cur_full = PF && vec && tile < ntiles && tile * 1024 + 1024 <= n;
    uint4 cur[2 * CB];
    if (cur_full) load_chunks<CB>(in, tile * 1024, lane, cur);
    for (; tile < ntiles; tile += stride) {
        if constexpr (!PF) {
            cur_full = vec && tile * 1024 + 1024 <= n;
            if (cur_full) load_chunks<CB>(in, tile * 1024, lane, cur);
        }
        const int64_t nt = tile + stride;
        const bool nxt_full = PF && vec && nt < ntiles && nt * 1024 + 1024 <= n;
        uint4 nxt[2 * CB];
        if (nxt_full) load_chunks<CB>(in, nt * 1024, lane, nxt);
        if (cur_full) {
#pragma unroll
            for (int k = 0; k < 2 * CB; ++k) reinterpret_cast<uint4*>(s)[lane + 32 * k] = cur[k];
        } else {
            stage_load_tile<CB>(s, in, tile * 1024, n, false, lane);
        }
        __syncwarp();
        uint32_t w[8 * CB], x[8 * CB];
        stage_read_column<CB>(s, lane, w);
        __syncwarp();   /* the next tile may overwrite the staging area */
        rows_to_planes<CB>(w, x);
        uint32_t* o = out + tile * 32 + lane;
#pragma unroll
        for (int b = 0; b < B; ++b) __stcs(o + b * S, rotl32(x[b], rho));
        if constexpr (PF) {
            if (nxt_full) {
#pragma unroll
                for (int k = 0; k < 2 * CB; ++k) cur[k] = nxt[k];
            }
            cur_full = nxt_full;
        }
    }
}

/* The lane's B plane words of a tile's column. */
template <int B>
__device__ __forceinline__ void load_planes(const uint32_t* __restrict__ in, int64_t S, int64_t tile, int lane,
                                            uint32_t* v) {
    const uint32_t* src = in + tile * 32 + lane;
#pragma unroll
    for (int b = 0; b < B; ++b) v[b] = __ldcs(src + b * S);
}

/* Each warp loads the next tile's plane words before it transposes and
 * stores the current one, so that two tiles' loads are in flight per warp
 * (tp_prefetch). */
template <int B>
__global__ void __launch_bounds__(32 * TP_WARPS) unpack_kernel(const uint32_t* __restrict__ in, int64_t S,
                                                               void* __restrict__ out, int64_t n, bool vec) {
    constexpr int CB = container_of(B);
    constexpr bool PF = tp_prefetch(CB);
    __shared__ __align__(16) uint8_t sm[TP_WARPS][1024 * CB];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t* s = sm[warp];
    const int rho = stage_rho<CB>(lane);
    const int64_t ntiles = (n + 1023) / 1024;
    const int64_t stride = (int64_t)gridDim.x * TP_WARPS;
    int64_t tile = (int64_t)blockIdx.x * TP_WARPS + warp;
    uint32_t cur[B];
    if (PF && tile < ntiles) load_planes<B>(in, S, tile, lane, cur);
    for (; tile < ntiles; tile += stride) {
        if constexpr (!PF) load_planes<B>(in, S, tile, lane, cur);
        const bool more = PF && tile + stride < ntiles;
        uint32_t nxt[B];
        if (more) load_planes<B>(in, S, tile + stride, lane, nxt);
        uint32_t x[8 * CB], w[8 * CB];
#pragma unroll
        for (int b = 0; b < 8 * CB; ++b) x[b] = (b < B) ? rotr32(cur[(b < B) ? b : 0], rho) : 0u;
        planes_to_rows<CB>(x, w);
        stage_write_column<CB>(s, lane, w);
        __syncwarp();
        stage_store_tile<CB>(s, out, tile * 1024, n, vec, lane);
        __syncwarp();   /* the next tile may overwrite the staging area */
        if (more) {
#pragma unroll
            for (int b = 0; b < B; ++b) cur[b] = nxt[b];
        }
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

/* Grid: enough blocks to cover the tiles, at most the resident blocks of
 * every SM (occupancy of the kernel, looked up once). */
static int tp_grid(const void* kernel, int* occ_cache, int64_t ntiles) {
    if (*occ_cache <= 0) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 32 * TP_WARPS, 0) != cudaSuccess || occ <= 0) {
            cudaGetLastError();
            occ = 4;
        }
        *occ_cache = occ;
    }
    const int64_t want = (ntiles + TP_WARPS - 1) / TP_WARPS;
    const int64_t cap = (int64_t)num_sms() * *occ_cache;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

/* One pack and one unpack kernel per plane count B (1..32), the container
 * width following from B. */
struct TransposeEntry {
    const void* pack;
    const void* unpack;
    int occ_pack, occ_unpack;   /* resident blocks per SM, looked up once */
};
static TransposeEntry g_tp[33];

template <int B>
static void fill_tp() {
    g_tp[B] = TransposeEntry{(const void*)pack_kernel<B>, (const void*)unpack_kernel<B>, 0, 0};
    if constexpr (B < 32) fill_tp<B + 1>();
}

static const TransposeEntry* tp_entry(int cb, int B) {
    static bool filled = false;
    if (!filled) {
        fill_tp<1>();
        filled = true;
    }
    if (B < 1 || B > 32 || container_of(B) != cb) return nullptr;
    return &g_tp[B];
}

cudaError_t launch_pack(int cb, const void* in, int64_t n, int B, uint32_t* out, int64_t S, cudaStream_t st) {
    TransposeEntry* e = const_cast<TransposeEntry*>(tp_entry(cb, B));
    if (!e) return cudaErrorInvalidValue;
    bool vec = aligned16(in);
    void* args[] = {(void*)&in, (void*)&n, (void*)&out, (void*)&S, (void*)&vec};
    return cudaLaunchKernel(e->pack, dim3(tp_grid(e->pack, &e->occ_pack, S / 32)), dim3(32 * TP_WARPS), args, 0, st);
}

cudaError_t launch_unpack(int cb, const uint32_t* in, int64_t S, int B, void* out, int64_t n, cudaStream_t st) {
    TransposeEntry* e = const_cast<TransposeEntry*>(tp_entry(cb, B));
    if (!e) return cudaErrorInvalidValue;
    bool vec = aligned16(out);
    void* args[] = {(void*)&in, (void*)&S, (void*)&out, (void*)&n, (void*)&vec};
    return cudaLaunchKernel(e->unpack, dim3(tp_grid(e->unpack, &e->occ_unpack, (n + 1023) / 1024)),
                            dim3(32 * TP_WARPS), args, 0, st);
}

int device_num_sms() { return num_sms(); }

}  // namespace bsfp
