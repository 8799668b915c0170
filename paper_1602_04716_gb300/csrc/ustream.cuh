/*
 * ustream.cuh -- the unified streamed batch kernel: one launch per op class
 * (add/sub, mul) streams the tiles of every job of the batched formats
 * (1/4/3, 1/4/4, 1/5/7, 1/5/10, 1/8/7; RN and RZ) through one shared-memory
 * ring, whatever their format.
 *
 * The per-format streamed kernels (stream.cuh) need one launch per (format,
 * rounding, op class), and each launch ramps up and drains on its own.  Here
 * one persistent block per SM serves all ten kinds:
 *
 *   producer (lane 0 of the last warp): claims tiles of the op class from
 *     an atomic counter, UCHUNK at a time and a chunk ahead, and prefetches
 *     the next tile's job descriptor (only at job boundaries: tiles are
 *     numbered job by job), waits until ring slot k % NST is free, writes the
 *     tile's metadata (kind, output, stride, first column, tail mask, sign
 *     flip) into the slot's header and issues one cp.async.bulk per input
 *     plane, completing on the slot's `full` mbarrier.  When the tiles run
 *     out it posts one empty tile (kind -1): every consumer warp takes every
 *     slot in the same order, so all of them stop there;
 *   NC consumer warps: wait on `full`, read the metadata, copy their columns
 *     of every plane into registers, release the slot (one arrive per warp
 *     on `empty`), then run the kind's circuit -- a switch over the ten
 *     kinds, each the printed netlist of binop.cuh -- and store each output
 *     column (a coalesced 128-byte row per warp and plane).
 *
 * A slot holds SLOT_WORDS words.  A tile of kind k spans TW_k = WPT_k * 32 *
 * NC word columns of its job, WPT_k = the columns per consumer thread that
 * fit 2 * B_k planes into the slot (at least 1, at most 2), so narrow
 * formats move more columns per tile.  Thread t of the consumers owns the
 * columns t + i * 32 * NC of the tile (i < WPT_k): shared-memory reads and
 * global stores are consecutive across the warp.
 *
 * Dynamic tiles balance the light and heavy kinds across SMs: a block that
 * draws cheap tiles simply draws more of them.  Waits are bounded as in
 * stream.cuh; a block whose wait gives up stops, lets its copies in flight
 * land and sets the fault word.
 */
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "batch.cuh"
#include "binop.cuh"
#include "tma.cuh"

namespace bsfp {

/* Metadata of the tile in one ring slot (written by the producer before the
 * arrive that releases the slot's phase). */
struct UTileMeta {
    uint32_t* out;
    int64_t S;
    int64_t nwords;
    int64_t w0;          /* first word column of the tile */
    uint32_t tailmask;
    uint32_t negb;
    int32_t kind;        /* -1: no more tiles */
    int32_t cols;        /* word columns of the tile (<= TW of the kind) */
};

/* Tiles a producer claims from the counter at once. */
constexpr int UCHUNK = 4;

template <int NC, int SLOT_WORDS>
struct UShape {
    static constexpr int THREADS = 32 * (NC + 1);
    static constexpr int HDR = 512;   /* barriers, then one metadata record per slot */
    static constexpr int META_OFF = 128;
    static constexpr int B_MAX = 16;  /* planes of the widest batched format */
    static_assert(2 * B_MAX * 32 * NC <= SLOT_WORDS, "a slot holds one column per consumer of the widest format");
    /* columns per consumer thread for a kind of B planes */
    __host__ __device__ static constexpr int wpt(int B) { return (SLOT_WORDS / (2 * B * 32 * NC)) >= 2 ? 2 : 1; }
    __host__ __device__ static constexpr int tw(int B) { return wpt(B) * 32 * NC; }
};

/* Planes of each kind (kind = 2 * format index + rounding), on the device. */
template <int F>
struct UFmtBits {
    static constexpr int value = 1 + BATCH_E[F] + BATCH_M[F];
};
__device__ __forceinline__ int ukind_bits(int kind) {
    switch (kind >> 1) {
        case 0: return UFmtBits<0>::value;
        case 1: return UFmtBits<1>::value;
        case 2: return UFmtBits<2>::value;
        case 3: return UFmtBits<3>::value;
        default: return UFmtBits<4>::value;
    }
}

/* One consumer's share of a tile of kind K: read its columns of the 2B
 * planes, release the slot, compute, store. */
template <int OPC, int NC, int SLOT_WORDS, int K>
__device__ __forceinline__ void ustream_consume(const uint32_t* slot, const UTileMeta& m, uint32_t empty_bar, int warp,
                                                int lane) {
    constexpr int F = K / 2;
    constexpr int E = BATCH_E[F], M = BATCH_M[F], B = 1 + E + M;
    constexpr int R = K & 1;
    using SH = UShape<NC, SLOT_WORDS>;
    constexpr int WPT = SH::wpt(B), TW = SH::tw(B);
    const int t = warp * 32 + lane;
    uint32_t xa[WPT][B], xb[WPT][B];
#pragma unroll
    for (int i = 0; i < WPT; ++i) {
        const int j = t + i * 32 * NC;
#pragma unroll
        for (int q = 0; q < B; ++q) {
            xa[i][q] = slot[q * TW + j];
            xb[i][q] = slot[(B + q) * TW + j];
        }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(empty_bar);
#pragma unroll
    for (int i = 0; i < WPT; ++i) {
        const int j = t + i * 32 * NC;
        if (j >= m.cols) continue;
        const int64_t w = m.w0 + j;
        uint32_t z[B], r[B];
#pragma unroll
        for (int q = 0; q < B; ++q) z[q] = 0u;
        column_op<E, M, R, OPC>(xa[i], xb[i], z, r, m.negb);
        const uint32_t mask = (w + 1 < m.nwords) ? ~0u : (w + 1 == m.nwords ? m.tailmask : 0u);
#pragma unroll
        for (int q = 0; q < B; ++q) __stcs(m.out + q * m.S + w, r[q] & mask);
    }
}

template <int OPC, int NC, int NST, int SLOT_WORDS>
__global__ void __launch_bounds__(UShape<NC, SLOT_WORDS>::THREADS) ustream_kernel(
    const JobDesc* __restrict__ jobs, const int32_t* __restrict__ tile_job, int64_t ntiles,
    unsigned long long* counter, int* fault) {
    using SH = UShape<NC, SLOT_WORDS>;
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + NST;
    UTileMeta* meta = reinterpret_cast<UTileMeta*>(smem + SH::META_OFF);
    uint32_t* ring = reinterpret_cast<uint32_t*>(smem + SH::HDR);
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < NST; ++s) {
            mbar_init(smem_addr(&full[s]), 1);
            mbar_init(smem_addr(&empty[s]), NC);
        }
        mbar_init_fence();
    }
    __syncthreads();
    volatile int* ab = &abort_flag;

    if (warp == NC) {
        if (lane == 0) {
            int64_t k = 0;   /* slots filled by this block */
            /* tiles are claimed UCHUNK at a time, the next chunk while the
             * current one is issued; a tile of the same job as the one
             * before needs no descriptor load (tiles are numbered job by
             * job), so the producer's chain of dependent loads is paid only
             * at job boundaries */
            int64_t c0 = (int64_t)atomicAdd(counter, (unsigned long long)UCHUNK);
            int64_t c1 = (int64_t)atomicAdd(counter, (unsigned long long)UCHUNK);
            int i = 0;
            int64_t t = c0;
            JobDesc J;
            if (t < ntiles) J = jobs[tile_job[t]];
            while (true) {
                const int s = (int)(k % NST);
                const uint32_t bar = smem_addr(&full[s]);
                UTileMeta& m = meta[s];
                if (t >= ntiles) {
                    /* no more tiles: one empty tile stops every consumer
                     * (they all take every slot in the same order) */
                    if (k >= NST && !mbar_wait(smem_addr(&empty[s]), (uint32_t)((k / NST - 1) & 1), ab,
                                               STREAM_WAIT_CYCLES))
                        break;
                    m.kind = -1;
                    mbar_arrive(bar);
                    ++k;
                    break;
                }
                const int kind = J.kind;
                const int B = ukind_bits(kind);
                const int TW = SH::tw(B);
                /* the next tile and its descriptor, while this one waits for its slot */
                int64_t tn;
                if (i + 1 < UCHUNK) {
                    tn = c0 + i + 1;
                    ++i;
                } else {
                    tn = c0 = c1;
                    c1 = (int64_t)atomicAdd(counter, (unsigned long long)UCHUNK);
                    i = 0;
                }
                JobDesc Jn = J;
                if (tn < ntiles && tn >= J.tile0 + (J.S + TW - 1) / TW) Jn = jobs[tile_job[tn]];
                if (k >= NST &&
                    !mbar_wait(smem_addr(&empty[s]), (uint32_t)((k / NST - 1) & 1), ab, STREAM_WAIT_CYCLES))
                    break;
                const int64_t w0 = (t - J.tile0) * TW;
                const int64_t rem = J.S - w0;   /* > 0, a multiple of 32 */
                const int cols = (int)(rem < TW ? rem : TW);
                m.out = J.out;
                m.S = J.S;
                m.nwords = J.nwords;
                m.w0 = w0;
                m.tailmask = J.tailmask;
                m.negb = J.negb;
                m.kind = kind;
                m.cols = cols;
                const uint32_t bytes = (uint32_t)cols * 4u;
                mbar_arrive_expect_tx(bar, bytes * (uint32_t)(2 * B));   /* release: the metadata is visible */
                const uint32_t dst = smem_addr(ring + (size_t)s * SLOT_WORDS);
#pragma unroll 1
                for (int q = 0; q < 2 * B; ++q) {
                    const uint32_t* src = (q < B) ? J.a + (int64_t)q * J.S : J.b + (int64_t)(q - B) * J.S;
                    bulk_copy_g2s(dst + (uint32_t)(q * TW * 4), src + w0, bytes, bar);
                }
                ++k;
                t = tn;
                J = Jn;
            }
            /* the last phase issued on each slot has landed before the block
             * exits (at once, unless a wait gave up) */
            for (int64_t j = k > NST ? k - NST : 0; j < k; ++j)
                mbar_drain(smem_addr(&full[j % NST]), (uint32_t)((j / NST) & 1), STREAM_WAIT_CYCLES);
            if (*ab && fault) atomicExch(fault, 1);
        }
        return;
    }

    int64_t k = 0;
    while (true) {
        const int s = (int)(k % NST);
        const bool ok = mbar_wait(smem_addr(&full[s]), (uint32_t)((k / NST) & 1), ab, STREAM_WAIT_CYCLES);
        if (!__all_sync(0xFFFFFFFFu, ok)) break;
        const UTileMeta m = meta[s];
        const uint32_t* slot = ring + (size_t)s * SLOT_WORDS;
        const uint32_t eb = smem_addr(&empty[s]);
        if (m.kind < 0) break;
        switch (m.kind) {
            case 0: ustream_consume<OPC, NC, SLOT_WORDS, 0>(slot, m, eb, warp, lane); break;
            case 1: ustream_consume<OPC, NC, SLOT_WORDS, 1>(slot, m, eb, warp, lane); break;
            case 2: ustream_consume<OPC, NC, SLOT_WORDS, 2>(slot, m, eb, warp, lane); break;
            case 3: ustream_consume<OPC, NC, SLOT_WORDS, 3>(slot, m, eb, warp, lane); break;
            case 4: ustream_consume<OPC, NC, SLOT_WORDS, 4>(slot, m, eb, warp, lane); break;
            case 5: ustream_consume<OPC, NC, SLOT_WORDS, 5>(slot, m, eb, warp, lane); break;
            case 6: ustream_consume<OPC, NC, SLOT_WORDS, 6>(slot, m, eb, warp, lane); break;
            case 7: ustream_consume<OPC, NC, SLOT_WORDS, 7>(slot, m, eb, warp, lane); break;
            case 8: ustream_consume<OPC, NC, SLOT_WORDS, 8>(slot, m, eb, warp, lane); break;
            case 9: ustream_consume<OPC, NC, SLOT_WORDS, 9>(slot, m, eb, warp, lane); break;
            default: break;
        }
        ++k;
    }
    if (lane == 0 && *ab && fault) atomicExch(fault, 1);
}

}  // namespace bsfp

namespace bsfp {

typedef cudaError_t (*ustream_launch_fn)(const JobDesc* jobs, const int32_t* tile_job, int64_t ntiles,
                                         unsigned long long* counter, int* fault, int grid, cudaStream_t s);
typedef cudaError_t (*ustream_prepare_fn)();

/* One compiled unified kernel: launcher, shared-memory opt-in, and the word
 * columns per tile of each kind (for the host's tile maps). */
struct UStreamEntry {
    ustream_launch_fn launch = nullptr;
    ustream_prepare_fn prepare = nullptr;
    int tw[2 * BATCH_NFMT] = {};
};

template <int OPC, int NC, int NST, int SLOT_WORDS>
cudaError_t ustream_launch(const JobDesc* jobs, const int32_t* tile_job, int64_t ntiles, unsigned long long* counter,
                           int* fault, int grid, cudaStream_t s) {
    using SH = UShape<NC, SLOT_WORDS>;
    ustream_kernel<OPC, NC, NST, SLOT_WORDS>
        <<<grid, SH::THREADS, SH::HDR + (size_t)NST * SLOT_WORDS * 4, s>>>(jobs, tile_job, ntiles, counter, fault);
    return cudaGetLastError();
}

template <int OPC, int NC, int NST, int SLOT_WORDS>
cudaError_t ustream_prepare() {
    using SH = UShape<NC, SLOT_WORDS>;
    static_assert(SH::HDR + (size_t)NST * SLOT_WORDS * 4 <= 232448, "ring fits the shared memory of one block");
    static_assert(SH::META_OFF + NST * sizeof(UTileMeta) <= (size_t)SH::HDR && 2 * NST * 8 <= SH::META_OFF,
                  "barriers and metadata fit the header");
    return cudaFuncSetAttribute(ustream_kernel<OPC, NC, NST, SLOT_WORDS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(SH::HDR + (size_t)NST * SLOT_WORDS * 4));
}

template <int OPC, int NC, int NST, int SLOT_WORDS>
UStreamEntry make_ustream_entry() {
    UStreamEntry e;
    e.launch = ustream_launch<OPC, NC, NST, SLOT_WORDS>;
    e.prepare = ustream_prepare<OPC, NC, NST, SLOT_WORDS>;
    for (int k = 0; k < 2 * BATCH_NFMT; ++k) e.tw[k] = UShape<NC, SLOT_WORDS>::tw(1 + BATCH_E[k / 2] + BATCH_M[k / 2]);
    return e;
}

/* The compiled unified kernels (ustream_inst.cu): op class 0 (add/sub) or 1
 * (mul). */
UStreamEntry ustream_entry(int opc);

}  // namespace bsfp
