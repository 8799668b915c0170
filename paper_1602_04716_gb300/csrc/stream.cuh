/*
 * stream.cuh -- the streamed element-wise kernel: the same circuits as
 * binop.cuh, with the operands' planes brought into a shared-memory ring by
 * TMA bulk copies instead of per-thread global loads.
 *
 * Layout and semantics are those of binop.cuh (Sec. 2, Fig. 1; Sec. 4,
 * Table 1); only the movement of the input slices differs.  The grid-stride
 * kernel alternates, warp by warp, between waiting for its loads and
 * running the logic, so with few resident warps (the mul circuits need
 * 120-170 registers a thread) the logic pipe idles while loads are in
 * flight.  Here one block per SM splits the roles:
 *
 *   producer warp (lane 0): for each tile of TW word columns, waits until
 *     ring stage k % NST is free, then issues one cp.async.bulk per input
 *     plane (2B copies of TW*4 bytes) completing on that stage's `full`
 *     mbarrier (expect_tx = all bytes of the stage);
 *   NC consumer warps: wait on `full`, copy their 2 words of every plane
 *     from shared memory into registers, release the stage (one arrive per
 *     warp on `empty`) and run the circuit, storing the results straight to
 *     global memory with 64-bit streaming stores.
 *
 * The ring keeps NST tiles of loads in flight whatever the consumers are
 * doing, and the consumers never wait on global memory.  Tiles go to blocks
 * round-robin (tile t to block t mod gridDim).  Shapes (consumer warps x
 * stages) are fixed per plane count B and op class so that the registers of
 * NC+1 warps and the ring fit one SM: 11 x 4 for B <= 9, 11 x 3 (add) and
 * 15 x 2 (mul) for B = 13, 12 x 2 for B = 16 and 14 x 2 for mul 1/8/7
 * (measured against neighbouring shapes on 2^28-element operands).
 *
 * Waits are bounded (tma.cuh); a block whose wait gives up stops, lets its
 * copies in flight land, and sets *p.fault, which bsfp_fault_status reports.
 * bsfp_stream_selftest exercises that path: it withholds the copies of one
 * tile (p.withhold_tile) with a short bound, so the waits on that tile run
 * out while every other wait completes.
 */
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "binop.cuh"
#include "tma.cuh"

namespace bsfp {

/* Formats and op classes compiled with a streamed kernel:
 *   the tuned formats of at most 16 planes: add/sub and mul, every mode, and
 *     their job-list form; division and fma2, every mode, where their bands
 *     below include the format (stream_inst.cu);
 *   every other format, RN and RZ (stream_band_inst.cu): mul of 12 to 24
 *     planes -- the band where the multiplier sits near the crossover of
 *     logic and HBM bounds and the grid-stride kernel, with few warps
 *     resident, leaves both pipes idle part of the time; division of 8 to 24
 *     planes with at least 3 fraction bits, where the same holds: the divider
 *     needs 64-168 registers a thread in the grid-stride kernel (3-8 warps
 *     per scheduler), while with 2 fraction bits it is light and HBM-bound
 *     and the grid-stride kernel was faster; fma2 of 10 to 19 planes with
 *     at least 4 fraction bits, bound by the logic pipe from about 11 planes
 *     on, whose grid-stride kernel holds all 3B input slices while the
 *     multiplier runs (with fewer fraction bits the multiplier is light, the
 *     op HBM-bound, and the grid-stride kernel was faster). */
constexpr bool stream_format(int E, int M) { return tuned_format(E, M) && 1 + E + M <= 16; }
constexpr bool stream_div_format(int E, int M) { return 1 + E + M >= 8 && 1 + E + M <= 24 && M >= 3; }
constexpr bool stream_fma2_format(int E, int M) { return 1 + E + M >= 10 && 1 + E + M <= 19 && M >= 4; }
constexpr bool stream_band_format(int E, int M, int opc) {
    return opc == OPC_MUL    ? (1 + E + M >= 12 && 1 + E + M <= 24)
         : opc == OPC_DIV    ? stream_div_format(E, M)
         : opc == OPC_FMA2   ? stream_fma2_format(E, M)
                             : false;
}

template <int E, int M, int OPC>
struct StreamShape {
    static constexpr int B = 1 + E + M;
    static constexpr int WPT = 2;                                   /* words per consumer thread */
    /* consumer warps x ring stages, each the fastest of its neighbours on
     * 2^28-element operands: 11 x 4 for B <= 9; for B = 13, 11 x 3 for the
     * adder (deeper ring, and its light circuit needs fewer warps) and 15 x 2
     * for mul (more warps feed its logic pipe); 12 x 2 for B = 16, except
     * mul 1/8/7 at 14 x 2 (1/5/10 mul gained nothing and its job-list form
     * spills there, and the adders stream at the copy bandwidth with 12).
     * Wider formats: 11 x 2 up to 20 planes, 8 x 2 up to 24, 6 x 2 beyond,
     * so that the ring of 2B planes fits and each thread may hold the wide
     * multipliers' registers (up to 168).  The consumer warps are spread over
     * the four schedulers by warp index mod 4, so a logic-bound kernel wants
     * a count that loads them evenly: 8 (2 each) and 11 (3, 3, 3 and 2 beside
     * the producer) ran 7-13% faster than 9 and 10 on six multipliers of
     * 17-20 planes, and 11 x 2 beat 8 x 2 by 4-8% there. */
    static constexpr int NC_ADDMUL = B <= 9 ? 11
                            : (B <= 13 ? (OPC == OPC_ADDSUB ? 11 : 15)
                                       : (B <= 16 ? ((OPC == OPC_MUL && E == 8) ? 14 : 12)
                                                  : (B <= 20 ? 11 : (B <= 24 ? 8 : 6))));
    /* division (8 to 24 planes): 15 x 2 up to 13 planes, 12 x 2 up to 17,
     * each faster than 11 x 3, 8 x 3 and the one-word-per-thread shapes on
     * 2^27-element operands; then, as for mul, 11 x 2 up to 20 planes and
     * 8 x 2 up to 24 (1-6% faster than the grid-stride kernel on seven
     * dividers of 18-22 planes at 2^26 elements).  fma2 (10 to 19 planes): 11 x 2 with the
     * addend's planes in the ring up to 13 planes; 12 x 2 beyond, where the
     * ring holds only a and b and the consumers load the addend from global
     * memory once the product is done (3B planes of 12 warps' tiles would
     * not fit).  Both were 9-14% faster than the grid-stride kernel on nine
     * formats at 2^27 elements; 15 x 2, 15 x 3 and 12 x 2 at one word per
     * thread, and 10 x 2, were slower.  18 and 19 planes take 11 x 2 with
     * the addend from global memory, so that 2B planes still fit. */
    static constexpr int NC_FMA2 = B <= 13 ? 11 : (B <= 17 ? 12 : 11);
    static constexpr int NC_DIV = B <= 13 ? 15 : (B <= 17 ? 12 : (B <= 20 ? 11 : 8));
    static constexpr int NC = OPC == OPC_DIV ? NC_DIV : (OPC == OPC_FMA2 ? NC_FMA2 : NC_ADDMUL);
    static constexpr int NST = (OPC == OPC_DIV || OPC == OPC_FMA2) ? 2
                             : (B <= 9 ? 4 : ((B <= 13 && OPC == OPC_ADDSUB) ? 3 : 2));   /* ring stages */
    static constexpr bool Z_IN_RING = OPC == OPC_FMA2 && B <= 13;   /* fma2: the addend's planes in the ring */
    static constexpr int NIN = (Z_IN_RING ? 3 : 2) * B;             /* input planes per tile */
    static constexpr int TW = 32 * NC * WPT;                        /* words per plane per tile */
    static constexpr int THREADS = 32 * (NC + 1);
    static constexpr int HDR = 128;                                 /* barriers */
    static constexpr size_t SMEM = HDR + (size_t)NST * NIN * TW * 4;
    static_assert(2 * NST * 8 <= HDR, "barriers fit the header");
    static_assert(SMEM <= 232448, "ring fits the shared memory one block may opt in to");
    static_assert((size_t)NIN * TW * 4 < (1u << 20), "a stage's bytes fit the transaction count");
};

/* One fma2 tile column pair of a consumer thread: the product of its a and b
 * slices (rounded once, kept in registers), then the addend's slices -- from
 * the ring when the shape holds them there, else from global memory -- and
 * the sum (rounded again): fma2 = round(round(a*b) + c).  The stage
 * is released once the thread has read everything it needs from it.  Reading
 * the addend only after the product keeps its B slices out of the registers
 * the multiplier needs. */
template <int E, int M, int R, class SH>
__device__ __forceinline__ void stream_fma2_tile(const BinopArgs& p, const uint32_t* src, int64_t w0, int lane,
                                                 uint32_t empty_bar) {
    constexpr int B = SH::B, TW = SH::TW, WPT = SH::WPT;
    uint32_t pr[B][WPT], z[B][WPT];
#pragma unroll
    for (int w = 0; w < WPT; ++w) {
        uint32_t x[B], y[B], o[B];
#pragma unroll
        for (int i = 0; i < B; ++i) {
            x[i] = src[i * TW + w];
            y[i] = src[(B + i) * TW + w];
        }
        column_op<E, M, R, OPC_MUL>(x, y, y, o, 0u);
#pragma unroll
        for (int i = 0; i < B; ++i) pr[i][w] = o[i];
    }
    if constexpr (SH::Z_IN_RING) {
#pragma unroll
        for (int i = 0; i < B; ++i)
#pragma unroll
            for (int w = 0; w < WPT; ++w) z[i][w] = src[(2 * B + i) * TW + w];
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(empty_bar);
    /* S is a multiple of 32, so a pair of columns is all in or all out */
    if (w0 >= p.S) return;
    if constexpr (!SH::Z_IN_RING) {
#pragma unroll
        for (int i = 0; i < B; ++i) vload<WPT>(p.c + i * p.S + w0, z[i]);
    }
    uint32_t r[B][WPT];
#pragma unroll
    for (int w = 0; w < WPT; ++w) {
        uint32_t x[B], y[B], o[B];
#pragma unroll
        for (int i = 0; i < B; ++i) {
            x[i] = pr[i][w];
            y[i] = z[i][w];
        }
        column_op<E, M, R, OPC_ADDSUB>(x, y, y, o, 0u);
#pragma unroll
        for (int i = 0; i < B; ++i) r[i][w] = o[i];
    }
    masked_store<B, WPT>(p, w0, r);
}

/* The bound is on threads only: the block size alone caps registers at
 * 65536 / THREADS.  Adding a minimum of one block per SM changes ptxas's
 * register target and schedule and made the adders about 9% slower. */
template <int E, int M, int R, int OPC>
__global__ void __launch_bounds__(StreamShape<E, M, OPC>::THREADS) stream_kernel(const BinopArgs p) {
    using SH = StreamShape<E, M, OPC>;
    constexpr int B = SH::B, NC = SH::NC, NST = SH::NST, NIN = SH::NIN, TW = SH::TW, WPT = SH::WPT;
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + NST;
    uint32_t* ring = reinterpret_cast<uint32_t*>(smem + SH::HDR);
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = (p.S + TW - 1) / TW;
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
        /* producer */
        if (lane == 0) {
            int64_t k = 0;   /* tiles issued by this block */
            for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
                const int s = (int)(k % NST);
                if (k >= NST && !mbar_wait(smem_addr(&empty[s]), (uint32_t)((k / NST - 1) & 1), ab, p.wait_cycles))
                    break;
                if (t == p.withhold_tile) continue;   /* self-test: nothing completes this stage */
                const int64_t rem = p.S - t * TW;   /* > 0, a multiple of 32 */
                const uint32_t bytes = (uint32_t)((rem < TW ? rem : TW) * 4);
                const uint32_t bar = smem_addr(&full[s]);
                mbar_arrive_expect_tx(bar, bytes * NIN);
                const uint32_t dst = smem_addr(ring + (size_t)s * NIN * TW);
#pragma unroll 1
                for (int q = 0; q < NIN; ++q) {
                    /* NIN == 2B outside the fma2 ring: the addend test folds away */
                    const uint32_t* src = (q < B) ? p.a + (int64_t)q * p.S
                                        : ((NIN == 2 * B || q < 2 * B) ? p.b + (int64_t)(q - B) * p.S
                                                                       : p.c + (int64_t)(q - 2 * B) * p.S);
                    bulk_copy_g2s(dst + (uint32_t)(q * TW * 4), src + t * TW, bytes, bar);
                }
            }
            /* the last phase issued on each stage has landed before the
             * block exits (at once, unless a wait gave up) */
            for (int64_t j = k > NST ? k - NST : 0; j < k; ++j)
                if ((int64_t)blockIdx.x + j * gridDim.x != p.withhold_tile)
                    mbar_drain(smem_addr(&full[j % NST]), (uint32_t)((j / NST) & 1), p.wait_cycles);
            if (*ab && p.fault) atomicExch(p.fault, 1);
        }
        return;
    }

    /* consumers: thread (warp, lane) owns word columns j0, j0+1 of a tile */
    const int j0 = (warp * 32 + lane) * WPT;
    int64_t k = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int s = (int)(k % NST);
        const bool ok = mbar_wait(smem_addr(&full[s]), (uint32_t)((k / NST) & 1), ab, p.wait_cycles);
        if (!__all_sync(0xFFFFFFFFu, ok)) break;   /* the warp leaves together */
        const uint32_t* src = ring + (size_t)s * NIN * TW + j0;
        if constexpr (OPC == OPC_FMA2) {
            stream_fma2_tile<E, M, R, SH>(p, src, t * TW + j0, lane, smem_addr(&empty[s]));
            continue;
        }
        uint32_t xa[B][WPT], xb[B][WPT], xc[1][WPT];
#pragma unroll
        for (int i = 0; i < B; ++i) {
#pragma unroll
            for (int w = 0; w < WPT; ++w) {
                xa[i][w] = src[i * TW + w];
                xb[i][w] = src[(B + i) * TW + w];
            }
        }
        /* every lane's slices are in registers: release the stage */
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&empty[s]));
        const int64_t w0 = t * TW + j0;
        /* S is a multiple of 32, so a pair of columns is all in or all out */
        if (w0 < p.S) binop_compute_store<E, M, R, OPC, WPT>(p, w0, xa, xb, xc);
    }
    if (lane == 0 && *ab && p.fault) atomicExch(p.fault, 1);
}

/* ------------------------------------------------------------ job lists ---
 * stream_batch_kernel: the same pipeline over the tiles of many vectors of
 * one (format, rounding, op class), for the batched plans (bsfp.h,
 * BSFP_BATCH_STREAMED).  Each vector is cut into tiles of TW word columns;
 * tile_job[t] names the vector of tile t, and tiles go to blocks
 * round-robin.  The producer reads the tile's descriptor (prefetched one
 * tile ahead), writes what the consumers need -- output, stride, tail mask,
 * sign flip, first column -- into the stage's metadata slot, then arrives
 * with the stage's byte count and issues the copies; the consumers take the
 * metadata into registers before they release the stage. */
struct StreamJob {
    const uint32_t* a;
    const uint32_t* b;
    uint32_t* out;
    int64_t S;
    int64_t nwords;
    int64_t tile0;      /* first tile of this vector in the plan's tile list */
    uint32_t tailmask;
    uint32_t negb;
};

struct StreamTileMeta {
    uint32_t* out;
    int64_t S;
    int64_t nwords;
    int64_t w0;         /* first word column of the tile */
    uint32_t tailmask;
    uint32_t negb;
};

template <int E, int M, int OPC>
struct StreamBatchShape {
    using SH = StreamShape<E, M, OPC>;
    static constexpr int HDR = 256;   /* barriers, then one metadata slot per stage */
    static constexpr int META_OFF = 64;
    static constexpr size_t SMEM = HDR + (size_t)SH::NST * SH::NIN * SH::TW * 4;
    static_assert(2 * SH::NST * 8 <= META_OFF, "barriers fit before the metadata");
    static_assert(META_OFF + SH::NST * sizeof(StreamTileMeta) <= HDR, "metadata fits the header");
    static_assert(SMEM <= 232448, "ring fits the shared memory one block may opt in to");
};

template <int E, int M, int R, int OPC>
__global__ void __launch_bounds__(StreamShape<E, M, OPC>::THREADS) stream_batch_kernel(
    const StreamJob* __restrict__ jobs, const int32_t* __restrict__ tile_job, int64_t ntiles, int* fault) {
    using SH = StreamShape<E, M, OPC>;
    using SB = StreamBatchShape<E, M, OPC>;
    constexpr int B = SH::B, NC = SH::NC, NST = SH::NST, NIN = SH::NIN, TW = SH::TW, WPT = SH::WPT;
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + NST;
    StreamTileMeta* meta = reinterpret_cast<StreamTileMeta*>(smem + SB::META_OFF);
    uint32_t* ring = reinterpret_cast<uint32_t*>(smem + SB::HDR);
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
            int64_t k = 0;
            StreamJob nj;
            if ((int64_t)blockIdx.x < ntiles) nj = jobs[tile_job[blockIdx.x]];
            for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
                const StreamJob J = nj;
                const int64_t tn = t + gridDim.x;
                if (tn < ntiles) nj = jobs[tile_job[tn]];   /* next descriptor, in flight meanwhile */
                const int s = (int)(k % NST);
                if (k >= NST && !mbar_wait(smem_addr(&empty[s]), (uint32_t)((k / NST - 1) & 1), ab, STREAM_WAIT_CYCLES))
                    break;
                const int64_t w0 = (t - J.tile0) * TW;
                const int64_t rem = J.S - w0;   /* > 0, a multiple of 32 */
                const uint32_t bytes = (uint32_t)((rem < TW ? rem : TW) * 4);
                StreamTileMeta& m = meta[s];
                m.out = J.out;
                m.S = J.S;
                m.nwords = J.nwords;
                m.w0 = w0;
                m.tailmask = J.tailmask;
                m.negb = J.negb;
                const uint32_t bar = smem_addr(&full[s]);
                mbar_arrive_expect_tx(bar, bytes * NIN);   /* release: the metadata is visible with the phase */
                const uint32_t dst = smem_addr(ring + (size_t)s * NIN * TW);
#pragma unroll 1
                for (int q = 0; q < NIN; ++q) {
                    const uint32_t* src = (q < B) ? J.a + (int64_t)q * J.S : J.b + (int64_t)(q - B) * J.S;
                    bulk_copy_g2s(dst + (uint32_t)(q * TW * 4), src + w0, bytes, bar);
                }
            }
            for (int64_t j = k > NST ? k - NST : 0; j < k; ++j)
                mbar_drain(smem_addr(&full[j % NST]), (uint32_t)((j / NST) & 1), STREAM_WAIT_CYCLES);
            if (*ab && fault) atomicExch(fault, 1);
        }
        return;
    }

    const int j0 = (warp * 32 + lane) * WPT;
    int64_t k = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int s = (int)(k % NST);
        const bool ok = mbar_wait(smem_addr(&full[s]), (uint32_t)((k / NST) & 1), ab, STREAM_WAIT_CYCLES);
        if (!__all_sync(0xFFFFFFFFu, ok)) break;
        BinopArgs p;
        p.out = meta[s].out;
        p.S = meta[s].S;
        p.nwords = meta[s].nwords;
        p.tailmask = meta[s].tailmask;
        p.negb = meta[s].negb;
        const int64_t w0 = meta[s].w0 + j0;
        const uint32_t* src = ring + (size_t)s * NIN * TW + j0;
        uint32_t xa[B][WPT], xb[B][WPT], xc[1][WPT];
#pragma unroll
        for (int i = 0; i < B; ++i) {
#pragma unroll
            for (int w = 0; w < WPT; ++w) {
                xa[i][w] = src[i * TW + w];
                xb[i][w] = src[(B + i) * TW + w];
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&empty[s]));
        /* the tile may be the shorter last one of its vector */
        if (w0 < p.S) binop_compute_store<E, M, R, OPC, WPT>(p, w0, xa, xb, xc);
    }
    if (lane == 0 && *ab && fault) atomicExch(fault, 1);
}

template <int E, int M, int R, int OPC>
cudaError_t stream_batch_launch(const StreamJob* jobs, const int32_t* tile_job, int64_t ntiles, int* fault, int grid,
                                cudaStream_t s) {
    stream_batch_kernel<E, M, R, OPC>
        <<<grid, StreamShape<E, M, OPC>::THREADS, StreamBatchShape<E, M, OPC>::SMEM, s>>>(jobs, tile_job, ntiles, fault);
    return cudaGetLastError();
}

template <int E, int M, int R, int OPC>
cudaError_t stream_batch_prepare() {
    return cudaFuncSetAttribute(stream_batch_kernel<E, M, R, OPC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)StreamBatchShape<E, M, OPC>::SMEM);
}

template <int E, int M, int R, int OPC>
cudaError_t stream_launch(const BinopArgs& p, int grid, cudaStream_t s) {
    using SH = StreamShape<E, M, OPC>;
    stream_kernel<E, M, R, OPC><<<grid, SH::THREADS, SH::SMEM, s>>>(p);
    return cudaGetLastError();
}

/* Opt the kernel in to its ring's shared memory on the current device. */
template <int E, int M, int R, int OPC>
cudaError_t stream_prepare() {
    return cudaFuncSetAttribute(stream_kernel<E, M, R, OPC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)StreamShape<E, M, OPC>::SMEM);
}

}  // namespace bsfp
