/*
 * batch.cuh -- the batched persistent launch: many independent vectors of
 * mixed formats and ops in one kernel per op class.
 *
 * Work list.  Each job (one vector op) is cut into tiles of TILE = 128 * WPT *
 * R word columns; tiles of all jobs of one op class are numbered 0..ntiles-1
 * and tile_job[t] names the job of tile t.  A persistent CTA takes tiles from
 * an atomic counter until they run out: thread 0 claims the next tile (and
 * reads its job index and descriptor) while the block computes the current
 * one, so the scheduling latency overlaps compute.  Within a tile, thread t
 * handles R chunks of WPT columns, chunk r at column 128*WPT*r + WPT*t, so
 * each round of loads is one coalesced row per plane, as in the plain kernel.
 *
 * The job's format and rounding select a branch of a compile-time switch
 * over the formats the kernel is built for; every branch is the same
 * binop_chunk as the plain kernels, so results are bit-identical to them.
 */
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "binop.cuh"

namespace bsfp {

/* The formats compiled into the batched kernels: the mixed-format set
 * 1/4/3, 1/4/4, 1/5/7, 1/5/10, 1/8/7.  Kind = 2 * format index + rounding. */
constexpr int BATCH_NFMT = 5;
constexpr int BATCH_E[BATCH_NFMT] = {4, 4, 5, 5, 8};
constexpr int BATCH_M[BATCH_NFMT] = {3, 4, 7, 10, 7};
/* R: chunks per thread per tile.  One chunk (8,192 elements per tile at 2
 * words per thread) balances the CTAs best: against R = 4 and 2 it made
 * persistent plans of 256-4,096 vectors 2-9% faster (measured). */
constexpr int BATCH_ROUNDS = 1;

struct JobDesc {
    const uint32_t* a;
    const uint32_t* b;
    const uint32_t* c;
    uint32_t* out;
    int64_t S;
    int64_t nwords;
    int64_t tile0;       /* first tile of this job in its op class */
    uint32_t tailmask;
    uint32_t negb;
    int32_t kind;
    int32_t pad;
};

template <int OPC, int WPT, int K>
__device__ __forceinline__ void batch_chunk_kind(const BinopArgs& p, int64_t w0) {
    constexpr int F = K / 2;
    constexpr bool RZ = (K & 1) != 0;
    binop_chunk<BATCH_E[F], BATCH_M[F], RZ, OPC, WPT>(p, w0);
}

template <int OPC, int WPT>
__device__ __forceinline__ void batch_chunk(int kind, const BinopArgs& p, int64_t w0) {
    switch (kind) {
        case 0: batch_chunk_kind<OPC, WPT, 0>(p, w0); break;
        case 1: batch_chunk_kind<OPC, WPT, 1>(p, w0); break;
        case 2: batch_chunk_kind<OPC, WPT, 2>(p, w0); break;
        case 3: batch_chunk_kind<OPC, WPT, 3>(p, w0); break;
        case 4: batch_chunk_kind<OPC, WPT, 4>(p, w0); break;
        case 5: batch_chunk_kind<OPC, WPT, 5>(p, w0); break;
        case 6: batch_chunk_kind<OPC, WPT, 6>(p, w0); break;
        case 7: batch_chunk_kind<OPC, WPT, 7>(p, w0); break;
        case 8: batch_chunk_kind<OPC, WPT, 8>(p, w0); break;
        case 9: batch_chunk_kind<OPC, WPT, 9>(p, w0); break;
        default: break;
    }
}

/* Persistent kernel over the tiles of one op class.  counter must be zero at
 * launch (the plan's graph clears it first). */
template <int OPC, int WPT>
__global__ void __launch_bounds__(128) batch_kernel(const JobDesc* __restrict__ jobs,
                                                    const int32_t* __restrict__ tile_job, int64_t ntiles,
                                                    unsigned long long* counter) {
    constexpr int64_t TILE = 128 * WPT * BATCH_ROUNDS;
    __shared__ int64_t s_tile[2];
    __shared__ JobDesc s_job[2];
    int cur = 0;
    if (threadIdx.x == 0) {
        const int64_t t = (int64_t)atomicAdd(counter, 1ull);
        s_tile[0] = t;
        if (t < ntiles) s_job[0] = jobs[tile_job[t]];
    }
    __syncthreads();
    while (true) {
        const int64_t t = s_tile[cur];
        if (t >= ntiles) break;
        /* claim the next tile while this one is computed */
        if (threadIdx.x == 0) {
            const int64_t tn = (int64_t)atomicAdd(counter, 1ull);
            s_tile[cur ^ 1] = tn;
            if (tn < ntiles) s_job[cur ^ 1] = jobs[tile_job[tn]];
        }
        const JobDesc& d = s_job[cur];
        BinopArgs p;
        p.a = d.a;
        p.b = d.b;
        p.c = d.c;
        p.out = d.out;
        p.S = d.S;
        p.nwords = d.nwords;
        p.tailmask = d.tailmask;
        p.negb = d.negb;
        p.fault = nullptr;
        p.wait_cycles = 0;
        p.withhold_tile = -1;
        const int kind = d.kind;
        const int64_t base = (t - d.tile0) * TILE + (int64_t)threadIdx.x * WPT;
#pragma unroll 1
        for (int r = 0; r < BATCH_ROUNDS; ++r) {
            const int64_t w0 = base + (int64_t)r * 128 * WPT;
            if (w0 < p.S) batch_chunk<OPC, WPT>(kind, p, w0);
        }
        __syncthreads();
        cur ^= 1;
    }
}

/* Host launchers, one per (op class, WPT); defined in batch_inst.cu. */
typedef cudaError_t (*batch_launch_fn)(const JobDesc* jobs, const int32_t* tile_job, int64_t ntiles,
                                       unsigned long long* counter, int grid, cudaStream_t s);
batch_launch_fn batch_launcher(int opc, int wpt);
const void* batch_kernel_ptr(int opc, int wpt);

/* Kind of a format in the batched set, or -1 (also for the flush-to-zero
 * modes, which run as plain kernels). */
inline int batch_kind(int E, int M, int rnd) {
    if (rnd != 0 && rnd != 1) return -1;
    for (int i = 0; i < BATCH_NFMT; ++i)
        if (BATCH_E[i] == E && BATCH_M[i] == M) return 2 * i + (rnd ? 1 : 0);
    return -1;
}

}  // namespace bsfp
