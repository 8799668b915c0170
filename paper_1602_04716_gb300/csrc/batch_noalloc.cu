/*
 * batch_noalloc.cu -- the batched launch for callers that cannot allocate
 * device memory (bsfp_batch_run_noalloc in bsfp.h).
 *
 * A batch plan keeps its scratch (job descriptors, the tile-to-job map and
 * the tile counters) in a buffer it allocates.  This entry point keeps the
 * same scratch in one file-scope __device__ array instead, of a fixed size
 * set by BSFP_NOALLOC_MAX_JOBS and BSFP_NOALLOC_MAX_TILES, so a call performs
 * no allocation of any kind.  It runs the same persistent kernels as a plan
 * (batch_kernel, 2 words per thread), so its results are bit-identical to a
 * plan's.
 *
 * One call:
 *   1. validates every job on the host (nothing is launched on an error);
 *   2. copies the caller's bsfp_job array into the scratch array;
 *   3. launches a one-block prologue kernel that turns the raw jobs into the
 *      descriptors and tile map the persistent kernels read, per op class,
 *      and zeroes the tile counters (checking its class totals against the
 *      host's, see noalloc_prologue);
 *   4. launches one persistent kernel per op class present, then a plain
 *      kernel for each job whose format is outside the persistent set.
 *
 * Scratch layout (byte offsets into g_noalloc_scratch):
 *   [0, 256)       tile counters, one per op class
 *   OFF_RAW        the caller's jobs as copied, BSFP_NOALLOC_MAX_JOBS entries
 *   OFF_DESC       descriptors, grouped by op class (class g from desc0[g])
 *   OFF_MAP        tile -> class-local job index, grouped by op class
 *
 * The host never dereferences g_noalloc_scratch: in host code that name is a
 * stand-in, not a device address.  The device address comes from
 * cudaGetSymbolAddress, once per device, with that device current.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "batch.cuh"
#include "bsfp.h"
#include "internal.h"

namespace bsfp {
namespace {

constexpr int NA_WPT = 2;
constexpr int64_t NA_TILE = 128LL * NA_WPT * BATCH_ROUNDS; /* words per tile, as in a plan */
constexpr int NA_THREADS = 1024;                          /* prologue block size */
constexpr int NA_PER_THREAD = BSFP_NOALLOC_MAX_JOBS / NA_THREADS;
static_assert(BSFP_NOALLOC_MAX_JOBS % NA_THREADS == 0, "jobs per prologue thread must be whole");

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t OFF_CNT = 0;
constexpr size_t OFF_RAW = 256;
constexpr size_t OFF_DESC = OFF_RAW + align256(sizeof(bsfp_job) * BSFP_NOALLOC_MAX_JOBS);
constexpr size_t OFF_MAP = OFF_DESC + align256(sizeof(JobDesc) * BSFP_NOALLOC_MAX_JOBS);
constexpr size_t SCRATCH_BYTES = OFF_MAP + sizeof(int32_t) * (size_t)BSFP_NOALLOC_MAX_TILES;

/* First descriptor and first map entry of each op class, and each class's
 * job and tile totals (host-computed from the validated jobs). */
struct ClassBase {
    int32_t desc0[OPC_COUNT];
    int32_t map0[OPC_COUNT];
    int32_t njob[OPC_COUNT];
    int32_t ntile[OPC_COUNT];
};

__device__ int dev_opclass(int op) {
    return (op == BSFP_OP_ADD || op == BSFP_OP_SUB) ? OPC_ADDSUB
           : op == BSFP_OP_MUL                       ? OPC_MUL
           : op == BSFP_OP_FMA2                      ? OPC_FMA2
                                                     : -1;
}

/* Kind of a format in the batched set (as batch_kind on the host), or -1. */
template <int I = 0>
__device__ int dev_kind(int E, int M, int rnd) {
    if (rnd != 0 && rnd != 1) return -1;
    if constexpr (I == BATCH_NFMT) {
        return -1;
    } else {
        constexpr int e = BATCH_E[I], m = BATCH_M[I];
        return (E == e && M == m) ? 2 * I + (rnd ? 1 : 0) : dev_kind<I + 1>(E, M, rnd);
    }
}

/* Exclusive prefix sums over the block of V per-thread counts. */
template <int V>
__device__ void block_exclusive_scan(int32_t (&v)[V]) {
    __shared__ int32_t warp_tot[V][NA_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t incl[V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
        int32_t x = v[k];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        incl[k] = x;
        if (lane == 31) warp_tot[k][warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < V; ++k) {
            int32_t x = warp_tot[k][lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, x, d);
                if (lane >= d) x += y;
            }
            warp_tot[k][lane] = x;   /* inclusive over warps */
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < V; ++k) v[k] = incl[k] - v[k] + (warp ? warp_tot[k][warp - 1] : 0);
}

/* Raw jobs -> per-class descriptors and tile map; counters to zero.  The
 * host has validated every job, so the persistent subset and its tile counts
 * here equal the host's -- unless the copied jobs differ from the validated
 * ones (page-locked jobs changed before the copy ran).  Writes stay inside
 * the scratch whatever the jobs hold, and at the end the last thread, whose
 * running counts are then the class totals, compares them with the host's:
 * on a mismatch it sets every class counter past any tile, so the persistent
 * kernels take no tile, and raises the fault word. */
__global__ void __launch_bounds__(NA_THREADS) noalloc_prologue(unsigned char* scratch, int32_t njobs, ClassBase base,
                                                             int* fault) {
    const bsfp_job* raw = reinterpret_cast<const bsfp_job*>(scratch + OFF_RAW);
    JobDesc* desc = reinterpret_cast<JobDesc*>(scratch + OFF_DESC);
    int32_t* map = reinterpret_cast<int32_t*>(scratch + OFF_MAP);
    unsigned long long* counters = reinterpret_cast<unsigned long long*>(scratch + OFF_CNT);
    if (threadIdx.x < OPC_COUNT) counters[threadIdx.x] = 0ull;

    int cls[NA_PER_THREAD];
    int32_t ntl[NA_PER_THREAD];
    int32_t cnt[2 * OPC_COUNT] = {0, 0, 0, 0, 0, 0};   /* jobs per class, tiles per class */
#pragma unroll
    for (int k = 0; k < NA_PER_THREAD; ++k) {
        const int j = threadIdx.x * NA_PER_THREAD + k;
        cls[k] = -1;
        ntl[k] = 0;
        if (j < njobs) {
            const bsfp_job J = raw[j];
            const int g = dev_opclass(J.op);
            if (g >= 0 && J.n > 0 && dev_kind(J.f.exp_bits, J.f.man_bits, J.f.rnd) >= 0) {
                const int64_t S = ((J.n + 31) / 32 + 31) / 32 * 32;
                const int64_t t = (S + NA_TILE - 1) / NA_TILE;
                cls[k] = g;
                /* clamped so that the sums stay in range; more than the
                 * limit can only come from changed jobs, a mismatch anyway */
                ntl[k] = (int32_t)(t < BSFP_NOALLOC_MAX_TILES ? t : BSFP_NOALLOC_MAX_TILES + 1);
                cnt[g] += 1;
                cnt[OPC_COUNT + g] += ntl[k];
            }
        }
    }
    block_exclusive_scan<2 * OPC_COUNT>(cnt);
#pragma unroll
    for (int k = 0; k < NA_PER_THREAD; ++k) {
        const int g = cls[k];
        if (g < 0) continue;
        const int j = threadIdx.x * NA_PER_THREAD + k;
        const bsfp_job J = raw[j];
        JobDesc d;
        d.a = J.a;
        d.b = J.b;
        d.c = J.c;
        d.out = J.out;
        d.S = ((J.n + 31) / 32 + 31) / 32 * 32;
        d.nwords = (J.n + 31) / 32;
        d.tile0 = cnt[OPC_COUNT + g];
        d.tailmask = (J.n % 32) ? ((1u << (J.n % 32)) - 1u) : ~0u;
        d.negb = (J.op == BSFP_OP_SUB) ? ~0u : 0u;
        d.kind = dev_kind(J.f.exp_bits, J.f.man_bits, J.f.rnd);
        d.pad = 0;
        const int32_t local = cnt[g];
        if (base.desc0[g] + local < BSFP_NOALLOC_MAX_JOBS) desc[base.desc0[g] + local] = d;
        for (int32_t q = 0; q < ntl[k]; ++q) {
            const int64_t m = (int64_t)base.map0[g] + cnt[OPC_COUNT + g] + q;
            if (m < BSFP_NOALLOC_MAX_TILES) map[m] = local;
        }
        cnt[g] += 1;
        cnt[OPC_COUNT + g] += ntl[k];
    }
    if (threadIdx.x == NA_THREADS - 1) {
        bool same = true;
#pragma unroll
        for (int g = 0; g < OPC_COUNT; ++g) same = same && cnt[g] == base.njob[g] && cnt[OPC_COUNT + g] == base.ntile[g];
        if (!same) {
#pragma unroll
            for (int g = 0; g < OPC_COUNT; ++g) counters[g] = 1ull << 62;
            if (fault) atomicExch(fault, 1);
        }
    }
}

}  // namespace
}  // namespace bsfp

/* The scratch: shared by every call on a device, kept until the process
 * exits, holding whatever the last call left in it. */
static __device__ __align__(256) unsigned char g_noalloc_scratch[bsfp::SCRATCH_BYTES];

namespace {

constexpr int NA_MAX_DEVICES = 64;

/* Per-device set-up, done once by the first call on that device. */
struct NoallocDevice {
    std::atomic<bool> ready{false};
    unsigned char* scratch = nullptr;   /* device address of g_noalloc_scratch */
    int grid_cap[bsfp::OPC_COUNT] = {0, 0, 0};
};
NoallocDevice g_na_dev[NA_MAX_DEVICES];
std::mutex g_na_mu;

bsfp_status noalloc_setup(int dev, NoallocDevice** out) {
    if (dev < 0 || dev >= NA_MAX_DEVICES) return BSFP_ERR_UNSUPPORTED;
    NoallocDevice& d = g_na_dev[dev];
    if (!d.ready.load(std::memory_order_acquire)) {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!d.ready.load(std::memory_order_relaxed)) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return bsfp::set_cuda_error(e);
            for (int g = 0; g < bsfp::OPC_COUNT; ++g) {
                int occ = 0;
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bsfp::batch_kernel_ptr(g, bsfp::NA_WPT), 128,
                                                                  0);
                if (e != cudaSuccess) return bsfp::set_cuda_error(e);
                d.grid_cap[g] = bsfp::device_num_sms() * (occ > 0 ? occ : 1);
            }
            d.scratch = static_cast<unsigned char*>(p);
            d.ready.store(true, std::memory_order_release);
        }
    }
    *out = &d;
    return BSFP_OK;
}

}  // namespace

using namespace bsfp;

extern "C" bsfp_status bsfp_batch_run_noalloc(const bsfp_job* jobs, int32_t njobs, bsfp_stream_t s) {
    NvtxRange range("bsfp_batch_run_noalloc");
    if (njobs < 0 || njobs > BSFP_NOALLOC_MAX_JOBS) return BSFP_ERR_SIZE;
    if (njobs == 0) return BSFP_OK;
    if (!jobs) return BSFP_ERR_NULL;
    const cudaStream_t st = (cudaStream_t)s;

    /* 1. validate everything; count the persistent jobs and tiles per class */
    int32_t njob_c[OPC_COUNT] = {0, 0, 0};
    int64_t ntile_c[OPC_COUNT] = {0, 0, 0};
    bool any_plain = false;
    for (int32_t i = 0; i < njobs; ++i) {
        const bsfp_job& j = jobs[i];
        PreparedOp po;
        const bsfp_status v = prepare_binop(j.f, j.op, j.a, j.b, j.c, j.out, j.n, &po);
        if (v != BSFP_OK) return v;
        if (po.skip) continue;
        if (po.opc >= OPC_COUNT || batch_kind(j.f.exp_bits, j.f.man_bits, j.f.rnd) < 0) {
            any_plain = true;
            continue;
        }
        njob_c[po.opc] += 1;
        ntile_c[po.opc] += (po.args.S + NA_TILE - 1) / NA_TILE;
    }
    const int64_t tiles = ntile_c[0] + ntile_c[1] + ntile_c[2];
    if (tiles > BSFP_NOALLOC_MAX_TILES) return BSFP_ERR_SIZE;

    int64_t launched = 0;
    bsfp_status rc = BSFP_OK;
    if (tiles > 0) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return set_cuda_error(e);
        NoallocDevice* D = nullptr;
        const bsfp_status su = noalloc_setup(dev, &D);
        if (su != BSFP_OK) return su;

        /* 2. the raw jobs into the scratch */
        e = cudaMemcpyAsync(D->scratch + OFF_RAW, jobs, sizeof(bsfp_job) * (size_t)njobs, cudaMemcpyHostToDevice,
                            st);
        if (e != cudaSuccess) return set_cuda_error(e);

        /* 3. descriptors, tile map, zeroed counters */
        ClassBase base;
        int32_t d0 = 0, m0 = 0;
        for (int g = 0; g < OPC_COUNT; ++g) {
            base.desc0[g] = d0;
            base.map0[g] = m0;
            base.njob[g] = njob_c[g];
            base.ntile[g] = (int32_t)ntile_c[g];
            d0 += njob_c[g];
            m0 += (int32_t)ntile_c[g];
        }
        noalloc_prologue<<<1, NA_THREADS, 0, st>>>(D->scratch, njobs, base, current_fault_word());
        e = cudaGetLastError();
        if (e != cudaSuccess) return set_cuda_error(e);
        launched += 1;

        /* 4. one persistent kernel per op class present */
        unsigned long long* counters = reinterpret_cast<unsigned long long*>(D->scratch + OFF_CNT);
        const JobDesc* desc = reinterpret_cast<const JobDesc*>(D->scratch + OFF_DESC);
        const int32_t* map = reinterpret_cast<const int32_t*>(D->scratch + OFF_MAP);
        for (int g = 0; g < OPC_COUNT && rc == BSFP_OK; ++g) {
            if (ntile_c[g] == 0) continue;
            const int grid = (int)(ntile_c[g] < D->grid_cap[g] ? ntile_c[g] : D->grid_cap[g]);
            e = batch_launcher(g, NA_WPT)(desc + base.desc0[g], map + base.map0[g], ntile_c[g], counters + g, grid,
                                          st);
            if (e != cudaSuccess) rc = set_cuda_error(e);
            else launched += 1;
        }
    }
    /* jobs outside the persistent formats: their plain kernels */
    for (int32_t i = 0; i < njobs && any_plain && rc == BSFP_OK; ++i) {
        const bsfp_job& j = jobs[i];
        if (opclass(j.op) < OPC_COUNT && batch_kind(j.f.exp_bits, j.f.man_bits, j.f.rnd) >= 0) continue;
        PreparedOp po;
        rc = prepare_binop(j.f, j.op, j.a, j.b, j.c, j.out, j.n, &po);
        if (rc == BSFP_OK && !po.skip) {
            rc = launch_prepared(po, st);
            if (rc == BSFP_OK) launched += 1;
        }
    }
    count_launches(launched);
    return rc;
}
