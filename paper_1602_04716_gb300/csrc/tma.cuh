/*
 * tma.cuh -- inline-PTX helpers for the streamed kernels: shared-memory
 * mbarriers and TMA bulk copies (cp.async.bulk) from global into shared
 * memory, completed on an mbarrier through its transaction count.
 *
 * Every wait is bounded: mbar_wait gives up after `limit` SM clock cycles
 * (STREAM_WAIT_CYCLES, about two seconds at 2 GHz, unless a self-test asks
 * for less), raises the block's abort flag and returns false, so a pipeline
 * that stops making progress ends with an error status instead of hanging
 * the GPU.  mbar_drain is the same bound without the abort check, used
 * before a block exits to let copies still in flight land in its shared
 * memory.
 */
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bsfp {

constexpr long long STREAM_WAIT_CYCLES = 1ll << 32;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

/* Makes the initialised barriers visible to the other threads and to the
 * TMA unit (async proxy). */
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

/* true once the phase with the given parity has completed */
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > limit) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

/* Arrive and add `bytes` to the transaction count of the current phase. */
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

/* TMA bulk copy of `bytes` (a multiple of 16, both addresses 16-byte
 * aligned) from global to shared memory, completing on barrier `bar`. */
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

}  // namespace bsfp
