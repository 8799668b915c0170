/*
 * synth_gen.cu -- seeded synthetic operands on the device (declared in
 * bsfp_bench.h).  Input generation only: none of the method's arithmetic is
 * here.
 *
 * The generator is SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used counter-based: draw i of
 * a stream is the SplitMix64 finaliser applied to key + (i+1) * gamma, with
 * gamma = 0x9E3779B97F4A7C15 and the finaliser's published constants.  The key
 * is the finaliser applied to seed * gamma + stream * 0xD1B54A32D192ED03.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "bsfp_bench.h"

namespace bsfp {

__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <typename T>
__global__ void synth_fp_kernel(T* out, int64_t n, uint64_t key, int64_t start, int E, int M) {
    const uint64_t emax = (1ull << E) - 1ull;
    const uint64_t fmask = (1ull << M) - 1ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t r = sm64_mix(key + (uint64_t)(start + i + 1) * 0x9E3779B97F4A7C15ull);
        const uint64_t s = r & 1ull;
        const uint64_t f = (r >> 1) & fmask;
        const uint64_t h = r >> 32;
        const uint64_t t = h % 100ull;
        const uint64_t e = (t == 0) ? 0ull : (t == 1 ? emax : 1ull + (h / 100ull) % (emax - 1ull));
        out[i] = (T)((s << (E + M)) | (e << M) | f);
    }
}

}  // namespace bsfp

extern "C" bsfp_status bsfp_synth_fp_values(bsfp_format f, int64_t n, uint64_t seed, uint64_t stream, int64_t start,
                                            void* out, bsfp_stream_t s) {
    const int cb = bsfp_container_bytes(f);
    if (cb < 0) return BSFP_ERR_FORMAT;
    if (n < 0 || n > BSFP_MAX_N || start < 0) return BSFP_ERR_SIZE;
    if (n == 0) return BSFP_OK;
    if (!out) return BSFP_ERR_NULL;
    if (((uintptr_t)out & (uintptr_t)(cb - 1)) != 0) return BSFP_ERR_ALIGN;
    const uint64_t key = bsfp::sm64_mix(seed * 0x9E3779B97F4A7C15ull + stream * 0xD1B54A32D192ED03ull);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256, cap = (int64_t)(sms > 0 ? sms : 1) * 16;
    const int grid = (int)(want < cap ? want : cap);
    cudaStream_t st = (cudaStream_t)s;
    const int E = f.exp_bits, M = f.man_bits;
    if (cb == 1) bsfp::synth_fp_kernel<uint8_t><<<grid, 256, 0, st>>>((uint8_t*)out, n, key, start, E, M);
    else if (cb == 2) bsfp::synth_fp_kernel<uint16_t><<<grid, 256, 0, st>>>((uint16_t*)out, n, key, start, E, M);
    else bsfp::synth_fp_kernel<uint32_t><<<grid, 256, 0, st>>>((uint32_t*)out, n, key, start, E, M);
    return cudaGetLastError() == cudaSuccess ? BSFP_OK : BSFP_ERR_CUDA;
}
