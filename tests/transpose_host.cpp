/* Test harness: runs the in-register transposes and the shared-memory
 * staging of the CUDA library's bit_transpose.cuh on the host, lane by lane
 * and tile by tile in the order the pack and unpack kernels use them, so the
 * index and rotation logic can be compared with the oracle on a CPU.  Test
 * infrastructure only; nothing in the library calls it.  Built by the tests
 * with g++. */
#include <stdint.h>
#include <string.h>

#include <vector>

#include "bit_transpose.cuh"

using namespace bsfp;

template <int CB>
static void pack_t(const uint8_t* in, long n, int B, uint32_t* out, long S) {
    std::vector<uint8_t> s(1024 * CB);
    for (long tile = 0; tile < S / 32; ++tile) {
        const long e0 = tile * 1024;
        for (int i = 0; i < 1024; ++i)
            for (int k = 0; k < CB; ++k) s[i * CB + k] = (e0 + i < n) ? in[(e0 + i) * CB + k] : 0;
        for (int lane = 0; lane < 32; ++lane) {
            uint32_t w[8 * CB], x[8 * CB];
            stage_read_column<CB>(s.data(), lane, w);
            rows_to_planes<CB>(w, x);
            for (int b = 0; b < B; ++b) out[b * S + tile * 32 + lane] = rotl32(x[b], stage_rho<CB>(lane));
        }
    }
}

template <int CB>
static void unpack_t(const uint32_t* in, long S, int B, uint8_t* out, long n) {
    std::vector<uint8_t> s(1024 * CB);
    for (long tile = 0; tile < (n + 1023) / 1024; ++tile) {
        const long e0 = tile * 1024;
        for (int lane = 0; lane < 32; ++lane) {
            const int rho = stage_rho<CB>(lane);
            uint32_t x[8 * CB], w[8 * CB];
            for (int b = 0; b < 8 * CB; ++b) x[b] = (b < B) ? rotr32(in[b * S + tile * 32 + lane], rho) : 0u;
            planes_to_rows<CB>(x, w);
            stage_write_column<CB>(s.data(), lane, w);
        }
        for (int i = 0; i < 1024 && e0 + i < n; ++i) memcpy(out + (e0 + i) * CB, &s[i * CB], CB);
    }
}

extern "C" {

int tp_pack(int cb, const void* in, long n, int B, uint32_t* out, long S) {
    switch (cb) {
        case 1: pack_t<1>((const uint8_t*)in, n, B, out, S); return 0;
        case 2: pack_t<2>((const uint8_t*)in, n, B, out, S); return 0;
        case 4: pack_t<4>((const uint8_t*)in, n, B, out, S); return 0;
    }
    return -1;
}

int tp_unpack(int cb, const uint32_t* in, long S, int B, void* out, long n) {
    switch (cb) {
        case 1: unpack_t<1>(in, S, B, (uint8_t*)out, n); return 0;
        case 2: unpack_t<2>(in, S, B, (uint8_t*)out, n); return 0;
        case 4: unpack_t<4>(in, S, B, (uint8_t*)out, n); return 0;
    }
    return -1;
}

/* Byte offset within the warp's staging area of lane's q-th 16-byte access
 * (stage_read_column / stage_write_column). */
long tp_stage_offset(int cb, int lane, int q) {
    switch (cb) {
        case 1: return 32L * cb * lane + 16L * ((q + stage_delta<1>(lane)) & 1);
        case 2: return 32L * cb * lane + 16L * ((q + stage_delta<2>(lane)) & 3);
        case 4: return 32L * cb * lane + 16L * ((q + stage_delta<4>(lane)) & 7);
    }
    return -1;
}

}
