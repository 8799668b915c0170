/*
 * bit_transpose.cuh -- the bit-matrix transposes between the standard
 * representation and the bitslice layout (Sec. 2, Fig. 1), done inside one
 * thread's registers, and the shared-memory staging that gives each thread
 * the 32 elements of its word column.
 *
 * A thread owns one word column: elements 32c .. 32c+31.  Held one element
 * per row, the column is a 32 x 32 bit matrix whose transpose is the B plane
 * words of the column (row j = element j, word b = bit b of every element).
 * The transpose swaps the row index with the bit index one index bit at a
 * time: for K = 16, 8, 4, 2, 1 the rows j and j+K (j without bit K) exchange
 * the K-bit blocks that sit off the diagonal.  Each stage costs two
 * instructions per row pair: a byte permute for K = 16 and 8, a shift and a
 * 3-input select for K = 4, 2, 1.  Narrow containers need fewer stages:
 *   CB = 4 (32-bit rows):   stages 16, 8, 4, 2, 1 on 32 registers;
 *   CB = 2 (16-bit rows):   rows j and j+16 share a register (low and high
 *                           half), so stage 16 is the gather itself and
 *                           stages 8, 4, 2, 1 run on 16 registers;
 *   CB = 1 (8-bit rows):    rows j, j+8, j+16, j+24 share a register (one
 *                           byte each), gathered by a 4 x 4 byte transpose,
 *                           and stages 4, 2, 1 run on 8 registers.
 * The stages commute, so the same functions serve both directions.
 *
 * Staging.  A warp owns a tile of 32 columns (1024 elements, 1024*CB bytes of
 * the standard array) in shared memory, column c at byte 32*CB*c.  Lane l
 * reads or writes its column as 2*CB 16-byte chunks, starting at chunk
 * delta(l) and wrapping, so the eight lanes of each quarter-warp touch eight
 * different bank groups (no conflicts).  The thread's registers then hold its
 * column rotated by rho(l) = delta(l) * 16/CB elements: register slot r is
 * element (r + rho) mod 32.  Transposing that, plane word b comes out rotated
 * the same way, and one funnel rotate per plane word puts it right.
 */
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#include <cuda_runtime.h>
#define BSFP_TP_FN __device__ __forceinline__
#else
/* Host build (the CPU tests of the transposes): the three intrinsics and the
 * vector type the functions below use, with their CUDA semantics. */
#define BSFP_TP_FN inline
struct uint4 { uint32_t x, y, z, w; };
inline uint4 make_uint4(uint32_t x, uint32_t y, uint32_t z, uint32_t w) { return uint4{x, y, z, w}; }
inline uint32_t __byte_perm(uint32_t x, uint32_t y, uint32_t s) {
    const uint64_t v = ((uint64_t)y << 32) | x;
    uint32_t r = 0;
    for (int i = 0; i < 4; ++i) r |= (uint32_t)((v >> (8 * ((s >> (4 * i)) & 7u))) & 0xFFu) << (8 * i);
    return r;
}
inline uint32_t __funnelshift_l(uint32_t lo, uint32_t hi, uint32_t sh) {
    const uint64_t v = ((uint64_t)hi << 32) | lo;
    return (uint32_t)((v << (sh & 31u)) >> 32);
}
inline uint32_t __funnelshift_r(uint32_t lo, uint32_t hi, uint32_t sh) {
    const uint64_t v = ((uint64_t)hi << 32) | lo;
    return (uint32_t)(v >> (sh & 31u));
}
#endif

namespace bsfp {

BSFP_TP_FN uint32_t bperm(uint32_t a, uint32_t b, uint32_t sel) { return __byte_perm(a, b, sel); }

/* Stage K on the row pair (a = row j, b = row j+K): a takes b's low K-bit
 * blocks into its high blocks, b takes a's high blocks into its low ones. */
template <int K>
BSFP_TP_FN void tp_swap(uint32_t& a, uint32_t& b) {
    if constexpr (K == 16) {
        const uint32_t x = bperm(a, b, 0x5410u), y = bperm(a, b, 0x7632u);
        a = x; b = y;
    } else if constexpr (K == 8) {
        const uint32_t x = bperm(a, b, 0x6240u), y = bperm(a, b, 0x7351u);
        a = x; b = y;
    } else {
        constexpr uint32_t m = K == 4 ? 0x0F0F0F0Fu : (K == 2 ? 0x33333333u : 0x55555555u);
        const uint32_t x = (a & m) | ((b << K) & ~m);
        const uint32_t y = ((a >> K) & m) | (b & ~m);
        a = x; b = y;
    }
}

/* Stage K over the first N registers. */
template <int N, int K>
BSFP_TP_FN void tp_stage(uint32_t* x) {
#pragma unroll
    for (int j = 0; j < N; ++j)
        if ((j & K) == 0) tp_swap<K>(x[j], x[j + K]);
}

/* 32 rows of 32 bits -> 32 words: x[b] bit j = bit b of row j. */
BSFP_TP_FN void transpose32(uint32_t* x) {
    tp_stage<32, 16>(x);
    tp_stage<32, 8>(x);
    tp_stage<32, 4>(x);
    tp_stage<32, 2>(x);
    tp_stage<32, 1>(x);
}

/* 16 registers holding rows j (low half) and j+16 (high half) of 16-bit rows
 * -> 16 words: x[b] bit j = bit b of row j, for j in 0..31. */
BSFP_TP_FN void transpose16x2(uint32_t* x) {
    tp_stage<16, 8>(x);
    tp_stage<16, 4>(x);
    tp_stage<16, 2>(x);
    tp_stage<16, 1>(x);
}

/* 8 registers holding rows j, j+8, j+16, j+24 of 8-bit rows in bytes 0..3
 * -> 8 words: x[b] bit j = bit b of row j. */
BSFP_TP_FN void transpose8x4(uint32_t* x) {
    tp_stage<8, 4>(x);
    tp_stage<8, 2>(x);
    tp_stage<8, 1>(x);
}

/* 16-bit rows: w[i] = rows 2i, 2i+1 (as stored) <-> x[j] = rows j, j+16. */
BSFP_TP_FN void gather16(const uint32_t* w, uint32_t* x) {
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = bperm(w[j >> 1], w[8 + (j >> 1)], (j & 1) ? 0x7632u : 0x5410u);
}
BSFP_TP_FN void scatter16(const uint32_t* x, uint32_t* w) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        w[i] = bperm(x[2 * i], x[2 * i + 1], 0x5410u);
        w[8 + i] = bperm(x[2 * i], x[2 * i + 1], 0x7632u);
    }
}

/* 8-bit rows: w[i] = rows 4i..4i+3 (as stored) <-> x[j] = rows j, j+8, j+16,
 * j+24.  A 4 x 4 byte transpose of (w[g], w[2+g], w[4+g], w[6+g]) for g = 0,
 * 1; it is its own inverse, so it also maps x back to w. */
BSFP_TP_FN void bytes4x4(const uint32_t* in, uint32_t* out) {
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const uint32_t A = in[g], Bv = in[2 + g], C = in[4 + g], D = in[6 + g];
        const uint32_t P = bperm(A, Bv, 0x5140u), Q = bperm(A, Bv, 0x7362u);
        const uint32_t R = bperm(C, D, 0x5140u), S = bperm(C, D, 0x7362u);
        const uint32_t y0 = bperm(P, R, 0x5410u), y1 = bperm(P, R, 0x7632u);
        const uint32_t y2 = bperm(Q, S, 0x5410u), y3 = bperm(Q, S, 0x7632u);
        /* y_r = bytes r of A, B, C, D = rows 4g+r, 8+4g+r, 16+4g+r, 24+4g+r */
        out[4 * g + 0] = y0; out[4 * g + 1] = y1; out[4 * g + 2] = y2; out[4 * g + 3] = y3;
    }
}
BSFP_TP_FN void unbytes4x4(const uint32_t* x, uint32_t* w) {
    /* x[4g+r] = (rows 4g+r, 8+4g+r, 16+4g+r, 24+4g+r); w[g + 2q] = rows
     * 8q+4g .. 8q+4g+3 = byte q of x[4g .. 4g+3] */
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const uint32_t A = x[4 * g], Bv = x[4 * g + 1], C = x[4 * g + 2], D = x[4 * g + 3];
        const uint32_t P = bperm(A, Bv, 0x5140u), Q = bperm(A, Bv, 0x7362u);
        const uint32_t R = bperm(C, D, 0x5140u), S = bperm(C, D, 0x7362u);
        w[g] = bperm(P, R, 0x5410u);
        w[2 + g] = bperm(P, R, 0x7632u);
        w[4 + g] = bperm(Q, S, 0x5410u);
        w[6 + g] = bperm(Q, S, 0x7632u);
    }
}

/* Column c of a staged tile -> plane words of the column, rotated by rho:
 * out[b] bit r = bit b of element (r + rho) mod 32.  `w` is the column as
 * read (8*CB words), already rotated by rho. */
template <int CB>
BSFP_TP_FN void rows_to_planes(const uint32_t* w, uint32_t* out) {
    if constexpr (CB == 4) {
#pragma unroll
        for (int j = 0; j < 32; ++j) out[j] = w[j];
        transpose32(out);
    } else if constexpr (CB == 2) {
        gather16(w, out);
        transpose16x2(out);
    } else {
        bytes4x4(w, out);
        transpose8x4(out);
    }
}

/* The inverse: plane words (rotated by rho; 8*CB of them, zero above B) ->
 * the column's 8*CB row words in stored order, rotated by rho. */
template <int CB>
BSFP_TP_FN void planes_to_rows(uint32_t* x, uint32_t* w) {
    if constexpr (CB == 4) {
        transpose32(x);
#pragma unroll
        for (int j = 0; j < 32; ++j) w[j] = x[j];
    } else if constexpr (CB == 2) {
        transpose16x2(x);
        scatter16(x, w);
    } else {
        transpose8x4(x);
        unbytes4x4(x, w);
    }
}

/* Chunk rotation of lane l for containers of CB bytes (see the header). */
template <int CB>
BSFP_TP_FN int stage_delta(int lane) {
    return CB == 4 ? (lane & 7) : (CB == 2 ? ((lane >> 1) & 3) : ((lane >> 2) & 1));
}
template <int CB>
BSFP_TP_FN int stage_rho(int lane) {
    return stage_delta<CB>(lane) * (16 / CB);
}

/* Lane's column out of the warp's staged tile `s` (1024*CB bytes), rotated. */
template <int CB>
BSFP_TP_FN void stage_read_column(const uint8_t* s, int lane, uint32_t* w) {
    constexpr int NCH = 2 * CB;
    const int d = stage_delta<CB>(lane);
    const uint4* col = reinterpret_cast<const uint4*>(s + 32 * CB * lane);
#pragma unroll
    for (int q = 0; q < NCH; ++q) {
        const uint4 v = col[(q + d) & (NCH - 1)];
        w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
    }
}

/* Lane's column (rotated register order) into the warp's staged tile. */
template <int CB>
BSFP_TP_FN void stage_write_column(uint8_t* s, int lane, const uint32_t* w) {
    constexpr int NCH = 2 * CB;
    const int d = stage_delta<CB>(lane);
    uint4* col = reinterpret_cast<uint4*>(s + 32 * CB * lane);
#pragma unroll
    for (int q = 0; q < NCH; ++q) col[(q + d) & (NCH - 1)] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
}

BSFP_TP_FN uint32_t rotl32(uint32_t x, int r) { return __funnelshift_l(x, x, r); }
BSFP_TP_FN uint32_t rotr32(uint32_t x, int r) { return __funnelshift_r(x, x, r); }

}  // namespace bsfp
