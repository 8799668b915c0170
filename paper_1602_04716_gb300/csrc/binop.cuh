/*
 * binop.cuh -- the element-wise bitslice kernels (add/sub, mul, fma2).
 *
 * Layout (Sec. 2, Fig. 1; Sec. 4, Fig. 3): an operand of format 1/E/M and n
 * elements is B = 1+E+M planes of S 32-bit words each, plane b at word offset
 * b*S.  Word w of plane b holds bit b of elements 32w .. 32w+31 (element 32w+j
 * in bit j).  S = ceil(n/32) rounded up to a multiple of 32 words, so every
 * plane starts on a 128-byte boundary relative to the base pointer.
 *
 * One thread evaluates the circuit of circuit.cuh on WPT consecutive word
 * columns: it loads WPT words from each of the 2B (3B for fma2) input planes
 * with one vector load per plane (128-bit when WPT = 4), keeps every slice in
 * registers while the circuit runs, and stores WPT words to each of the B
 * output planes.  Neighbouring threads take neighbouring columns, so each warp
 * instruction moves 32*WPT*4 contiguous bytes of one plane.  There is no
 * shared memory and no synchronisation; the grid strides over the columns.
 *
 * Columns at or beyond the last partly filled word are masked: lanes past n
 * and every padding word of the output are written as zero, whatever the
 * inputs' padding holds.
 */
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "circuit.cuh"
#include "gen_circuit.cuh"

namespace bsfp {

/* Operation classes with a kernel of their own (sub shares the adder).  The
 * batched persistent kernels cover the first OPC_COUNT classes; division
 * runs as its plain kernel everywhere. */
enum OpClass : int { OPC_ADDSUB = 0, OPC_MUL = 1, OPC_FMA2 = 2, OPC_COUNT = 3, OPC_DIV = 3, OPC_ALL = 4 };

struct BinopArgs {
    const uint32_t* a;
    const uint32_t* b;
    const uint32_t* c;   /* fma2 addend; unused otherwise */
    uint32_t* out;
    int64_t S;           /* plane stride in words (multiple of 32) */
    int64_t nwords;      /* ceil(n / 32): columns that hold elements */
    uint32_t tailmask;   /* valid lanes of column nwords-1 */
    uint32_t negb;       /* ~0 flips b's sign slice (sub), 0 otherwise */
    int* fault;          /* device word set to 1 if a streamed kernel's wait
                            ran out of time; unused by the other kernels */
    long long wait_cycles;   /* bound of each streamed-kernel wait (SM cycles) */
    int64_t withhold_tile;   /* streamed kernel: tile whose copies are not issued
                                (bsfp_stream_selftest); -1 otherwise */
};

template <int WPT> struct VecT;
template <> struct VecT<1> { using T = uint32_t; };
template <> struct VecT<2> { using T = uint2; };
template <> struct VecT<4> { using T = uint4; };

template <int WPT>
__device__ __forceinline__ void vload(const uint32_t* p, uint32_t* w) {
    if constexpr (WPT == 1) {
        w[0] = __ldcs(p);
    } else if constexpr (WPT == 2) {
        const uint2 v = __ldcs(reinterpret_cast<const uint2*>(p));
        w[0] = v.x; w[1] = v.y;
    } else {
        const uint4 v = __ldcs(reinterpret_cast<const uint4*>(p));
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    }
}

template <int WPT>
__device__ __forceinline__ void vstore(uint32_t* p, const uint32_t* w) {
    if constexpr (WPT == 1) {
        __stcs(p, w[0]);
    } else if constexpr (WPT == 2) {
        __stcs(reinterpret_cast<uint2*>(p), make_uint2(w[0], w[1]));
    } else {
        __stcs(reinterpret_cast<uint4*>(p), make_uint4(w[0], w[1], w[2], w[3]));
    }
}

/* The circuit for one word column.  OPC_ADDSUB takes the sign flip at run
 * time (one extra gate) so that add and sub share a kernel.  Formats with a
 * generated netlist (gen_circuit.cuh) run it -- fma2 as the printed mul then
 * the printed add where only those two are printed; the others run the
 * templates. */
template <int E, int M, int R, int OPC>
__device__ __forceinline__ void column_op(uint32_t* x, uint32_t* y, const uint32_t* z, uint32_t* r, uint32_t negb) {
    constexpr int B = 1 + E + M;
    constexpr bool RZ = mode_rz(R), FTZ = mode_ftz(R);
    if constexpr (GenCircuit<E, M, R, OPC>::available) {
        if constexpr (OPC == OPC_ADDSUB) y[B - 1] ^= negb;
        GenCircuit<E, M, R, OPC>::eval(x, y, z, r);
    } else if constexpr (OPC == OPC_FMA2 && GenCircuit<E, M, R, OPC_MUL>::available &&
                         GenCircuit<E, M, R, OPC_ADDSUB>::available) {
        /* the two printed circuits in a row, the rounded product in registers */
        uint32_t p[B];
        GenCircuit<E, M, R, OPC_MUL>::eval(x, y, z, p);
        GenCircuit<E, M, R, OPC_ADDSUB>::eval(p, z, z, r);
    } else if constexpr (OPC == OPC_ADDSUB) {
        y[B - 1] ^= negb;
        fp_add<E, M, RZ, false, FTZ>(x, y, r);
    } else if constexpr (OPC == OPC_MUL) {
        fp_mul<E, M, RZ, FTZ>(x, y, r);
    } else if constexpr (OPC == OPC_DIV) {
        fp_div<E, M, RZ, FTZ>(x, y, r);
    } else {
        uint32_t p[B];
        fp_mul<E, M, RZ, FTZ>(x, y, p);
        fp_add<E, M, RZ, false, FTZ>(p, z, r);
    }
}

/* The B result slices of WPT word columns starting at w0 (a multiple of
 * WPT) to the output planes.  Masked tail: the partly filled column keeps
 * only its valid lanes and padding columns become zero. */
template <int B, int WPT>
__device__ __forceinline__ void masked_store(const BinopArgs& p, int64_t w0, uint32_t (*r)[WPT]) {
    if (w0 + WPT >= p.nwords) {
#pragma unroll
        for (int k = 0; k < WPT; ++k) {
            const int64_t w = w0 + k;
            const uint32_t m = (w + 1 < p.nwords) ? ~0u : (w + 1 == p.nwords ? p.tailmask : 0u);
#pragma unroll
            for (int i = 0; i < B; ++i) r[i][k] &= m;
        }
    }
#pragma unroll
    for (int i = 0; i < B; ++i) vstore<WPT>(p.out + i * p.S + w0, r[i]);
}

/* The circuit on WPT word columns starting at w0 (a multiple of WPT) whose
 * input slices are already in registers, then the masked stores. */
template <int E, int M, int R, int OPC, int WPT>
__device__ __forceinline__ void binop_compute_store(const BinopArgs& p, int64_t w0, const uint32_t (*xa)[WPT],
                                                    const uint32_t (*xb)[WPT], const uint32_t (*xc)[WPT]) {
    constexpr int B = 1 + E + M;
    uint32_t r[B][WPT];
#pragma unroll
    for (int k = 0; k < WPT; ++k) {
        uint32_t x[B], y[B], z[B], o[B];
#pragma unroll
        for (int i = 0; i < B; ++i) {
            x[i] = xa[i][k];
            y[i] = xb[i][k];
            z[i] = (OPC == OPC_FMA2) ? xc[(OPC == OPC_FMA2) ? i : 0][k] : 0u;
        }
        column_op<E, M, R, OPC>(x, y, z, o, p.negb);
#pragma unroll
        for (int i = 0; i < B; ++i) r[i][k] = o[i];
    }
    masked_store<B, WPT>(p, w0, r);
}

/* WPT word columns starting at w0 (a multiple of WPT). */
template <int E, int M, int R, int OPC, int WPT>
__device__ __forceinline__ void binop_chunk(const BinopArgs& p, int64_t w0) {
    constexpr int B = 1 + E + M;
    uint32_t xa[B][WPT], xb[B][WPT], xc[(OPC == OPC_FMA2) ? B : 1][WPT];
#pragma unroll
    for (int i = 0; i < B; ++i) vload<WPT>(p.a + i * p.S + w0, xa[i]);
#pragma unroll
    for (int i = 0; i < B; ++i) vload<WPT>(p.b + i * p.S + w0, xb[i]);
    if constexpr (OPC == OPC_FMA2) {
#pragma unroll
        for (int i = 0; i < B; ++i) vload<WPT>(p.c + i * p.S + w0, xc[i]);
    }
    binop_compute_store<E, M, R, OPC, WPT>(p, w0, xa, xb, xc);
}

template <int E, int M, int R, int OPC, int WPT>
__global__ void __launch_bounds__(128) binop_kernel(const BinopArgs p) {
    const int64_t nchunks = p.S / WPT;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < nchunks; ch += stride)
        binop_chunk<E, M, R, OPC, WPT>(p, ch * WPT);
}

/* Words-per-thread variants compiled per (format, op class).  Every format
 * gets a default; the formats of the mixed-format workloads (1/4/3, 1/4/4,
 * 1/5/7, 1/5/10, 1/8/7) and the paper's FP32 (1/8/23) get every variant whose
 * input slices fit comfortably in registers, for the autotuner to choose. */
constexpr bool tuned_format(int E, int M) {
    return (E == 4 && M == 3) || (E == 4 && M == 4) || (E == 5 && M == 7) || (E == 5 && M == 10) ||
           (E == 8 && M == 7) || (E == 8 && M == 23);
}
constexpr int op_inputs(int opc) { return opc == OPC_FMA2 ? 3 : 2; }
constexpr int default_wpt(int E, int M, int opc) { return op_inputs(opc) * (1 + E + M) <= 40 ? 2 : 1; }
constexpr unsigned wpt_mask(int E, int M, int opc) {
    if (!tuned_format(E, M)) return default_wpt(E, M, opc) == 2 ? 2u : 1u;
    const int in = op_inputs(opc) * (1 + E + M);
    return 1u | (in * 2 <= 128 ? 2u : 0u) | (in * 4 <= 128 ? 4u : 0u);
}

/* Host side: one launcher per (E, M, rounding mode R, OPC), covering the WPT
 * variants. */
typedef cudaError_t (*binop_launch_fn)(const BinopArgs& p, int wpt, int grid, cudaStream_t s);
typedef const void* (*binop_kernel_fn)(int wpt);
typedef cudaError_t (*stream_launch_fn)(const BinopArgs& p, int grid, cudaStream_t s);
typedef cudaError_t (*stream_prepare_fn)();
struct StreamJob;
typedef cudaError_t (*stream_batch_launch_fn)(const StreamJob* jobs, const int32_t* tile_job, int64_t ntiles,
                                              int* fault, int grid, cudaStream_t s);

/* Variant code of the streamed kernel (stream.cuh) beside the words-per-
 * thread codes 1, 2 and 4 of the grid-stride kernel. */
constexpr int VARIANT_STREAMED = 8;

struct BinopEntry {
    binop_launch_fn launch;
    binop_kernel_fn kernel;   /* the __global__ function, for occupancy queries */
    unsigned wpt_mask;        /* compiled variants: bit 0 = 1, bit 1 = 2, bit 2 = 4,
                                 bit 3 = the streamed kernel */
    int default_wpt;          /* the grid-stride default (and the streamed variant's fallback) */
    int preferred = 0;        /* the variant a call takes when no shape is set (0 = default_wpt) */
    /* the streamed kernel, where compiled (filled by stream_inst.cu) */
    stream_launch_fn stream_launch = nullptr;
    stream_prepare_fn stream_prepare = nullptr;   /* opts in to its shared memory */
    int stream_tw = 0;                            /* words per plane per tile */
    int stream_nst = 0;                           /* ring stages */
    /* its job-list form, for the batched plans */
    stream_batch_launch_fn stream_batch_launch = nullptr;
    stream_prepare_fn stream_batch_prepare = nullptr;
};

template <int E, int M, int R, int OPC>
cudaError_t binop_launch(const BinopArgs& p, int wpt, int grid, cudaStream_t s) {
    constexpr unsigned mask = wpt_mask(E, M, OPC);
    if (wpt == 1 && (mask & 1u)) {
        if constexpr ((mask & 1u) != 0) binop_kernel<E, M, R, OPC, 1><<<grid, 128, 0, s>>>(p);
    } else if (wpt == 2 && (mask & 2u)) {
        if constexpr ((mask & 2u) != 0) binop_kernel<E, M, R, OPC, 2><<<grid, 128, 0, s>>>(p);
    } else if (wpt == 4 && (mask & 4u)) {
        if constexpr ((mask & 4u) != 0) binop_kernel<E, M, R, OPC, 4><<<grid, 128, 0, s>>>(p);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int E, int M, int R, int OPC>
const void* binop_kernel_ptr(int wpt) {
    constexpr unsigned mask = wpt_mask(E, M, OPC);
    if constexpr ((mask & 1u) != 0) if (wpt == 1) return (const void*)binop_kernel<E, M, R, OPC, 1>;
    if constexpr ((mask & 2u) != 0) if (wpt == 2) return (const void*)binop_kernel<E, M, R, OPC, 2>;
    if constexpr ((mask & 4u) != 0) if (wpt == 4) return (const void*)binop_kernel<E, M, R, OPC, 4>;
    return nullptr;
}

template <int E, int M, int R, int OPC>
constexpr BinopEntry make_entry() {
    return BinopEntry{binop_launch<E, M, R, OPC>, binop_kernel_ptr<E, M, R, OPC>, wpt_mask(E, M, OPC),
                      (wpt_mask(E, M, OPC) & 2u) ? 2 : 1};
}

/* Table of every compiled (E, M, rounding, op class); filled by the
 * per-exponent translation units. */
constexpr int TAB_E = 9, TAB_M = 24, TAB_R = 4;
extern BinopEntry g_binop_table[TAB_E][TAB_M][TAB_R][OPC_ALL];

}  // namespace bsfp
