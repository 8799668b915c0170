/*
 * gen_circuit.cuh -- circuits printed gate by gate from their netlists.
 *
 * GenCircuit<E, M, R, OPC>::eval(a, b, c, r) computes the same function as
 * the circuit.cuh template for that format, rounding mode R (bit 0 toward
 * zero, bit 1 flush to zero) and op class, with one
 * 3-input logic instruction (LOP3, truth table as immediate) per gate of the
 * recorded netlist, so the instruction count is exactly the gate count G.
 * The specialisations come from gen_circuits.cuh, which circuitgen writes at
 * build time for the formats the build lists (every op and mode), and from
 * the header of the translation unit's part (add and mul under RN and RZ of
 * every other format, or, in a division unit, div under RN and RZ); where
 * `available` is false the kernels use the templates.
 *
 * Device code emits lop3.b32 through inline PTX, which the compiler keeps as
 * one instruction; host code evaluates the same truth tables bitwise (used by
 * the CPU tests of the generated netlists).
 */
#pragma once
#include <stdint.h>

namespace bsfp {

template <int E, int M, int R, int OPC>
struct GenCircuit {
    static constexpr bool available = false;
};

#if defined(__CUDA_ARCH__)
template <unsigned L>
__device__ __forceinline__ uint32_t lop3_gate(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(L));
    return d;
}
#else
/* Bit i = 4a+2b+c of L is the output for input bits a, b, c. */
template <unsigned L>
inline uint32_t lop3_gate(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t r = 0u;
    for (unsigned i = 0; i < 8; ++i)
        if ((L >> i) & 1u) r |= ((i & 4u) ? a : ~a) & ((i & 2u) ? b : ~b) & ((i & 1u) ? c : ~c);
    return r;
}
#endif

#if defined(__CUDACC__)
#define BSFP_GEN_FN __host__ __device__ __forceinline__
#else
#define BSFP_GEN_FN inline
#endif
#define BSFP_LOP3(L, x, y, z) lop3_gate<(L)>((x), (y), (z))

#if defined(BSFP_HAVE_GEN)
#include "gen_circuits.cuh"
/* add and mul (or div) under RN and RZ of the other formats of one
 * element-wise translation unit, whose build names its header */
#if defined(BSFP_GEN_PART)
#include BSFP_GEN_PART
#endif
#endif

}  // namespace bsfp
