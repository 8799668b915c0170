/*
 * bsfp_bench.h -- measurement support in libbsfp.  None of this is an
 * operation of the paper; it supplies the inputs and the roofline
 * denominator that the benchmarks need.  Same conventions as bsfp.h.
 */
#ifndef BSFP_BENCH_H
#define BSFP_BENCH_H

#include <stdint.h>

#include "bsfp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Seeded synthetic operands, written on the device: n B-bit encodings of
 * format 1/E/M in the standard representation (containers of
 * bsfp_container_bytes(f) bytes, out aligned to that size).  Draw i of the
 * stream (seed, stream) is SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) at
 * counter start+i+1 under a key mixed from seed and stream, and becomes:
 * sign = bit 0; fraction = bits 1..M; with h = the high 32 bits and
 * t = h mod 100, exponent field = 0 if t == 0, all ones if t == 1, else
 * 1 + (h div 100) mod (2^E - 2).  The host generator of the test suite draws
 * the identical values.  Errors as for bsfp_pack. */
bsfp_status bsfp_synth_fp_values(bsfp_format f, int64_t n, uint64_t seed, uint64_t stream, int64_t start,
                                 void* out, bsfp_stream_t s);

/* Logic-issue probe: launches grid x block threads, each running `iters`
 * rounds of BSFP_PROBE_LOP3_PER_ROUND dependent-chain 3-input logic
 * instructions (LOP3) from register operands, and writes one word per thread
 * to sink (grid*block words, 4-byte aligned).  Timed by the caller, it gives
 * the chip's sustained rate of 32-bit logic ops (lane-ops/s), the work
 * denominator of the logic roofline. */
#define BSFP_PROBE_LOP3_PER_ROUND 64
bsfp_status bsfp_lop3_probe(uint32_t* sink, int32_t grid, int32_t block, int32_t iters, uint32_t seed,
                            bsfp_stream_t s);

/* Open-loop replay of a request trace through a server: request i (job i)
 * is submitted at arrival_ns[i] nanoseconds after the start (non-decreasing;
 * the calling thread waits for each arrival time, polling completions
 * meanwhile), and done[i] receives its completion.  With release != 0 every
 * arena result is released as soon as it completes.  Returns when all have
 * completed, or BSFP_ERR_TIMEOUT after timeout_ms.  A job that fails
 * validation stops the replay with its error. */
bsfp_status bsfp_server_replay(bsfp_server srv, const bsfp_job* jobs, const int64_t* arrival_ns, int32_t n,
                               int32_t release, bsfp_completion* done, int64_t timeout_ms);

/* Number of streaming multiprocessors of the current device (0 on error). */
int32_t bsfp_num_sms(void);

#ifdef __cplusplus
}
#endif

#endif /* BSFP_BENCH_H */
