/*
 * bsfp.h -- C ABI of libbsfp: bitslice custom-precision floating point on
 * one NVIDIA GB300 (sm_103a).
 *
 * The operations are those of Xu & Gregg, "Customizable Precision of
 * Floating-Point Arithmetic with Bitslice Vector Types" (arXiv 1602.04716):
 * vectors of floats of a programmer-chosen format, stored in bitslice form,
 * with add/sub and mul computed by software logic circuits over whole words
 * (Sec. 3-4), rounding to nearest-even or toward zero (Sec. 4).
 *
 * FORMAT.  1/E/M: one sign bit, E exponent bits (bias 2^(E-1)-1), M fraction
 * bits, B = 1+E+M <= 32; 2 <= E <= 8, 1 <= M <= 23.  The paper's FP8, FP16
 * and FP32 (Sec. 5.2) are 1/4/3, 1/5/10 and 1/8/23.  Exponent field 0 encodes
 * zero and subnormals, the all-ones field Inf (fraction 0) and NaN (otherwise),
 * as in IEEE 754; results that are NaN are the canonical NaN (sign 0, fraction
 * 1 << (M-1)).  RN overflows to Inf, RZ to the largest finite value; an exact
 * zero sum is +0 unless both addends are -0.  Every result is the exact
 * result rounded once.
 *
 * STANDARD REPRESENTATION.  Element i is its B-bit encoding, right-aligned in
 * a uint8_t (B <= 8), uint16_t (B <= 16) or uint32_t (B <= 32) container at
 * index i.  Bits above B are ignored on input and zero on output.
 *
 * BITSLICE REPRESENTATION (Sec. 2, Fig. 1; Sec. 4, Fig. 3).  B planes of S =
 * bsfp_plane_stride(n) 32-bit words, plane b at word offset b*S.  Bit b of
 * element i is bit (i mod 32) of word b*S + i/32: plane 0 is the least
 * significant fraction bit, planes M..M+E-1 the exponent, plane B-1 the sign.
 * Lanes past n and words past ceil(n/32) are padding; every output of this
 * library writes them as zero.
 *
 * CONVENTIONS.  All pointers passed to pack/unpack/ops are device memory owned
 * by the caller; the library never allocates or frees on these calls and
 * keeps no pointer after it returns.  Bitslice pointers must be 16-byte
 * aligned; standard arrays aligned to their container size.  Calls are
 * asynchronous on the given stream (NULL = the legacy default stream); a
 * validation error returns before anything is launched, a launch error
 * returns BSFP_ERR_CUDA.  n == 0 is valid and launches nothing.  An output
 * may be the same pointer as an input; partial overlap is undefined.  Calls
 * act on the current CUDA device.
 */
#ifndef BSFP_H
#define BSFP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
struct CUstream_st;
typedef struct CUstream_st* bsfp_stream_t;

/* Rounding (Sec. 4): round to nearest, ties to even; round toward zero.
 * The _FTZ modes add flush to zero (not in the paper; the optional mode that
 * trades gradual underflow for fewer gates): an operand whose exponent field
 * is 0 is read as a zero of its sign, and a result whose exact magnitude is
 * below the smallest normal (tiny before rounding) is a zero of its sign.
 * The _FTZ modes are compiled for 1/4/3, 1/4/4, 1/5/7, 1/5/10, 1/8/7 and
 * 1/8/23; other formats return BSFP_ERR_UNSUPPORTED for them. */
typedef enum { BSFP_RN = 0, BSFP_RZ = 1, BSFP_RN_FTZ = 2, BSFP_RZ_FTZ = 3 } bsfp_round;

/* Format 1/E/M with rounding mode.  Passed by value. */
typedef struct {
    int32_t exp_bits; /* E, 2..8 */
    int32_t man_bits; /* M, 1..23 */
    int32_t rnd;      /* bsfp_round: 0..3 */
} bsfp_format;

typedef enum {
    BSFP_OK = 0,
    BSFP_ERR_FORMAT = -1,      /* E, M or rounding out of range */
    BSFP_ERR_NULL = -2,        /* required pointer is NULL */
    BSFP_ERR_ALIGN = -3,       /* pointer not aligned as required */
    BSFP_ERR_SIZE = -4,        /* n < 0 or n > BSFP_MAX_N, or a bad count */
    BSFP_ERR_UNSUPPORTED = -5, /* valid request that the compiled library does not cover */
    BSFP_ERR_CUDA = -6,        /* a CUDA call failed; see bsfp_last_cuda_error */
    BSFP_ERR_BUDGET = -7,      /* a request larger than a server's whole budget */
    BSFP_ERR_TIMEOUT = -8      /* a bounded wait ran out */
} bsfp_status;

/* Operation codes (bsfp_op_name, batch jobs, autotune, gate count). */
typedef enum { BSFP_OP_ADD = 0, BSFP_OP_SUB = 1, BSFP_OP_MUL = 2, BSFP_OP_FMA2 = 3, BSFP_OP_DIV = 4 } bsfp_op;

#define BSFP_MAX_N (((int64_t)1) << 40)

/* ---------------------------------------------------------------- sizes --- */
/* Plane stride in 32-bit words for n elements: ceil(n/32) rounded up to a
 * multiple of 32 (128-byte plane rows).  n < 0 returns -1. */
int64_t bsfp_plane_stride(int64_t n);
/* Bytes of one bitslice operand: B * stride * 4; -1 on a bad format or n. */
int64_t bsfp_bitslice_bytes(bsfp_format f, int64_t n);
/* Container bytes of the standard representation: 1, 2 or 4; -1 on a bad
 * format. */
int32_t bsfp_container_bytes(bsfp_format f);

/* ------------------------------------------------------- pack / unpack --- */
/* pack (Sec. 4, "helper operations for transforming data in the standard
 * format"; layout Sec. 2, Fig. 1): std_in[n] containers -> bs_out (B planes
 * of stride bsfp_plane_stride(n)).  Padding of bs_out is written as zero.
 * std_in must not overlap bs_out. */
bsfp_status bsfp_pack(bsfp_format f, const void* std_in, int64_t n, uint32_t* bs_out, bsfp_stream_t s);
/* unpack: the inverse of pack; writes exactly n containers of std_out. */
bsfp_status bsfp_unpack(bsfp_format f, const uint32_t* bs_in, int64_t n, void* std_out, bsfp_stream_t s);

/* --------------------------------------------------------- conversions --- */
/* Native floats <-> bitslice operands, fused with the transpose (not among
 * the paper's operations, whose inputs are already in the format: the step
 * before and after them for data held as ordinary floats).  Each is one
 * kernel: the values are transposed into slices in the warp and converted by
 * a logic circuit over whole words, like the ops. */
typedef enum { BSFP_FLOAT32 = 0, BSFP_BFLOAT16 = 1, BSFP_FLOAT16 = 2 } bsfp_float_type;

/* bs_out (B planes of stride bsfp_plane_stride(n)) = in[n] converted to
 * format f: the exact value of each IEEE binary32 / bfloat16 / binary16
 * element (type), rounded once in f's mode (RN or RZ, flush to zero with
 * the _FTZ modes); NaN becomes the canonical NaN, overflow follows f's
 * rounding (Inf for RN, the largest finite value for RZ).  in aligned to its
 * element size, bs_out to 16 bytes; padding written as zero.  Errors: as
 * bsfp_pack; an unknown type returns BSFP_ERR_UNSUPPORTED. */
bsfp_status bsfp_from_float(bsfp_format f, int32_t type, const void* in, int64_t n, uint32_t* bs_out,
                            bsfp_stream_t s);
/* out[n] (IEEE binary32) = the elements of bs_in, exactly (every value of a
 * format with E <= 8 and M <= 23 is a binary32 value); NaN becomes the
 * canonical binary32 NaN 0x7FC00000; with an _FTZ mode an element whose
 * exponent field is 0 reads as a zero of its sign.  out aligned to 4 bytes. */
bsfp_status bsfp_to_float(bsfp_format f, const uint32_t* bs_in, int64_t n, float* out, bsfp_stream_t s);

/* ------------------------------------------------------------------ ops --- */
/* out = a + b, element-wise, one rounding (Sec. 4, Table 1 row Add/Sub). */
bsfp_status bsfp_add(bsfp_format f, const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t n,
                     bsfp_stream_t s);
/* out = a - b = a + (-b) (Sec. 4, Table 1 row Add/Sub). */
bsfp_status bsfp_sub(bsfp_format f, const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t n,
                     bsfp_stream_t s);
/* out = a * b, one rounding (Sec. 4, Table 1 row Mul). */
bsfp_status bsfp_mul(bsfp_format f, const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t n,
                     bsfp_stream_t s);
/* out = (a * b) + c with two roundings: the product is rounded to the format,
 * kept in registers, then added and rounded again.  Not in the paper; its
 * register reuse follows the locality advice of Sec. 4. */
bsfp_status bsfp_fma2(bsfp_format f, const uint32_t* a, const uint32_t* b, const uint32_t* c, uint32_t* out,
                      int64_t n, bsfp_stream_t s);
/* out = a / b, one rounding (Sec. 4, Table 1 row Div: restoring division).
 * IEEE-754 cases: NaN for a NaN operand, 0/0 and Inf/Inf; x/0 and Inf/y are
 * infinities and 0/y, x/Inf zeros, each with the XOR of the signs.  Runs as a
 * plain kernel inside batch plans, the no-allocation launch and the server. */
bsfp_status bsfp_div(bsfp_format f, const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t n,
                     bsfp_stream_t s);

/* ----------------------------------------------------- integer vectors --- */
/* Integer bitslice vectors (Sec. 3, Fig. 2): elements are w-bit unsigned
 * integers, 1 <= w <= 32 ("vectors of numbers with 5, 9, or 13 bits"), in the
 * bitslice layout above with B = w planes; the standard representation is
 * the w-bit value right-aligned in a uint8/16/32 container.  add, sub and mul
 * return the low w bits of the exact result (arithmetic modulo 2^w, which is
 * also two's-complement arithmetic); add is the Fig. 2 ripple-carry adder.
 * Same pointer, alignment, n and error conventions as the float ops; a bad w
 * returns BSFP_ERR_FORMAT. */
bsfp_status bsfp_int_pack(int32_t bits, const void* std_in, int64_t n, uint32_t* bs_out, bsfp_stream_t s);
bsfp_status bsfp_int_unpack(int32_t bits, const uint32_t* bs_in, int64_t n, void* std_out, bsfp_stream_t s);
bsfp_status bsfp_int_add(int32_t bits, const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t n,
                         bsfp_stream_t s);
bsfp_status bsfp_int_sub(int32_t bits, const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t n,
                         bsfp_stream_t s);
bsfp_status bsfp_int_mul(int32_t bits, const uint32_t* a, const uint32_t* b, uint32_t* out, int64_t n,
                         bsfp_stream_t s);
/* 3-input logic gates per 32-element word of the integer op (0 add, 1 sub,
 * 2 mul) at width bits; -1 on bad arguments. */
int64_t bsfp_int_gate_count(int32_t bits, int32_t op);

/* -------------------------------------------------------------- batched --- */
/* One element-wise op on one vector: the unit of a batch.  c is used by
 * BSFP_OP_FMA2 only.  Same pointer, alignment and n rules as the single ops. */
typedef struct {
    bsfp_format f;
    int32_t op;          /* bsfp_op */
    const uint32_t* a;
    const uint32_t* b;
    const uint32_t* c;
    uint32_t* out;
    int64_t n;
} bsfp_job;

typedef struct bsfp_batch_plan_st* bsfp_batch_plan;

typedef enum {
    BSFP_BATCH_PERSISTENT = 0, /* one persistent kernel per op class over all tiles */
    BSFP_BATCH_PLAIN = 1,      /* one plain kernel launch per job, captured in the graph */
    BSFP_BATCH_STREAMED = 2,   /* one streamed kernel (BSFP_VARIANT_STREAMED, in its job-list
                                  form) per format, rounding and op class that has one, over the
                                  tiles of all its jobs; the remaining jobs as in PERSISTENT */
    BSFP_BATCH_UNIFIED = 3     /* the RN/RZ add/sub and mul jobs of the persistent formats in one
                                  streamed kernel per op class whatever their format (tiles from
                                  an atomic counter); the remaining jobs as in STREAMED */
} bsfp_batch_mode;

/* Launch shape of a plan.  wpt: words per thread in the persistent kernels
 * (1 or 2; 0 = 2).  blocks_per_sm: resident CTAs per SM for them (0 = the
 * occupancy maximum). */
typedef struct {
    int32_t mode;          /* bsfp_batch_mode */
    int32_t wpt;
    int32_t blocks_per_sm;
} bsfp_batch_options;

/* Build a plan for njobs independent jobs (not part of the paper: a batched
 * form of the Sec. 4 operations for many vectors of mixed formats).  Jobs
 * whose format is 1/4/3, 1/4/4, 1/5/7, 1/5/10 or 1/8/7 (RN or RZ) go to the
 * persistent kernels (one per op class: add/sub, mul, fma2; tiles handed
 * out by an atomic counter); any other compiled format runs as its plain
 * kernel in the same graph.  In BSFP_BATCH_STREAMED mode the add/sub and mul
 * jobs of those formats, in every rounding mode, go instead to one streamed
 * kernel per (format, rounding, op class), whose blocks take the tiles of
 * all its jobs round-robin.  The RN/RZ groups do so when they hold at least
 * 8 tiles per SM on average (bsfp_set_batch_stream_min_tiles); otherwise
 * they all stay with the persistent kernels.  Flush-to-zero groups, which
 * the persistent kernels do not cover, always stream.  In BSFP_BATCH_UNIFIED
 * mode the RN/RZ add/sub jobs of those five formats go to one streamed
 * kernel and their mul jobs to another, each a single launch that streams
 * the tiles of every format through one shared-memory ring, taking tiles
 * from an atomic counter; the other jobs go as in BSFP_BATCH_STREAMED.  The plan owns a device buffer (job descriptors, the tile-to-
 * job map and the counters, allocated here) and a CUDA graph capturing
 * counter reset + kernels; it keeps the job pointers, which must stay valid
 * while the plan is run.  opt may be NULL.  Validation errors (any job)
 * return before anything is allocated.  Synchronous w.r.t. the host (it
 * uploads the descriptors). */
bsfp_status bsfp_batch_plan_create(const bsfp_job* jobs, int32_t njobs, const bsfp_batch_options* opt,
                                   bsfp_batch_plan* plan_out);
/* Launch the plan's graph on stream s.  Runs of one plan must not overlap on
 * the GPU (they share the tile counters): use one stream per plan. */
bsfp_status bsfp_batch_run(bsfp_batch_plan plan, bsfp_stream_t s);
/* Minimum mean tiles per SM per RN/RZ group for a BSFP_BATCH_STREAMED plan
 * to stream them (default 8; 0 = always).  Applies to plans created
 * afterwards.  BSFP_ERR_SIZE outside [0, 2^20].  Not in the paper. */
bsfp_status bsfp_set_batch_stream_min_tiles(int32_t tiles_per_sm);
/* Kernel launches one run of the plan performs. */
int64_t bsfp_batch_launches(bsfp_batch_plan plan);
/* Release the plan; the caller must make sure no run of it is in flight. */
void bsfp_batch_free(bsfp_batch_plan plan);
/* The comparator: every job as its own plain kernel launch on stream s, no
 * graph, no allocation.  Stops at the first invalid job (jobs before it are
 * already queued). */
bsfp_status bsfp_launch_jobs(const bsfp_job* jobs, int32_t njobs, bsfp_stream_t s);

/* Limits of bsfp_batch_run_noalloc: jobs per call, and tiles per call (one
 * tile = 8,192 elements of one job, rounded up per job, counting only jobs in
 * the persistent formats).  Its fixed scratch is sized from these: about
 * 1.5 MB of device memory per GPU that loads the library. */
#define BSFP_NOALLOC_MAX_JOBS 4096
#define BSFP_NOALLOC_MAX_TILES (1 << 18)

/* The batched launch without any allocation.  The paper has no counterpart;
 * this serves callers that must not allocate device memory themselves: an
 * application whose own pool has reserved the device memory up front, so a
 * cudaMalloc from a library fails or takes memory it has budgeted, and
 * latency-bound loops, where cudaMalloc/cudaFree can synchronise the whole
 * device.  The jobs run exactly as in a persistent plan (same kernels, same
 * results), launched directly on s; jobs outside the persistent formats run as
 * their plain kernels.
 *
 * The scratch a plan would allocate (job descriptors, tile map, counters)
 * lives instead in one fixed array in device memory that every GPU loading
 * the library holds until the process exits; no call allocates or frees
 * anything, on the host or the device.  Every call shares that array and
 * leaves its contents behind; each call rebuilds what it reads and zeroes its
 * counters.  Calls on one stream run one after another; calls that overlap
 * on the GPU (other streams, other host threads) race on the array and give
 * wrong results.  The first call on a device also looks up the array's device
 * address and the kernels' occupancy.  The call is meant to be issued
 * directly on s, not captured into a CUDA graph: a captured call would copy
 * `jobs` again from the caller's host array at every replay (for repeated
 * batches in a graph, use a plan, bsfp_batch_plan_create).
 *
 * jobs is host memory read by an asynchronous copy on s: pageable memory is
 * staged before the call returns; page-locked memory must stay unchanged
 * until s has passed the call (if it changes in between so that the jobs the
 * kernels read differ from the ones validated, the persistent kernels skip
 * all their work and the fault word of bsfp_fault_status becomes 1).  s must
 * be a stream of the current device.  Errors: njobs < 0 or > BSFP_NOALLOC_MAX_JOBS,
 * or more than BSFP_NOALLOC_MAX_TILES tiles, return BSFP_ERR_SIZE; any
 * invalid job returns its bsfp_add/... error.  All checks come before
 * anything is launched. */
bsfp_status bsfp_batch_run_noalloc(const bsfp_job* jobs, int32_t njobs, bsfp_stream_t s);

/* ----------------------------------------------------- host-to-host path --- */
/* Vectors in host memory, results to host memory: standard form in, the ops
 * of Sec. 4 on the GPU, standard form out (not part of the paper: the
 * transfer pipeline around its operations).  The vectors are cut into chunks
 * that rotate over `depth` streams, each chunk copied to the device, packed,
 * run through every requested op, unpacked and copied back, so that the
 * copies in both directions overlap the kernels of other chunks; the inputs
 * cross the host link once for all the ops.  Results are identical to packing
 * the whole vectors and calling the ops once.
 *
 * The pipeline owns its streams and its device buffers (about
 * 7 + nops buffers of one chunk per stream, allocated on first use and grown
 * for wider formats or more ops).  One pipeline must not be run by two host
 * threads at once. */
typedef struct bsfp_pipeline_st* bsfp_pipeline;

#define BSFP_PIPE_MAX_OPS 4

/* chunk: elements per chunk, a multiple of 1024 in [1024, 2^30] (0 = 2^24);
 * depth: streams, 1..16 (0 = 4).  Created on the current device. */
bsfp_status bsfp_pipeline_create(int64_t chunk, int32_t depth, bsfp_pipeline* out);
/* outs[q][i] = ops[q](a[i], b[i] [, c[i]]) for i < n, q < nops (1..4; c is
 * read only when some op is BSFP_OP_FMA2).  a, b, c, outs[q]: standard
 * arrays (containers of bsfp_container_bytes(f)) in host memory; page-locked
 * memory lets the copies run asynchronously, pageable memory works but its
 * copies are staged by the CUDA driver and overlap less.  Blocks until every
 * result is in host memory.  Errors: as the single ops, before any copy;
 * CUDA failures BSFP_ERR_CUDA. */
bsfp_status bsfp_pipeline_run(bsfp_pipeline p, bsfp_format f, int32_t nops, const int32_t* ops, const void* a,
                              const void* b, const void* c, void* const* outs, int64_t n);
/* bsfp_pipeline_run without the final wait: the same checks (argument
 * errors return before anything is enqueued), then every chunk's copies and
 * kernels are enqueued and the call returns.  The chunks continue the
 * rotation over the streams where the previous submission stopped, so
 * several vectors (of any formats) submitted back to back keep both copy
 * directions busy across the boundary instead of draining the pipeline
 * between them.  The host arrays must stay valid and untouched until
 * bsfp_pipeline_wait returns.  A submission that needs larger device
 * buffers than the pipeline holds first waits for the work in flight. */
bsfp_status bsfp_pipeline_submit(bsfp_pipeline p, bsfp_format f, int32_t nops, const int32_t* ops, const void* a,
                                 const void* b, const void* c, void* const* outs, int64_t n);
/* Blocks until every result of the submissions so far is in host memory.
 * Returns the first failure among those submissions that had started
 * enqueueing work (BSFP_ERR_CUDA for a failed copy or launch), else BSFP_OK,
 * and clears it; BSFP_ERR_NULL for a NULL pipeline. */
bsfp_status bsfp_pipeline_wait(bsfp_pipeline p);
void bsfp_pipeline_free(bsfp_pipeline p);

/* -------------------------------------------------------------- serving --- */
/* A request server for element-wise ops on device-resident bitslice operands
 * (not part of the paper: a serving form of the Sec. 4 operations).  Requests
 * of any compiled format, op and length are submitted from any host thread;
 * a worker thread of the server admits them in arrival order while its
 * result memory and its in-flight slots allow, groups everything admitted at
 * once into a micro-batch and runs it as the persistent batched kernels on
 * one of several streams, so micro-batches admitted while others are still
 * on the GPU run alongside them (continuous batching).  Results stay on the
 * device until released, so they can be operands of later requests.
 *
 * Memory.  The server allocates, at creation, one device arena of
 * budget_bytes for results and small per-slot descriptor buffers; nothing is
 * allocated per request.  A request whose out is NULL gets its result planes
 * (bsfp_bitslice_bytes of its format and n, rounded up to 256 bytes; none
 * when n == 0) from the arena at admission; a request is admitted only when that fits, strictly in
 * arrival order (a request that does not fit waits, and so do those behind
 * it).  A request with its own out uses no arena memory.  The operands are
 * the caller's and must stay valid until the request completes. */
typedef struct bsfp_server_st* bsfp_server;

typedef struct {
    int64_t budget_bytes;    /* result arena, bytes (> 0) */
    int32_t slots;           /* micro-batches in flight at once, 1..16 (0 = 4) */
    int32_t max_batch_jobs;  /* requests per micro-batch, 1..4096 (0 = 1024) */
    int32_t max_batch_tiles; /* tiles of 8,192 elements (4,096 with wpt 1) per micro-batch, 128..2^20
                                (0 = 2^18) */
    int32_t wpt;             /* words per thread of the persistent kernels, 1 or 2 (0 = 2) */
    /* Admission.  While fewer than eager_slots micro-batches are in flight a
     * free slot takes the pending requests at once (latency first).  With
     * eager_slots or more in flight the GPU is already busy, so a free slot
     * waits until min_batch_tiles tiles are pending or the oldest pending
     * request has waited batch_wait_us, and then takes everything that fits
     * (throughput first: fewer, larger micro-batches). */
    int32_t eager_slots;     /* 1..slots (0 = slots: every free slot admits at once) */
    int32_t min_batch_tiles; /* 1..2^20 (0 = 2 x the SM count) */
    int32_t batch_wait_us;   /* 0..10^6 (0 = 20; -1 = admit without waiting) */
    int32_t reserved;        /* 0 */
} bsfp_server_options;

/* One finished request.  Times are host steady-clock nanoseconds: submission,
 * admission (its micro-batch launched) and completion (the worker saw the
 * micro-batch's event complete). */
typedef struct {
    int64_t id;
    int32_t status;      /* BSFP_OK, or the error that failed it */
    int32_t pad;
    uint32_t* out;       /* the result planes */
    int64_t n;
    int64_t t_submit_ns;
    int64_t t_admit_ns;
    int64_t t_done_ns;
} bsfp_completion;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t pending;          /* submitted, not yet admitted */
    int64_t inflight_batches; /* micro-batches on the GPU now */
    int64_t batches;          /* micro-batches launched so far */
    int64_t peak_inflight_batches;
    int64_t arena_bytes_in_use, arena_peak_bytes, budget_bytes;
    int64_t launches;         /* kernel launches so far */
} bsfp_server_stats;

/* Create a server on the current device (opt may be NULL only for defaults
 * with a 1 GiB budget).  Errors: bad options BSFP_ERR_SIZE; allocation or
 * stream creation failures BSFP_ERR_CUDA (nothing is left allocated). */
bsfp_status bsfp_server_create(const bsfp_server_options* opt, bsfp_server* out);
/* Submit one request.  job->out may be NULL (result from the arena).  The job
 * is validated here (same errors as bsfp_add etc.); a result larger than the
 * whole budget returns BSFP_ERR_BUDGET.  *id_out receives the request id
 * (increasing from 1).  Thread-safe; never blocks on the GPU. */
bsfp_status bsfp_server_submit(bsfp_server srv, const bsfp_job* job, int64_t* id_out);
/* Submit n requests at once (the same as n bsfp_server_submit calls in
 * order, under one lock): every job is validated first; if one fails, its
 * error is returned, *bad_index (if not NULL) gets its index and no job is
 * submitted.  ids_out (n entries, may be NULL) receives the ids.  Cheaper
 * per request than single submissions when requests arrive in bursts.
 * n == 0 does nothing; n < 0 returns BSFP_ERR_SIZE. */
bsfp_status bsfp_server_submit_n(bsfp_server srv, const bsfp_job* jobs, int32_t n, int64_t* ids_out,
                                 int32_t* bad_index);
/* Move up to max finished requests into done[] (oldest first); returns how
 * many.  Thread-safe. */
int32_t bsfp_server_poll(bsfp_server srv, bsfp_completion* done, int32_t max);
/* Give back a finished request's arena memory (its out is invalid after
 * this).  BSFP_ERR_SIZE if id is not a finished, unreleased request. */
bsfp_status bsfp_server_release(bsfp_server srv, int64_t id);
/* Wait until nothing is pending or in flight, at most timeout_ms
 * (BSFP_ERR_TIMEOUT when it runs out). */
bsfp_status bsfp_server_drain(bsfp_server srv, int64_t timeout_ms);
bsfp_status bsfp_server_get_stats(bsfp_server srv, bsfp_server_stats* st);
/* Stop the worker after the in-flight work ends and free everything; pending
 * requests are dropped, results become invalid. */
void bsfp_server_destroy(bsfp_server srv);

/* ----------------------------------------------------------- autotuning --- */
/* Time every compiled launch shape of (f, op) -- words per thread x resident
 * blocks per SM -- on scratch operands of 2^28 elements that this call
 * allocates and frees (zeros; the circuits' timing does not depend on the
 * values), keep the fastest for this process, and, if cache_path is not
 * NULL, record it in that text cache (one line per format, rounding and op;
 * an earlier line for the same key is replaced).  Synchronous; uses a stream
 * of its own.  The north-star's autotuner; not part of the paper.  Errors:
 * bad format or op as the ops; CUDA failures BSFP_ERR_CUDA; an unwritable
 * cache BSFP_ERR_NULL (the shape is still applied). */
bsfp_status bsfp_autotune(bsfp_format f, int32_t op, const char* cache_path);
/* Apply every shape recorded in a cache written by bsfp_autotune; returns how
 * many were applied, or -1 if the file cannot be read. */
int32_t bsfp_autotune_load(const char* cache_path);

/* ---------------------------------------------------------- diagnostics --- */
const char* bsfp_status_str(int32_t status);
/* The cudaError_t of the last BSFP_ERR_CUDA on this thread (0 if none). */
int32_t bsfp_last_cuda_error(void);
/* Number of 3-input logic gates per 32-element word of the circuit for
 * (format, op) as built (inversions folded, identical gates shared, dead
 * gates dropped): the work term of the logic roofline.  Table 1 of Sec. 4
 * gives only the asymptotic classes.  -1 on a bad argument. */
int64_t bsfp_gate_count(bsfp_format f, int32_t op);
/* Kernel variants of an element-wise op.  1, 2 and 4 are the grid-stride
 * kernel with that many words per thread.  BSFP_VARIANT_STREAMED is the
 * streamed kernel: one block per SM; a producer warp brings the operands'
 * planes into a shared-memory ring with TMA bulk copies (cp.async.bulk,
 * completed on mbarriers) while consumer warps run the circuit from it.  It
 * is compiled for add/sub and mul of 1/4/3, 1/4/4, 1/5/7, 1/5/10 and 1/8/7
 * in every rounding mode (and fma2 and division of those of them that lie in
 * the bands below); and for every other format under RN and RZ: mul of 12 to
 * 24 planes, fma2 of 10 to 19 planes with at least 4 fraction bits, and
 * division of 8 to 24 planes with at least 3 fraction bits, where it is the
 * default variant (the autotuner's choice instead for mul above 20 planes
 * and division with 3 fraction bits).  bsfp_variants_compiled tells which.
 * Results are identical in every variant; only the speed differs.  (Not a
 * construct of the paper, whose kernels are CPU loops; Sec. 4 leaves the
 * memory schedule to the implementation.) */
#define BSFP_VARIANT_STREAMED 8
/* Variant the op kernel will use for (format, op): 1, 2, 4 or
 * BSFP_VARIANT_STREAMED; -1 on a bad argument, 0 if the format is not
 * compiled. */
int32_t bsfp_variant(bsfp_format f, int32_t op);
/* Bit mask of the variants compiled for (format, op): bit 0 = 1, bit 1 = 2,
 * bit 2 = 4, bit 3 = BSFP_VARIANT_STREAMED. */
int32_t bsfp_variants_compiled(bsfp_format f, int32_t op);
/* Override the launch shape for (format, op): wpt in {1, 2, 4,
 * BSFP_VARIANT_STREAMED} (must be compiled; 0 restores the default) and
 * blocks_per_sm (0 = occupancy maximum, larger values are capped at it;
 * ignored by the streamed kernel, which runs one block per SM).  A
 * grid-stride shape (or 0) also becomes the fallback that the streamed
 * variant gives way to for calls too small for it (bsfp_set_stream_min_tiles);
 * setting BSFP_VARIANT_STREAMED keeps the fallback.  sub shares add's shape.
 * Used by the autotuner; returns BSFP_ERR_UNSUPPORTED for an uncompiled
 * variant.  Not synchronised with launches already queued: it affects later
 * calls. */
bsfp_status bsfp_set_variant(bsfp_format f, int32_t op, int32_t wpt, int32_t blocks_per_sm);
/* The variant a call of (format, op) on n elements launches: the one
 * bsfp_variant reports, except that the streamed variant gives way to the
 * fallback grid-stride shape (bsfp_set_variant) when the call has fewer than
 * tiles_per_sm x SMs tiles of the streamed kernel (its ring would never
 * fill).  -1 on a bad argument, 0 if the format is not compiled.  Needs the
 * device only for its SM count. */
int32_t bsfp_variant_for(bsfp_format f, int32_t op, int64_t n);
/* Shape of the streamed kernel of (format, op): *tile_words = word columns
 * per tile (a tile takes one ring stage), *stages = ring stages per block
 * (one block per SM).  BSFP_ERR_UNSUPPORTED if (format, op) has no streamed
 * kernel; BSFP_ERR_NULL for a NULL output.  No device is needed. */
bsfp_status bsfp_stream_shape(bsfp_format f, int32_t op, int32_t* tile_words, int32_t* stages);
/* Self-test of the streamed kernel's bounded waits: runs (format, op) on a,
 * b -> out (n elements) with the streamed kernel, but issues no copies for
 * tile withhold_tile (0 <= tile < number of tiles; -1 withholds none), and
 * bounds every wait at wait_cycles SM cycles (2^16 .. 2^34).  The waits on
 * the withheld tile run out, the block stops after letting its other copies
 * land, and the fault word (bsfp_fault_status) becomes 1; the output of the
 * blocks that stopped is incomplete, the device stays usable.  For tests of
 * the failure path; no counterpart in the paper.  Covers add, sub and mul:
 * BSFP_ERR_UNSUPPORTED for another op or if (format, op) has no streamed
 * kernel; BSFP_ERR_SIZE for an out-of-range tile or bound. */
bsfp_status bsfp_stream_selftest(bsfp_format f, int32_t op, const uint32_t* a, const uint32_t* b, uint32_t* out,
                                 int64_t n, int64_t withhold_tile, int64_t wait_cycles, bsfp_stream_t s);
/* Minimum tiles per SM for the streamed variant (default 2; 0 = always take
 * it when selected).  Process-wide; BSFP_ERR_SIZE outside [0, 1024]. */
bsfp_status bsfp_set_stream_min_tiles(int32_t tiles_per_sm);
/* Kernel launches this library has issued on this process so far. */
int64_t bsfp_launch_count(void);
/* Fault word of the current device: 0 if no kernel has reported a fault,
 * 1 if a streamed kernel gave up a wait on its copy pipeline (each wait is
 * bounded at 2^32 SM clock cycles, about two seconds; the kernel then stops,
 * lets its copies in flight land and returns, leaving its output
 * incomplete).  Synchronises the device first; clear != 0 resets the word.
 * -1 if the word cannot be read (see bsfp_last_cuda_error).  No counterpart
 * in the paper. */
int32_t bsfp_fault_status(int32_t clear);

#ifdef __cplusplus
}
#endif

#endif /* BSFP_H */
