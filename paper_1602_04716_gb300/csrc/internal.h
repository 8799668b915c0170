/*
 * internal.h -- declarations shared by the library's host-side translation
 * units (not part of the public ABI).
 */
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include "binop.cuh"
#include "bsfp.h"

namespace bsfp {

/* An NVTX range for the library's coarse phases (batch plans and runs,
 * server micro-batches, pipeline runs, autotuning); free without a tool. */
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

/* A validated element-wise op, ready to launch. */
struct PreparedOp {
    BinopArgs args;
    const BinopEntry* entry;
    int opc;
    int wpt;
    int grid;
    bool skip;   /* n == 0: nothing to launch */
};

bool format_ok(const bsfp_format& f);
bool aligned(const void* p, uintptr_t a);
int opclass(int op);
int device_num_sms();
bsfp_status prepare_binop(const bsfp_format& f, int op, const uint32_t* a, const uint32_t* b, const uint32_t* c,
                          uint32_t* out, int64_t n, PreparedOp* po);
/* The argument checks of prepare_binop alone (no launch shape, no device
 * query, no lock): the same status for the same arguments; *opc_out gets
 * the op class when the format and op are valid. */
bsfp_status validate_binop(const bsfp_format& f, int op, const uint32_t* a, const uint32_t* b, const uint32_t* c,
                           const uint32_t* out, int64_t n, int* opc_out);
bsfp_status launch_prepared(const PreparedOp& po, cudaStream_t s);
void count_launches(int64_t k);
/* Device address of the fault word of the current device (bsfp_fault_status),
 * or NULL if it cannot be looked up. */
int* current_fault_word();
bsfp_status set_cuda_error(cudaError_t e);
/* Launch op (bsfp_op code) on stream s through the public entry points. */
bsfp_status run_op_by_code(const bsfp_format& f, int op, const uint32_t* a, const uint32_t* b, const uint32_t* c,
                           uint32_t* out, int64_t n, cudaStream_t s);

}  // namespace bsfp
