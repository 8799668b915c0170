/*
 * batch_inst.cu -- instantiates the persistent batched kernels of one op
 * class (compiled once per class with -DBSFP_BATCH_OPC=0|1|2, so the three
 * classes build in parallel), for 1 and 2 words per thread.
 */
#include "batch.cuh"

#ifndef BSFP_BATCH_OPC
#error "compile with -DBSFP_BATCH_OPC=<op class>"
#endif

namespace bsfp {

template <int WPT>
static cudaError_t launch_one(const JobDesc* jobs, const int32_t* tile_job, int64_t ntiles,
                              unsigned long long* counter, int grid, cudaStream_t s) {
    batch_kernel<BSFP_BATCH_OPC, WPT><<<grid, 128, 0, s>>>(jobs, tile_job, ntiles, counter);
    return cudaGetLastError();
}

#define BSFP_BCAT2(a, b) a##b
#define BSFP_BCAT(a, b) BSFP_BCAT2(a, b)

batch_launch_fn BSFP_BCAT(batch_launcher_opc, BSFP_BATCH_OPC)(int wpt) {
    return wpt == 1 ? launch_one<1> : (wpt == 2 ? launch_one<2> : nullptr);
}

const void* BSFP_BCAT(batch_kernel_ptr_opc, BSFP_BATCH_OPC)(int wpt) {
    return wpt == 1 ? (const void*)batch_kernel<BSFP_BATCH_OPC, 1>
                    : (wpt == 2 ? (const void*)batch_kernel<BSFP_BATCH_OPC, 2> : nullptr);
}

}  // namespace bsfp
