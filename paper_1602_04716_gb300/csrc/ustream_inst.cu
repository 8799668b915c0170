/*
 * ustream_inst.cu -- instantiates the unified streamed batch kernel
 * (ustream.cuh) for one op class, compiled once per class with
 * -DBSFP_USTREAM_OPC=0 (add/sub) or 1 (mul).  Shape: 12 consumer warps and
 * 2 ring slots of 96 KB, the best of four measured on the 4,096-vector
 * workload (12 x 2 x 96 KB: 1.69 ms; 14 x 2 x 96 KB: 1.97 ms; 11 x 3 x 72 KB:
 * 2.19 ms; 8 x 3 x 72 KB: 2.08 ms).
 */
#include "ustream.cuh"

#ifndef BSFP_USTREAM_OPC
#error "compile with -DBSFP_USTREAM_OPC=<0 or 1>"
#endif

namespace bsfp {

#define BSFP_UCAT2(a, b) a##b
#define BSFP_UCAT(a, b) BSFP_UCAT2(a, b)

UStreamEntry BSFP_UCAT(ustream_entry_opc, BSFP_USTREAM_OPC)() {
    return make_ustream_entry<BSFP_USTREAM_OPC, 12, 2, 24576>();
}

}  // namespace bsfp
