/*
 * c_consumer.c -- a plain C11 user of the public headers: includes bsfp.h
 * and bsfp_bench.h with no CUDA header on the include path, links against
 * libbsfp.so and calls the host-side part of the ABI (sizes, status strings
 * and the argument validation of an op, which returns before any launch, so
 * no GPU is needed).  Prints "ok" and exits 0 when every check holds.
 */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "bsfp.h"
#include "bsfp_bench.h"

static int failures = 0;

static void check(int cond, const char* what) {
    if (!cond) {
        printf("FAIL: %s\n", what);
        ++failures;
    }
}

int main(void) {
    const bsfp_format f157 = {5, 7, BSFP_RN};
    const bsfp_format f143 = {4, 3, BSFP_RZ};
    const bsfp_format bad = {9, 7, BSFP_RN};
    _Alignas(16) uint32_t words[8] = {0};
    bsfp_stream_t s = NULL;

    check(bsfp_plane_stride(0) == 0, "stride(0)");
    check(bsfp_plane_stride(1) == 32, "stride(1)");
    check(bsfp_plane_stride(1025) == 64, "stride(1025)");
    check(bsfp_plane_stride(((int64_t)1) << 28) == ((int64_t)1) << 23, "stride(2^28)");
    check(bsfp_plane_stride(-1) == -1, "stride(-1)");
    check(bsfp_bitslice_bytes(f157, ((int64_t)1) << 28) == 13 * (((int64_t)1) << 23) * 4, "bytes 1/5/7");
    check(bsfp_bitslice_bytes(bad, 10) == -1, "bytes of a bad format");
    check(bsfp_container_bytes(f143) == 1 && bsfp_container_bytes(f157) == 2, "container bytes");

    check(strlen(bsfp_status_str(BSFP_OK)) > 0, "status string of BSFP_OK");
    check(strcmp(bsfp_status_str(BSFP_OK), bsfp_status_str(BSFP_ERR_FORMAT)) != 0, "distinct status strings");

    /* validation paths of an op: each returns before anything is launched */
    check(bsfp_add(bad, words, words, words, 32, s) == BSFP_ERR_FORMAT, "add: bad format");
    check(bsfp_add(f157, NULL, words, words, 32, s) == BSFP_ERR_NULL, "add: NULL operand");
    check(bsfp_add(f157, words, words, words, -1, s) == BSFP_ERR_SIZE, "add: negative n");
    check(bsfp_mul(f143, (const uint32_t*)((uintptr_t)words + 4), words, words, 32, s) == BSFP_ERR_ALIGN,
          "mul: misaligned operand");
    check(bsfp_add(f157, NULL, NULL, NULL, 0, s) == BSFP_OK, "add: n == 0 is a no-op");

    if (failures) return 1;
    printf("ok\n");
    return 0;
}
