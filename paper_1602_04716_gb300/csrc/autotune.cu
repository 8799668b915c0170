/*
 * autotune.cu -- the native autotuner of bsfp.h (bsfp_autotune,
 * bsfp_autotune_load).
 *
 * For one (format, op) it times every compiled launch shape -- words per
 * thread x resident blocks per SM -- with CUDA events on a stream of its
 * own, on scratch operands it allocates (n elements, zeros: the circuits are
 * straight-line code without data-dependent branches, so operand values do
 * not change the timing), keeps the fastest shape for the process and, when
 * given a cache path, records it as one text line
 *     <E> <M> <rounding> <op> <wpt> <blocks_per_sm> <ms>
 * replacing an earlier line for the same (E, M, rounding, op).  Lines
 * starting with '#' are comments; the first names the GPU.
 */
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "bsfp.h"
#include "internal.h"

using namespace bsfp;

namespace {

struct ScratchOps {
    uint32_t* buf[4] = {nullptr, nullptr, nullptr, nullptr};
    ~ScratchOps() {
        for (uint32_t* p : buf)
            if (p) cudaFree(p);
    }
};

float median_ms(std::vector<float> v) {
    std::sort(v.begin(), v.end());
    return v[v.size() / 2];
}

}  // namespace

extern "C" {

bsfp_status bsfp_autotune(bsfp_format f, int32_t op, const char* cache_path) {
    NvtxRange range("bsfp_autotune");
    if (!format_ok(f)) return BSFP_ERR_FORMAT;
    if (opclass(op) < 0) return BSFP_ERR_UNSUPPORTED;
    const int32_t mask = bsfp_variants_compiled(f, op);
    if (mask <= 0) return BSFP_ERR_UNSUPPORTED;
    const int64_t n = (int64_t)1 << 28;   /* the at-scale size: shapes tuned small do not carry over */
    const int64_t bytes = bsfp_bitslice_bytes(f, n);
    ScratchOps ops;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
        e = cudaMalloc(reinterpret_cast<void**>(&ops.buf[k]), (size_t)bytes);
        if (e == cudaSuccess) e = cudaMemset(ops.buf[k], 0, (size_t)bytes);
    }
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int bps_choices[] = {0, 1, 2, 3, 4, 6, 8};
    int best_wpt = 0, best_bps = 0;
    float best = 1e30f;
    bsfp_status st = e == cudaSuccess ? BSFP_OK : set_cuda_error(e);
    for (int wpt = 1; wpt <= BSFP_VARIANT_STREAMED && st == BSFP_OK; wpt <<= 1) {
        if (!(mask & wpt)) continue;
        for (int bps : bps_choices) {
            /* the streamed kernel runs one block per SM: one shape only */
            if (wpt == BSFP_VARIANT_STREAMED && bps != 0) continue;
            st = bsfp_set_variant(f, op, wpt, bps);
            std::vector<float> t;
            for (int r = 0; r < 6 && st == BSFP_OK; ++r) {
                cudaEventRecord(e0, s);
                st = run_op_by_code(f, op, ops.buf[0], ops.buf[1], ops.buf[2], ops.buf[3], n, s);
                cudaEventRecord(e1, s);
                e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) st = set_cuda_error(e);
                float ms = 0.f;
                if (st == BSFP_OK) cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0) t.push_back(ms);   /* the first run is a warm-up */
            }
            if (st != BSFP_OK) break;
            const float m = median_ms(t);
            if (m < best) {
                best = m;
                best_wpt = wpt;
                best_bps = bps;
            }
        }
    }
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (s) cudaStreamDestroy(s);
    if (st != BSFP_OK) {
        bsfp_set_variant(f, op, 0, 0);
        return st;
    }
    /* back to the default first, so that a streamed best keeps the default
     * grid-stride shape as its fallback for calls too small for it (the
     * shapes timed here are the fastest at 2^28 elements, not for small
     * calls) */
    bsfp_set_variant(f, op, 0, 0);
    st = bsfp_set_variant(f, op, best_wpt, best_bps);
    if (st != BSFP_OK || !cache_path) return st;

    /* rewrite the cache with this (E, M, rounding, op) replaced */
    std::vector<std::string> lines;
    if (FILE* in = fopen(cache_path, "r")) {
        char buf[256];
        while (fgets(buf, sizeof buf, in)) {
            int E, M, R, O;
            if (buf[0] != '#' && sscanf(buf, "%d %d %d %d", &E, &M, &R, &O) == 4 && E == f.exp_bits &&
                M == f.man_bits && R == f.rnd && O == op)
                continue;
            if (buf[0] == '#') continue;
            lines.push_back(buf);
        }
        fclose(in);
    }
    char line[128];
    snprintf(line, sizeof line, "%d %d %d %d %d %d %.4f\n", f.exp_bits, f.man_bits, f.rnd, op, best_wpt, best_bps,
             best);
    lines.push_back(line);
    cudaDeviceProp prop;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) snprintf(prop.name, sizeof prop.name, "unknown");
    const std::string tmp = std::string(cache_path) + ".tmp";
    FILE* out = fopen(tmp.c_str(), "w");
    if (!out) return BSFP_ERR_NULL;
    fprintf(out, "# bsfp launch shapes for %s: E M rounding op wpt blocks_per_sm ms\n", prop.name);
    for (const std::string& l : lines) fputs(l.c_str(), out);
    if (fclose(out) != 0 || rename(tmp.c_str(), cache_path) != 0) return BSFP_ERR_NULL;
    return BSFP_OK;
}

int32_t bsfp_autotune_load(const char* cache_path) {
    if (!cache_path) return -1;
    FILE* in = fopen(cache_path, "r");
    if (!in) return -1;
    char buf[256];
    int applied = 0;
    while (fgets(buf, sizeof buf, in)) {
        int E, M, R, O, W, P;
        if (buf[0] == '#' || sscanf(buf, "%d %d %d %d %d %d", &E, &M, &R, &O, &W, &P) != 6) continue;
        bsfp_format f = {E, M, R};
        if (bsfp_set_variant(f, O, W, P) == BSFP_OK) ++applied;
    }
    fclose(in);
    return applied;
}

}  // extern "C"
