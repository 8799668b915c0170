/*
 * pipeline.cu -- host arrays in, host arrays out: the whole path of Sec. 4
 * (standard form -> bitslice, ops, bitslice -> standard form) for vectors
 * that live in host memory (bsfp_pipeline_* in bsfp.h).
 *
 * The vectors are cut into chunks of `chunk` elements.  Chunk k goes to slot
 * k mod depth; each slot owns a stream and device buffers for one chunk, and
 * on its stream it runs: copy the chunk of every input to the device, pack
 * each, then for every requested op the op kernel, unpack, and copy the
 * result chunk back.  Slots run concurrently, so the host-to-device copies of
 * one chunk, the kernels of another and the device-to-host copies of a third
 * overlap (the copy engines work in both directions at once), and the
 * inputs cross the host link once however many ops use them.  A slot's
 * buffers are reused by chunk k + depth on the same stream, which orders the
 * reuse after the earlier chunk's copies.
 *
 * Each chunk is an independent vector of its own length, so every chunk uses
 * the ordinary single-vector kernels and results equal those of one call
 * over the whole vector.  The device buffers are sized for the largest
 * format and op count seen so far and grown between runs.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "bsfp.h"
#include "internal.h"

using namespace bsfp;

namespace {

struct PipeSlot {
    cudaStream_t stream = nullptr;
    void* std_in[3] = {nullptr, nullptr, nullptr};
    uint32_t* bs_in[3] = {nullptr, nullptr, nullptr};
    uint32_t* bs_out = nullptr;
    void* std_out[BSFP_PIPE_MAX_OPS] = {};
};

}  // namespace

struct bsfp_pipeline_st {
    int64_t chunk = 0;
    int depth = 0;
    int device = 0;
    int64_t next = 0;         /* slot of the next chunk: the rotation goes on across submissions */
    bsfp_status pending = BSFP_OK;   /* first failure of the submissions since the last wait */
    int64_t cap_std = 0;      /* bytes of each standard buffer */
    int64_t cap_bs = 0;       /* bytes of each bitslice buffer */
    int cap_ops = 0;
    std::vector<PipeSlot> slots;
};

namespace {

void free_buffers(bsfp_pipeline_st* P) {
    for (PipeSlot& s : P->slots) {
        for (int k = 0; k < 3; ++k) {
            if (s.std_in[k]) cudaFree(s.std_in[k]);
            if (s.bs_in[k]) cudaFree(s.bs_in[k]);
            s.std_in[k] = nullptr;
            s.bs_in[k] = nullptr;
        }
        if (s.bs_out) cudaFree(s.bs_out);
        s.bs_out = nullptr;
        for (int k = 0; k < BSFP_PIPE_MAX_OPS; ++k) {
            if (s.std_out[k]) cudaFree(s.std_out[k]);
            s.std_out[k] = nullptr;
        }
    }
    P->cap_std = P->cap_bs = 0;
    P->cap_ops = 0;
}

/* Make every slot hold buffers of at least std_bytes / bs_bytes for nops. */
cudaError_t ensure_buffers(bsfp_pipeline_st* P, int64_t std_bytes, int64_t bs_bytes, int nops) {
    if (std_bytes <= P->cap_std && bs_bytes <= P->cap_bs && nops <= P->cap_ops) return cudaSuccess;
    for (PipeSlot& s : P->slots) {
        const cudaError_t e = cudaStreamSynchronize(s.stream);
        if (e != cudaSuccess) return e;
    }
    const int64_t sb = std_bytes > P->cap_std ? std_bytes : P->cap_std;
    const int64_t bb = bs_bytes > P->cap_bs ? bs_bytes : P->cap_bs;
    const int no = nops > P->cap_ops ? nops : P->cap_ops;
    free_buffers(P);
    cudaError_t e = cudaSuccess;
    for (PipeSlot& s : P->slots) {
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
            e = cudaMalloc(&s.std_in[k], (size_t)sb);
            if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s.bs_in[k]), (size_t)bb);
        }
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s.bs_out), (size_t)bb);
        for (int k = 0; k < no && e == cudaSuccess; ++k) e = cudaMalloc(&s.std_out[k], (size_t)sb);
    }
    if (e != cudaSuccess) {
        free_buffers(P);
        return e;
    }
    P->cap_std = sb;
    P->cap_bs = bb;
    P->cap_ops = no;
    return cudaSuccess;
}

bsfp_status run_op(int op, bsfp_format f, const uint32_t* a, const uint32_t* b, const uint32_t* c, uint32_t* out,
                   int64_t n, bsfp_stream_t s) {
    switch (op) {
        case BSFP_OP_ADD: return bsfp_add(f, a, b, out, n, s);
        case BSFP_OP_SUB: return bsfp_sub(f, a, b, out, n, s);
        case BSFP_OP_MUL: return bsfp_mul(f, a, b, out, n, s);
        case BSFP_OP_FMA2: return bsfp_fma2(f, a, b, c, out, n, s);
        case BSFP_OP_DIV: return bsfp_div(f, a, b, out, n, s);
    }
    return BSFP_ERR_UNSUPPORTED;
}

}  // namespace

extern "C" {

bsfp_status bsfp_pipeline_create(int64_t chunk, int32_t depth, bsfp_pipeline* out) {
    if (!out) return BSFP_ERR_NULL;
    *out = nullptr;
    if (chunk == 0) chunk = 1 << 24;
    if (depth == 0) depth = 4;
    if (chunk < 1024 || chunk > (1LL << 30) || chunk % 1024 != 0 || depth < 1 || depth > 16) return BSFP_ERR_SIZE;
    bsfp_pipeline_st* P = new bsfp_pipeline_st();
    P->chunk = chunk;
    P->depth = depth;
    cudaError_t e = cudaGetDevice(&P->device);
    P->slots.resize((size_t)depth);
    for (PipeSlot& s : P->slots)
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        for (PipeSlot& s : P->slots)
            if (s.stream) cudaStreamDestroy(s.stream);
        delete P;
        return set_cuda_error(e);
    }
    *out = P;
    return BSFP_OK;
}

bsfp_status bsfp_pipeline_submit(bsfp_pipeline P, bsfp_format f, int32_t nops, const int32_t* ops, const void* a,
                                 const void* b, const void* c, void* const* outs, int64_t n) {
    NvtxRange range("bsfp_pipeline_submit");
    if (!P || !ops || !outs) return BSFP_ERR_NULL;
    if (!format_ok(f)) return BSFP_ERR_FORMAT;
    if (nops < 1 || nops > BSFP_PIPE_MAX_OPS || n < 0 || n > BSFP_MAX_N) return BSFP_ERR_SIZE;
    bool need_c = false;
    for (int k = 0; k < nops; ++k) {
        if (opclass(ops[k]) < 0) return BSFP_ERR_UNSUPPORTED;
        if (!outs[k]) return BSFP_ERR_NULL;
        need_c |= ops[k] == BSFP_OP_FMA2;
    }
    if (n == 0) return BSFP_OK;
    if (!a || !b || (need_c && !c)) return BSFP_ERR_NULL;
    const int cb = bsfp_container_bytes(f);
    const int B = 1 + f.exp_bits + f.man_bits;
    const int64_t chunk = P->chunk < n ? P->chunk : n;
    cudaError_t e = ensure_buffers(P, chunk * cb, (int64_t)B * bsfp_plane_stride(chunk) * 4, nops);
    if (e != cudaSuccess) return set_cuda_error(e);

    const int nin = need_c ? 3 : 2;
    const unsigned char* in[3] = {static_cast<const unsigned char*>(a), static_cast<const unsigned char*>(b),
                                  static_cast<const unsigned char*>(c)};
    bsfp_status st = BSFP_OK;
    for (int64_t e0 = 0; e0 < n && st == BSFP_OK; e0 += chunk) {
        PipeSlot& s = P->slots[(size_t)(P->next % P->depth)];
        P->next = (P->next + 1) % P->depth;
        const int64_t m = (n - e0) < chunk ? (n - e0) : chunk;
        const bsfp_stream_t ss = reinterpret_cast<bsfp_stream_t>(s.stream);
        for (int i = 0; i < nin && st == BSFP_OK; ++i) {
            e = cudaMemcpyAsync(s.std_in[i], in[i] + e0 * cb, (size_t)(m * cb), cudaMemcpyHostToDevice, s.stream);
            if (e != cudaSuccess) st = set_cuda_error(e);
            if (st == BSFP_OK) st = bsfp_pack(f, s.std_in[i], m, s.bs_in[i], ss);
        }
        for (int q = 0; q < nops && st == BSFP_OK; ++q) {
            st = run_op(ops[q], f, s.bs_in[0], s.bs_in[1], s.bs_in[2], s.bs_out, m, ss);
            if (st == BSFP_OK) st = bsfp_unpack(f, s.bs_out, m, s.std_out[q], ss);
            if (st == BSFP_OK) {
                e = cudaMemcpyAsync(static_cast<unsigned char*>(outs[q]) + e0 * cb, s.std_out[q], (size_t)(m * cb),
                                    cudaMemcpyDeviceToHost, s.stream);
                if (e != cudaSuccess) st = set_cuda_error(e);
            }
        }
    }
    if (st != BSFP_OK && P->pending == BSFP_OK) P->pending = st;
    return st;
}

bsfp_status bsfp_pipeline_wait(bsfp_pipeline P) {
    if (!P) return BSFP_ERR_NULL;
    bsfp_status st = P->pending;
    P->pending = BSFP_OK;
    for (PipeSlot& s : P->slots) {
        const cudaError_t e = cudaStreamSynchronize(s.stream);
        if (e != cudaSuccess && st == BSFP_OK) st = set_cuda_error(e);
    }
    return st;
}

bsfp_status bsfp_pipeline_run(bsfp_pipeline P, bsfp_format f, int32_t nops, const int32_t* ops, const void* a,
                              const void* b, const void* c, void* const* outs, int64_t n) {
    NvtxRange range("bsfp_pipeline_run");
    if (!P) return BSFP_ERR_NULL;
    /* the call returns when every result chunk is in host memory */
    const bsfp_status st = bsfp_pipeline_submit(P, f, nops, ops, a, b, c, outs, n);
    const bsfp_status w = bsfp_pipeline_wait(P);
    return st != BSFP_OK ? st : w;
}

void bsfp_pipeline_free(bsfp_pipeline P) {
    if (!P) return;
    for (PipeSlot& s : P->slots)
        if (s.stream) cudaStreamSynchronize(s.stream);
    free_buffers(P);
    for (PipeSlot& s : P->slots)
        if (s.stream) cudaStreamDestroy(s.stream);
    delete P;
}

}  // extern "C"
