/*
 * serve.cu -- the request server of bsfp.h (continuous batching of
 * element-wise ops on device-resident bitslice operands) and its open-loop
 * trace replay (bsfp_bench.h).
 *
 * Structure.  Client threads submit requests into a FIFO under the server's
 * mutex (one at a time, or in bursts with bsfp_server_submit_n, which takes
 * the lock once).  One worker thread loops: it retires finished micro-batches
 * (a CUDA event per slot), then, for every free slot, admits requests from
 * the head of the FIFO while the slot's descriptor capacity and the result
 * arena allow -- at once while few micro-batches are in flight, otherwise
 * only once enough tiles are pending or the oldest request has waited a
 * tick, so that a busy GPU gets fewer, larger micro-batches -- and launches
 * them as one micro-batch on the slot's stream: one
 * host-to-device copy of the descriptors, the tile map and zeroed tile
 * counters from the slot's page-locked staging buffer, then one persistent
 * batched kernel per op class present (the kernels of batch.cuh), then a
 * plain kernel for any job outside the persistent formats, then the slot's
 * event.  Slots have their own streams, so a micro-batch admitted while
 * others are running overlaps them on the device.
 *
 * Result memory comes from one device arena allocated at creation: a
 * first-fit free list (offset -> size, adjacent free blocks merged) of
 * 256-byte-aligned blocks.  Admission is strictly in arrival order; the head
 * request waits until its result fits.
 *
 * Every wait here is on the host and bounded where a caller can ask for a
 * bound (drain, replay); the kernels contain no waits.
 */
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.cuh"
#include "bsfp.h"
#include "bsfp_bench.h"
#include "internal.h"

using namespace bsfp;

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

constexpr int64_t ARENA_ALIGN = 256;
int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

/* First-fit allocator over [0, size) with coalescing of free neighbours. */
class Arena {
public:
    explicit Arena(int64_t size) : size_(size) {
        if (size > 0) free_[0] = size;
    }
    bool alloc(int64_t bytes, int64_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const int64_t rest = it->second - bytes;
                const int64_t at = it->first + bytes;
                free_.erase(it);
                if (rest > 0) free_[at] = rest;
                used_ += bytes;
                if (used_ > peak_) peak_ = used_;
                return true;
            }
        }
        return false;
    }
    void release(int64_t off, int64_t bytes) {
        used_ -= bytes;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + bytes == nx->first) {
            bytes += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                pv->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    int64_t used() const { return used_; }
    int64_t peak() const { return peak_; }
    int64_t size() const { return size_; }

private:
    int64_t size_;
    std::map<int64_t, int64_t> free_;
    int64_t used_ = 0, peak_ = 0;
};

struct Request {
    int64_t id;
    bsfp_job job;
    bool own_out;        /* result from the arena */
    int64_t out_off, out_bytes;
    int kind, opc;       /* kind < 0: plain kernel */
    int64_t S, tiles;
    int64_t t_submit, t_admit, t_done;
    int32_t status;
    bool polled;         /* handed out by bsfp_server_poll */
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    unsigned char* host = nullptr;   /* page-locked staging */
    unsigned char* dev = nullptr;    /* counters | descriptors | tile map */
    std::vector<int64_t> reqs;
    bool busy = false;
};

}  // namespace

struct bsfp_server_st {
    bsfp_server_options opt;
    int device = 0;
    unsigned char* arena_base = nullptr;
    Arena arena{0};
    std::vector<Slot> slots;
    size_t off_desc = 0, off_map = 0, slot_bytes = 0;
    int grid_cap[OPC_COUNT] = {0, 0, 0};

    std::mutex mu;
    std::condition_variable cv_work;   /* worker: new submissions / stop */
    std::condition_variable cv_idle;   /* drain: pending and in-flight changed */
    std::deque<int64_t> pending;
    int64_t pending_tiles = 0;         /* tiles of the pending requests */
    std::unordered_map<int64_t, Request> reqs;
    std::deque<int64_t> finished;      /* completed, not yet polled */
    int64_t next_id = 1;
    int64_t submitted = 0, completed = 0, failed = 0, batches = 0, launches = 0, peak_inflight = 0;
    int inflight = 0;
    uint64_t wake_gen = 0;   /* advanced by submit, release and stop */
    bool stop = false;
    std::thread worker;

    void run();
    void retire_locked(Slot& s, bool ok, cudaError_t err);
    bool admit_locked(Slot& s);
    bool may_admit_locked(int64_t now) const;
    bsfp_status make_request(const bsfp_job& job, Request* r) const;
};

namespace {

void destroy_resources(bsfp_server_st* S) {
    for (Slot& s : S->slots) {
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.host) cudaFreeHost(s.host);
        if (s.dev) cudaFree(s.dev);
    }
    if (S->arena_base) cudaFree(S->arena_base);
}

}  // namespace

void bsfp_server_st::retire_locked(Slot& s, bool ok, cudaError_t err) {
    const int64_t t = now_ns();
    for (int64_t id : s.reqs) {
        auto it = reqs.find(id);
        if (it == reqs.end()) continue;
        Request& r = it->second;
        r.t_done = t;
        if (ok) {
            completed += 1;
        } else {
            r.status = set_cuda_error(err);
            failed += 1;
        }
        finished.push_back(id);
    }
    s.reqs.clear();
    s.busy = false;
    inflight -= 1;
}

/* Admit from the head of the FIFO into slot s and launch; false if nothing
 * could be admitted. */
bool bsfp_server_st::admit_locked(Slot& s) {
    NvtxRange range("bsfp_server micro-batch");
    int32_t njob_c[OPC_COUNT] = {0, 0, 0};
    int64_t ntile_c[OPC_COUNT] = {0, 0, 0};
    int64_t tiles = 0;
    std::vector<int64_t>& take = s.reqs;
    take.clear();
    while (!pending.empty() && (int32_t)take.size() < opt.max_batch_jobs) {
        Request& r = reqs[pending.front()];
        const bool pers = r.kind >= 0 && r.tiles <= opt.max_batch_tiles;
        if (pers && tiles + r.tiles > opt.max_batch_tiles) break;
        if (r.own_out && r.out_bytes > 0) {   /* n == 0 needs no memory */
            int64_t off = 0;
            if (!arena.alloc(r.out_bytes, &off)) break;
            r.out_off = off;
            r.job.out = reinterpret_cast<uint32_t*>(arena_base + off);
        }
        if (pers) {
            njob_c[r.opc] += 1;
            ntile_c[r.opc] += r.tiles;
            tiles += r.tiles;
        } else {
            r.kind = -1;
        }
        take.push_back(r.id);
        pending_tiles -= r.tiles;
        pending.pop_front();
    }
    if (take.empty()) return false;

    /* staging: zeroed counters | descriptors by class | tile map by class */
    int32_t desc0[OPC_COUNT], map0[OPC_COUNT];
    int32_t d = 0, m = 0;
    for (int g = 0; g < OPC_COUNT; ++g) {
        desc0[g] = d;
        map0[g] = m;
        d += njob_c[g];
        m += (int32_t)ntile_c[g];
    }
    /* the map follows the descriptors this micro-batch uses */
    const size_t map_at = off_desc + (size_t)round_up((int64_t)sizeof(JobDesc) * d, 256);
    memset(s.host, 0, off_desc);
    JobDesc* hdesc = reinterpret_cast<JobDesc*>(s.host + off_desc);
    int32_t* hmap = reinterpret_cast<int32_t*>(s.host + map_at);
    int32_t dfill[OPC_COUNT] = {0, 0, 0};
    int32_t tfill[OPC_COUNT] = {0, 0, 0};
    const int64_t t_admit = now_ns();
    for (int64_t id : take) {
        Request& r = reqs[id];
        r.t_admit = t_admit;
        if (r.kind < 0) continue;
        const int g = r.opc;
        JobDesc jd;
        memset(&jd, 0, sizeof jd);
        jd.a = r.job.a;
        jd.b = r.job.b;
        jd.c = r.job.c;
        jd.out = r.job.out;
        jd.S = r.S;
        jd.nwords = (r.job.n + 31) / 32;
        jd.tile0 = tfill[g];
        jd.tailmask = (r.job.n % 32) ? ((1u << (r.job.n % 32)) - 1u) : ~0u;
        jd.negb = (r.job.op == BSFP_OP_SUB) ? ~0u : 0u;
        jd.kind = r.kind;
        const int32_t local = dfill[g]++;
        hdesc[desc0[g] + local] = jd;
        for (int64_t q = 0; q < r.tiles; ++q) hmap[map0[g] + tfill[g] + q] = local;
        tfill[g] += (int32_t)r.tiles;
    }

    cudaError_t err = cudaSuccess;
    int64_t launched = 0;
    if (tiles > 0) {
        /* one copy: zeroed counters, the descriptors, the tile map */
        const size_t bytes = map_at + sizeof(int32_t) * (size_t)tiles;
        err = cudaMemcpyAsync(s.dev, s.host, bytes, cudaMemcpyHostToDevice, s.stream);
        for (int g = 0; g < OPC_COUNT && err == cudaSuccess; ++g) {
            if (ntile_c[g] == 0) continue;
            const int grid = (int)(ntile_c[g] < grid_cap[g] ? ntile_c[g] : grid_cap[g]);
            err = batch_launcher(g, opt.wpt)(reinterpret_cast<const JobDesc*>(s.dev + off_desc) + desc0[g],
                                             reinterpret_cast<const int32_t*>(s.dev + map_at) + map0[g],
                                             ntile_c[g],
                                             reinterpret_cast<unsigned long long*>(s.dev) + g, grid, s.stream);
            if (err == cudaSuccess) launched += 1;
        }
    }
    bsfp_status st = BSFP_OK;
    for (int64_t id : take) {
        if (err != cudaSuccess || st != BSFP_OK) break;
        Request& r = reqs[id];
        if (r.kind >= 0) continue;
        PreparedOp po;
        st = prepare_binop(r.job.f, r.job.op, r.job.a, r.job.b, r.job.c, r.job.out, r.job.n, &po);
        if (st == BSFP_OK && !po.skip) {
            st = launch_prepared(po, s.stream);
            if (st == BSFP_OK) launched += 1;
        }
    }
    if (err == cudaSuccess && st == BSFP_OK) err = cudaEventRecord(s.done, s.stream);
    count_launches(launched);
    launches += launched;
    batches += 1;
    s.busy = true;
    inflight += 1;
    if (inflight > peak_inflight) peak_inflight = inflight;
    if (err != cudaSuccess || st != BSFP_OK) {
        /* the launch failed: the micro-batch's requests fail at once (the
         * stream is synchronised first so that no kernel still uses them) */
        cudaStreamSynchronize(s.stream);
        retire_locked(s, false, err != cudaSuccess ? err : (cudaError_t)bsfp_last_cuda_error());
    }
    return true;
}

/* Validate one job (as the single ops do, without their launch shape) and
 * fill in what admission needs; no lock is taken. */
bsfp_status bsfp_server_st::make_request(const bsfp_job& job, Request* r) const {
    memset(r, 0, sizeof *r);
    r->job = job;
    r->own_out = job.out == nullptr;
    /* an arena result stands in as an aligned placeholder until admission */
    const uint32_t* out_check = r->own_out ? reinterpret_cast<const uint32_t*>((uintptr_t)ARENA_ALIGN) : job.out;
    int opc = -1;
    const bsfp_status v = validate_binop(job.f, job.op, job.a, job.b, job.c, out_check, job.n, &opc);
    if (v != BSFP_OK) return v;
    r->S = bsfp_plane_stride(job.n);
    r->out_bytes = round_up((int64_t)(1 + job.f.exp_bits + job.f.man_bits) * r->S * 4, ARENA_ALIGN);
    if (r->own_out && r->out_bytes > opt.budget_bytes) return BSFP_ERR_BUDGET;
    r->opc = opc;
    r->kind = (job.n == 0 || opc >= OPC_COUNT) ? -1 : batch_kind(job.f.exp_bits, job.f.man_bits, job.f.rnd);
    const int64_t tile = 128LL * opt.wpt * BATCH_ROUNDS;
    r->tiles = (r->S + tile - 1) / tile;
    r->status = BSFP_OK;
    return BSFP_OK;
}

/* Admission policy (bsfp_server_options): a free slot takes the pending
 * requests at once while fewer than eager_slots micro-batches are in flight;
 * beyond that, only when min_batch_tiles tiles are pending or the head has
 * waited batch_wait_us. */
bool bsfp_server_st::may_admit_locked(int64_t now) const {
    if (pending.empty()) return false;
    if (inflight < opt.eager_slots || opt.batch_wait_us < 0) return true;
    if (pending_tiles >= opt.min_batch_tiles) return true;
    const auto it = reqs.find(pending.front());
    return it == reqs.end() || now - it->second.t_submit >= (int64_t)opt.batch_wait_us * 1000;
}

void bsfp_server_st::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        bool changed = false;
        for (Slot& s : slots) {
            if (!s.busy) continue;
            const cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaErrorNotReady) continue;
            retire_locked(s, q == cudaSuccess, q);
            changed = true;
        }
        if (stop && inflight == 0) break;
        bool blocked = false;   /* the head does not fit the arena */
        if (!stop) {
            for (Slot& s : slots) {
                if (s.busy || pending.empty()) continue;
                if (!may_admit_locked(now_ns())) break;   /* let the batch grow; poll again */
                if (!admit_locked(s)) {
                    blocked = true;
                    break;
                }
                changed = true;
            }
        }
        if (changed) cv_idle.notify_all();
        if (inflight == 0) {
            if (stop) break;
            if (pending.empty() || blocked) {
                /* nothing can move until a submission, a release or stop */
                const uint64_t gen = wake_gen;
                cv_work.wait(lk, [&] { return stop || wake_gen != gen; });
            }
        } else if (!changed) {
            /* work on the GPU: poll again shortly, letting submitters in */
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        }
    }
    cv_idle.notify_all();
}

extern "C" {

bsfp_status bsfp_server_create(const bsfp_server_options* opt, bsfp_server* out) {
    if (!out) return BSFP_ERR_NULL;
    *out = nullptr;
    bsfp_server_options o;
    memset(&o, 0, sizeof o);
    o.budget_bytes = 1LL << 30;
    if (opt) o = *opt;
    if (o.slots == 0) o.slots = 4;
    if (o.max_batch_jobs == 0) o.max_batch_jobs = 1024;
    if (o.max_batch_tiles == 0) o.max_batch_tiles = 1 << 18;
    if (o.wpt == 0) o.wpt = 2;
    if (o.eager_slots == 0) o.eager_slots = o.slots;
    if (o.batch_wait_us == 0) o.batch_wait_us = 20;
    if (o.budget_bytes <= 0 || o.slots < 1 || o.slots > 16 || o.max_batch_jobs < 1 || o.max_batch_jobs > 4096 ||
        o.max_batch_tiles < 128 || o.max_batch_tiles > (1 << 20) || (o.wpt != 1 && o.wpt != 2) ||
        o.eager_slots < 1 || o.eager_slots > o.slots || o.min_batch_tiles < 0 || o.min_batch_tiles > (1 << 20) ||
        o.batch_wait_us < -1 || o.batch_wait_us > 1000000 || o.reserved != 0)
        return BSFP_ERR_SIZE;

    bsfp_server_st* S = new bsfp_server_st();
    S->opt = o;
    cudaError_t err = cudaGetDevice(&S->device);
    S->off_desc = 256;
    S->off_map = S->off_desc + (size_t)round_up((int64_t)sizeof(JobDesc) * o.max_batch_jobs, 256);
    S->slot_bytes = S->off_map + sizeof(int32_t) * (size_t)o.max_batch_tiles;
    if (err == cudaSuccess) err = cudaMalloc(&S->arena_base, (size_t)o.budget_bytes);
    S->arena = Arena(o.budget_bytes);
    S->slots.resize((size_t)o.slots);
    for (Slot& s : S->slots) {
        if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (err == cudaSuccess) err = cudaMallocHost(&s.host, S->slot_bytes);
        if (err == cudaSuccess) err = cudaMalloc(&s.dev, S->slot_bytes);
    }
    for (int g = 0; g < OPC_COUNT && err == cudaSuccess; ++g) {
        int occ = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel_ptr(g, o.wpt), 128, 0);
        S->grid_cap[g] = device_num_sms() * (occ > 0 ? occ : 1);
    }
    if (S->opt.min_batch_tiles == 0) S->opt.min_batch_tiles = 2 * device_num_sms();
    if (err != cudaSuccess) {
        destroy_resources(S);
        delete S;
        return set_cuda_error(err);
    }
    S->worker = std::thread([S] { S->run(); });
    *out = S;
    return BSFP_OK;
}

bsfp_status bsfp_server_submit(bsfp_server S, const bsfp_job* job, int64_t* id_out) {
    if (!S || !job) return BSFP_ERR_NULL;
    return bsfp_server_submit_n(S, job, 1, id_out, nullptr);
}

bsfp_status bsfp_server_submit_n(bsfp_server S, const bsfp_job* jobs, int32_t n, int64_t* ids_out,
                                 int32_t* bad_index) {
    if (!S || (n > 0 && !jobs)) return BSFP_ERR_NULL;
    if (n < 0) return BSFP_ERR_SIZE;
    if (n == 0) return BSFP_OK;
    std::vector<Request> rs((size_t)n);
    for (int32_t i = 0; i < n; ++i) {
        const bsfp_status v = S->make_request(jobs[i], &rs[(size_t)i]);
        if (v != BSFP_OK) {
            if (bad_index) *bad_index = i;
            return v;
        }
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return BSFP_ERR_UNSUPPORTED;
        const int64_t t = now_ns();
        for (int32_t i = 0; i < n; ++i) {
            Request& r = rs[(size_t)i];
            r.id = S->next_id++;
            r.t_submit = t;
            S->pending.push_back(r.id);
            S->pending_tiles += r.tiles;
            if (ids_out) ids_out[i] = r.id;
            S->reqs.emplace(r.id, r);
        }
        S->submitted += n;
        S->wake_gen += 1;
    }
    S->cv_work.notify_one();
    return BSFP_OK;
}

int32_t bsfp_server_poll(bsfp_server S, bsfp_completion* done, int32_t max) {
    if (!S || !done || max <= 0) return 0;
    std::lock_guard<std::mutex> lk(S->mu);
    int32_t k = 0;
    while (k < max && !S->finished.empty()) {
        const int64_t id = S->finished.front();
        S->finished.pop_front();
        Request& r = S->reqs[id];
        r.polled = true;
        bsfp_completion& c = done[k++];
        c.id = id;
        c.status = r.status;
        c.pad = 0;
        c.out = r.job.out;
        c.n = r.job.n;
        c.t_submit_ns = r.t_submit;
        c.t_admit_ns = r.t_admit;
        c.t_done_ns = r.t_done;
        if (!r.own_out) S->reqs.erase(id);   /* nothing left to release */
    }
    return k;
}

bsfp_status bsfp_server_release(bsfp_server S, int64_t id) {
    if (!S) return BSFP_ERR_NULL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end() || it->second.t_done == 0 || !it->second.polled) return BSFP_ERR_SIZE;
    if (it->second.own_out && it->second.out_bytes > 0) S->arena.release(it->second.out_off, it->second.out_bytes);
    S->reqs.erase(it);
    S->wake_gen += 1;
    S->cv_work.notify_one();   /* freed memory may admit the head */
    return BSFP_OK;
}

bsfp_status bsfp_server_drain(bsfp_server S, int64_t timeout_ms) {
    if (!S) return BSFP_ERR_NULL;
    std::unique_lock<std::mutex> lk(S->mu);
    const bool ok = S->cv_idle.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                        [&] { return S->pending.empty() && S->inflight == 0; });
    return ok ? BSFP_OK : BSFP_ERR_TIMEOUT;
}

bsfp_status bsfp_server_get_stats(bsfp_server S, bsfp_server_stats* st) {
    if (!S || !st) return BSFP_ERR_NULL;
    std::lock_guard<std::mutex> lk(S->mu);
    st->submitted = S->submitted;
    st->completed = S->completed;
    st->failed = S->failed;
    st->pending = (int64_t)S->pending.size();
    st->inflight_batches = S->inflight;
    st->batches = S->batches;
    st->peak_inflight_batches = S->peak_inflight;
    st->arena_bytes_in_use = S->arena.used();
    st->arena_peak_bytes = S->arena.peak();
    st->budget_bytes = S->arena.size();
    st->launches = S->launches;
    return BSFP_OK;
}

void bsfp_server_destroy(bsfp_server S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->pending.clear();
        S->wake_gen += 1;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (Slot& s : S->slots)
        if (s.stream) cudaStreamSynchronize(s.stream);
    destroy_resources(S);
    delete S;
}

bsfp_status bsfp_server_replay(bsfp_server S, const bsfp_job* jobs, const int64_t* arrival_ns, int32_t n,
                               int32_t release, bsfp_completion* done, int64_t timeout_ms) {
    if (!S || (n > 0 && (!jobs || !arrival_ns || !done))) return BSFP_ERR_NULL;
    if (n < 0) return BSFP_ERR_SIZE;
    std::unordered_map<int64_t, int32_t> index;
    index.reserve((size_t)n * 2 + 1);
    std::vector<bsfp_completion> buf(256);
    int32_t got = 0;
    const int64_t t0 = now_ns();
    const int64_t deadline = t0 + timeout_ms * 1000000LL;
    auto collect = [&]() {
        const int32_t k = bsfp_server_poll(S, buf.data(), (int32_t)buf.size());
        for (int32_t i = 0; i < k; ++i) {
            const bsfp_completion& c = buf[(size_t)i];
            auto it = index.find(c.id);
            if (it == index.end()) continue;   /* not one of ours */
            done[it->second] = c;
            got += 1;
            if (release && jobs[it->second].out == nullptr) bsfp_server_release(S, c.id);
        }
        return k;
    };
    std::vector<int64_t> ids;
    for (int32_t i = 0; i < n;) {
        /* every request whose arrival time has come, in one submission */
        const int64_t now = now_ns();
        int32_t j = i;
        while (j < n && t0 + arrival_ns[j] <= now) ++j;
        if (j == i) {
            if (collect() == 0) std::this_thread::yield();
            continue;
        }
        ids.resize((size_t)(j - i));
        const bsfp_status st = bsfp_server_submit_n(S, jobs + i, j - i, ids.data(), nullptr);
        if (st != BSFP_OK) return st;
        for (int32_t k = i; k < j; ++k) index[ids[(size_t)(k - i)]] = k;
        i = j;
    }
    while (got < n) {
        if (collect() == 0) {
            if (now_ns() > deadline) return BSFP_ERR_TIMEOUT;
            std::this_thread::yield();
        }
    }
    return BSFP_OK;
}

}  // extern "C"
