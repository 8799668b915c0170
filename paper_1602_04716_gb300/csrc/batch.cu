/*
 * batch.cu -- host side of the batched launch (bsfp.h): plan building,
 * CUDA-graph capture, runs, and the per-job plain-launch comparator.
 */
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <vector>

#include "batch.cuh"
#include "bsfp.h"
#include "internal.h"
#include "stream.cuh"
#include "ustream.cuh"

namespace bsfp {

batch_launch_fn batch_launcher_opc0(int wpt);
batch_launch_fn batch_launcher_opc1(int wpt);
batch_launch_fn batch_launcher_opc2(int wpt);
const void* batch_kernel_ptr_opc0(int wpt);
const void* batch_kernel_ptr_opc1(int wpt);
const void* batch_kernel_ptr_opc2(int wpt);

batch_launch_fn batch_launcher(int opc, int wpt) {
    switch (opc) {
        case OPC_ADDSUB: return batch_launcher_opc0(wpt);
        case OPC_MUL: return batch_launcher_opc1(wpt);
        case OPC_FMA2: return batch_launcher_opc2(wpt);
    }
    return nullptr;
}

UStreamEntry ustream_entry_opc0();
UStreamEntry ustream_entry_opc1();

UStreamEntry ustream_entry(int opc) {
    return opc == OPC_ADDSUB ? ustream_entry_opc0() : (opc == OPC_MUL ? ustream_entry_opc1() : UStreamEntry());
}

const void* batch_kernel_ptr(int opc, int wpt) {
    switch (opc) {
        case OPC_ADDSUB: return batch_kernel_ptr_opc0(wpt);
        case OPC_MUL: return batch_kernel_ptr_opc1(wpt);
        case OPC_FMA2: return batch_kernel_ptr_opc2(wpt);
    }
    return nullptr;
}

}  // namespace bsfp

using namespace bsfp;

/* The RN/RZ groups of a BSFP_BATCH_STREAMED plan run as streamed kernels only
 * with at least this many tiles per SM per group on average; otherwise they
 * go to the persistent kernels, whose two launches cost less than ramping up
 * and draining a launch per group (measured crossover between 5 and 10). */
static std::atomic<int32_t> g_batch_stream_min_tiles{8};

struct bsfp_batch_plan_st {
    void* dev = nullptr;           /* descriptors | tile maps | counters */
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;
};

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static void plan_destroy(bsfp_batch_plan p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->dev) cudaFree(p->dev);
    delete p;
}

extern "C" {

bsfp_status bsfp_batch_plan_create(const bsfp_job* jobs, int32_t njobs, const bsfp_batch_options* opt,
                                   bsfp_batch_plan* plan_out) {
    NvtxRange range("bsfp_batch_plan_create");
    if (!plan_out) return BSFP_ERR_NULL;
    *plan_out = nullptr;
    if (njobs < 0) return BSFP_ERR_SIZE;
    if (njobs > 0 && !jobs) return BSFP_ERR_NULL;
    bsfp_batch_options o = {BSFP_BATCH_PERSISTENT, 2, 0};
    if (opt) o = *opt;
    if (o.wpt == 0) o.wpt = 2;
    if ((o.mode != BSFP_BATCH_PERSISTENT && o.mode != BSFP_BATCH_PLAIN && o.mode != BSFP_BATCH_STREAMED &&
         o.mode != BSFP_BATCH_UNIFIED) ||
        (o.wpt != 1 && o.wpt != 2) || o.blocks_per_sm < 0 || o.blocks_per_sm > 64)
        return BSFP_ERR_SIZE;

    /* validate every job and sort it into a streamed group (BSFP_BATCH_STREAMED:
     * one per format, rounding and op class with a streamed kernel), a
     * persistent group (one per op class) or the plain list */
    std::vector<PreparedOp> prep((size_t)njobs);
    std::vector<int> group((size_t)njobs, -1);
    struct SGroup {
        const BinopEntry* e;
        int* fault;
        bool persistent_ok;           /* RN/RZ: the persistent kernels cover it */
        int64_t tiles = 0;
        std::vector<int32_t> members; /* job indices */
        std::vector<StreamJob> jobs;
        std::vector<int32_t> tmap;
    };
    std::vector<SGroup> sgroups;
    const bool unified = o.mode == BSFP_BATCH_UNIFIED;
    const bool streamed = o.mode == BSFP_BATCH_STREAMED || unified;
    constexpr int UGROUP = OPC_COUNT + 1;   /* group[i] = UGROUP + op class: a unified kernel */
    for (int32_t i = 0; i < njobs; ++i) {
        const bsfp_job& j = jobs[i];
        PreparedOp& po = prep[(size_t)i];
        const bsfp_status st = prepare_binop(j.f, j.op, j.a, j.b, j.c, j.out, j.n, &po);
        if (st != BSFP_OK) return st;
        if (po.skip) continue;
        if (unified && (po.opc == OPC_ADDSUB || po.opc == OPC_MUL) &&
            batch_kind(j.f.exp_bits, j.f.man_bits, j.f.rnd) >= 0) {
            group[(size_t)i] = UGROUP + po.opc;
            continue;
        }
        if (streamed && (po.opc == OPC_ADDSUB || po.opc == OPC_MUL) &&
            (po.entry->wpt_mask & (unsigned)VARIANT_STREAMED) && po.entry->stream_batch_launch) {
            size_t gi = 0;
            while (gi < sgroups.size() && sgroups[gi].e != po.entry) ++gi;
            if (gi == sgroups.size())
                sgroups.push_back(SGroup{po.entry, po.args.fault,
                                         batch_kind(j.f.exp_bits, j.f.man_bits, j.f.rnd) >= 0});
            sgroups[gi].members.push_back(i);
            sgroups[gi].tiles += (po.args.S + po.entry->stream_tw - 1) / po.entry->stream_tw;
            group[(size_t)i] = OPC_COUNT;   /* handled by a streamed group */
            continue;
        }
        if (o.mode != BSFP_BATCH_PLAIN && po.opc < OPC_COUNT && batch_kind(j.f.exp_bits, j.f.man_bits, j.f.rnd) >= 0)
            group[(size_t)i] = po.opc;
    }
    /* one choice for the whole plan: the RN/RZ groups stream when they have
     * at least min tiles per SM on average, else they all go to the
     * persistent kernels (streaming only some of them adds launches whose
     * ramp-up and drain the rest does not hide); the other groups stream */
    {
        const int64_t min_tiles =
            (int64_t)g_batch_stream_min_tiles.load(std::memory_order_relaxed) * device_num_sms();
        int64_t tiles = 0, ngroups = 0;
        for (const SGroup& g : sgroups)
            if (g.persistent_ok) {
                tiles += g.tiles;
                ++ngroups;
            }
        const bool stream_rnrz = ngroups == 0 || tiles >= min_tiles * ngroups;
        std::vector<SGroup> kept;
        for (SGroup& g : sgroups) {
            if (g.persistent_ok && !stream_rnrz) {
                for (int32_t i : g.members) group[(size_t)i] = prep[(size_t)i].opc;
                continue;
            }
            for (int32_t i : g.members) {
                const BinopArgs& a = prep[(size_t)i].args;
                StreamJob sj;
                sj.a = a.a;
                sj.b = a.b;
                sj.out = a.out;
                sj.S = a.S;
                sj.nwords = a.nwords;
                sj.tile0 = (int64_t)g.tmap.size();
                sj.tailmask = a.tailmask;
                sj.negb = a.negb;
                const int64_t nt = (a.S + g.e->stream_tw - 1) / g.e->stream_tw;
                const int32_t idx = (int32_t)g.jobs.size();
                g.jobs.push_back(sj);
                for (int64_t t = 0; t < nt; ++t) g.tmap.push_back(idx);
            }
            kept.push_back(std::move(g));
        }
        sgroups.swap(kept);
    }
    for (SGroup& g : sgroups) {
        const cudaError_t e = g.e->stream_batch_prepare();
        if (e != cudaSuccess) return set_cuda_error(e);
    }

    /* unified kernels: per op class, the jobs' descriptors and tile map (tile
     * widths per kind from the kernel's shape) */
    UStreamEntry uent[2];
    std::vector<JobDesc> udesc[2];
    std::vector<int32_t> umap[2];
    for (int32_t i = 0; i < njobs && unified; ++i) {
        const int g = group[(size_t)i] - UGROUP;
        if (g < 0 || g > 1) continue;
        if (!uent[g].launch) {
            uent[g] = ustream_entry(g);
            if (!uent[g].launch) return BSFP_ERR_UNSUPPORTED;
            const cudaError_t e = uent[g].prepare();
            if (e != cudaSuccess) return set_cuda_error(e);
        }
        const bsfp_job& j = jobs[i];
        const BinopArgs& a = prep[(size_t)i].args;
        JobDesc d;
        memset(&d, 0, sizeof d);
        d.a = a.a;
        d.b = a.b;
        d.out = a.out;
        d.S = a.S;
        d.nwords = a.nwords;
        d.tile0 = (int64_t)umap[g].size();
        d.tailmask = a.tailmask;
        d.negb = a.negb;
        d.kind = batch_kind(j.f.exp_bits, j.f.man_bits, j.f.rnd);
        const int64_t tw = uent[g].tw[d.kind];
        const int64_t nt = (a.S + tw - 1) / tw;
        const int32_t idx = (int32_t)udesc[g].size();
        udesc[g].push_back(d);
        for (int64_t t = 0; t < nt; ++t) umap[g].push_back(idx);
    }

    /* tiles per group */
    const int64_t TILE = 128LL * o.wpt * BATCH_ROUNDS;
    std::vector<JobDesc> desc[OPC_COUNT];
    std::vector<int32_t> tmap[OPC_COUNT];
    for (int32_t i = 0; i < njobs; ++i) {
        const int g = group[(size_t)i];
        if (g < 0 || g >= OPC_COUNT) continue;
        const bsfp_job& j = jobs[i];
        const BinopArgs& a = prep[(size_t)i].args;
        JobDesc d;
        memset(&d, 0, sizeof d);
        d.a = a.a;
        d.b = a.b;
        d.c = a.c;
        d.out = a.out;
        d.S = a.S;
        d.nwords = a.nwords;
        d.tile0 = (int64_t)tmap[g].size();
        d.tailmask = a.tailmask;
        d.negb = a.negb;
        d.kind = batch_kind(j.f.exp_bits, j.f.man_bits, j.f.rnd);
        const int64_t nt = (a.S + TILE - 1) / TILE;
        const int32_t idx = (int32_t)desc[g].size();
        desc[g].push_back(d);
        for (int64_t t = 0; t < nt; ++t) tmap[g].push_back(idx);
    }

    /* one device buffer: descriptors, tile maps, counters; then the streamed
     * groups' job lists and tile maps */
    size_t off_desc[OPC_COUNT], off_map[OPC_COUNT], off_cnt[OPC_COUNT], total = 0;
    for (int g = 0; g < OPC_COUNT; ++g) {
        off_desc[g] = total;
        total = align_up(total + desc[g].size() * sizeof(JobDesc), 256);
        off_map[g] = total;
        total = align_up(total + tmap[g].size() * sizeof(int32_t), 256);
        off_cnt[g] = total;
        total = align_up(total + sizeof(unsigned long long), 256);
    }
    std::vector<size_t> off_sjobs(sgroups.size()), off_smap(sgroups.size());
    for (size_t g = 0; g < sgroups.size(); ++g) {
        off_sjobs[g] = total;
        total = align_up(total + sgroups[g].jobs.size() * sizeof(StreamJob), 256);
        off_smap[g] = total;
        total = align_up(total + sgroups[g].tmap.size() * sizeof(int32_t), 256);
    }
    size_t off_udesc[2], off_umap[2], off_ucnt[2];
    for (int g = 0; g < 2; ++g) {
        off_udesc[g] = total;
        total = align_up(total + udesc[g].size() * sizeof(JobDesc), 256);
        off_umap[g] = total;
        total = align_up(total + umap[g].size() * sizeof(int32_t), 256);
        off_ucnt[g] = total;
        total = align_up(total + sizeof(unsigned long long), 256);
    }

    bsfp_batch_plan p = new bsfp_batch_plan_st();
    cudaError_t err = cudaMalloc(&p->dev, total);
    if (err != cudaSuccess) {
        plan_destroy(p);
        return set_cuda_error(err);
    }
    char* base = static_cast<char*>(p->dev);
    for (int g = 0; g < OPC_COUNT && err == cudaSuccess; ++g) {
        if (!desc[g].empty()) err = cudaMemcpy(base + off_desc[g], desc[g].data(), desc[g].size() * sizeof(JobDesc),
                                               cudaMemcpyHostToDevice);
        if (err == cudaSuccess && !tmap[g].empty())
            err = cudaMemcpy(base + off_map[g], tmap[g].data(), tmap[g].size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice);
    }
    for (size_t g = 0; g < sgroups.size() && err == cudaSuccess; ++g) {
        err = cudaMemcpy(base + off_sjobs[g], sgroups[g].jobs.data(), sgroups[g].jobs.size() * sizeof(StreamJob),
                         cudaMemcpyHostToDevice);
        if (err == cudaSuccess)
            err = cudaMemcpy(base + off_smap[g], sgroups[g].tmap.data(), sgroups[g].tmap.size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice);
    }
    for (int g = 0; g < 2 && err == cudaSuccess; ++g) {
        if (udesc[g].empty()) continue;
        err = cudaMemcpy(base + off_udesc[g], udesc[g].data(), udesc[g].size() * sizeof(JobDesc),
                         cudaMemcpyHostToDevice);
        if (err == cudaSuccess)
            err = cudaMemcpy(base + off_umap[g], umap[g].data(), umap[g].size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice);
    }
    if (err != cudaSuccess) {
        plan_destroy(p);
        return set_cuda_error(err);
    }

    /* capture: per group, clear the counter and run the persistent kernel;
     * then the plain launches */
    /* persistent grids: resident CTAs per SM x SMs, at most one CTA per tile */
    int grid[OPC_COUNT] = {0, 0, 0};
    for (int g = 0; g < OPC_COUNT; ++g) {
        if (tmap[g].empty()) continue;
        int occ = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel_ptr(g, o.wpt), 128, 0);
        if (err != cudaSuccess) {
            plan_destroy(p);
            return set_cuda_error(err);
        }
        if (occ < 1) occ = 1;
        const int bps = (o.blocks_per_sm > 0 && o.blocks_per_sm < occ) ? o.blocks_per_sm : occ;
        const int64_t ntiles = (int64_t)tmap[g].size();
        const int64_t cap = (int64_t)device_num_sms() * bps;
        grid[g] = (int)(ntiles < cap ? ntiles : cap);
    }

    cudaStream_t cs;
    err = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (err != cudaSuccess) {
        plan_destroy(p);
        return set_cuda_error(err);
    }
    bsfp_status st = BSFP_OK;
    /* side streams and events for the plan's parallel branches */
    constexpr int NBRANCH = 8;
    bool any_plain = false;
    for (int32_t i = 0; i < njobs; ++i) any_plain = any_plain || (group[(size_t)i] < 0 && !prep[(size_t)i].skip);
    size_t npersistent = 0;
    for (int g = 0; g < OPC_COUNT; ++g) npersistent += tmap[g].empty() ? 0 : 1;
    const size_t nbranches = sgroups.size() + (udesc[0].empty() ? 0 : 1) + (udesc[1].empty() ? 0 : 1) + npersistent +
                             (any_plain ? 1 : 0);
    const int nside = (int)(nbranches < (size_t)NBRANCH ? nbranches : (size_t)NBRANCH);
    cudaStream_t side[NBRANCH] = {};
    cudaEvent_t fork = nullptr, join[NBRANCH] = {};
    for (int i = 0; i < nside && err == cudaSuccess; ++i) {
        err = cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming);
    }
    if (err == cudaSuccess && nside) err = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
        /* Every kernel of the plan is independent of the others, so each
         * group -- a unified or streamed group, a persistent op class, and
         * the plain launches together -- is captured as a parallel branch
         * (branch b on side stream b mod 8): one group's blocks take the SMs
         * that another's last tiles leave idle, instead of each launch
         * ramping up and draining on its own.  Streamed groups run one block
         * per SM, at most one per tile. */
        if (nside) {
            cudaError_t e2 = cudaEventRecord(fork, cs);
            for (int i = 0; i < nside && e2 == cudaSuccess; ++i) e2 = cudaStreamWaitEvent(side[i], fork, 0);
            if (e2 != cudaSuccess) st = set_cuda_error(e2);
        }
        size_t branch = 0;
        /* the unified kernels first: the longest branches */
        for (int g = 0; g < 2 && st == BSFP_OK; ++g) {
            if (udesc[g].empty()) continue;
            const int64_t ntiles = (int64_t)umap[g].size();
            const int64_t sms = device_num_sms();
            cudaStream_t bs = side[branch++ % NBRANCH];
            unsigned long long* cnt = reinterpret_cast<unsigned long long*>(base + off_ucnt[g]);
            cudaError_t e2 = cudaMemsetAsync(cnt, 0, sizeof *cnt, bs);
            if (e2 == cudaSuccess)
                e2 = uent[g].launch(reinterpret_cast<const JobDesc*>(base + off_udesc[g]),
                                    reinterpret_cast<const int32_t*>(base + off_umap[g]), ntiles, cnt,
                                    current_fault_word(), (int)(ntiles < sms ? ntiles : sms), bs);
            if (e2 != cudaSuccess) st = set_cuda_error(e2);
            else p->launches += 1;
        }
        /* then the persistent kernels, one branch per op class */
        for (int g = 0; g < OPC_COUNT && st == BSFP_OK; ++g) {
            if (tmap[g].empty()) continue;
            cudaStream_t bs = side[branch++ % NBRANCH];
            unsigned long long* cnt = reinterpret_cast<unsigned long long*>(base + off_cnt[g]);
            cudaError_t e2 = cudaMemsetAsync(cnt, 0, sizeof *cnt, bs);
            if (e2 == cudaSuccess)
                e2 = batch_launcher(g, o.wpt)(reinterpret_cast<const JobDesc*>(base + off_desc[g]),
                                              reinterpret_cast<const int32_t*>(base + off_map[g]),
                                              (int64_t)tmap[g].size(), cnt, grid[g], bs);
            if (e2 != cudaSuccess) st = set_cuda_error(e2);
            else p->launches += 1;
        }
        for (size_t g = 0; g < sgroups.size() && st == BSFP_OK; ++g) {
            const int64_t ntiles = (int64_t)sgroups[g].tmap.size();
            const int64_t sms = device_num_sms();
            const cudaError_t e2 = sgroups[g].e->stream_batch_launch(
                reinterpret_cast<const StreamJob*>(base + off_sjobs[g]),
                reinterpret_cast<const int32_t*>(base + off_smap[g]), ntiles, sgroups[g].fault,
                (int)(ntiles < sms ? ntiles : sms), side[branch++ % NBRANCH]);
            if (e2 != cudaSuccess) st = set_cuda_error(e2);
            else p->launches += 1;
        }
        /* the plain launches, one after another on one branch */
        if (any_plain && st == BSFP_OK) {
            cudaStream_t bs = side[branch++ % NBRANCH];
            for (int32_t i = 0; i < njobs && st == BSFP_OK; ++i) {
                if (group[(size_t)i] >= 0 || prep[(size_t)i].skip) continue;
                st = launch_prepared(prep[(size_t)i], bs);
                if (st == BSFP_OK) p->launches += 1;
            }
        }
        /* join every branch back (also after an error: the capture must end
         * with all its streams joined) */
        for (int i = 0; i < nside; ++i) {
            cudaError_t e2 = cudaEventRecord(join[i], side[i]);
            if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(cs, join[i], 0);
            if (e2 != cudaSuccess && st == BSFP_OK) st = set_cuda_error(e2);
        }
        cudaGraph_t g = nullptr;
        const cudaError_t e3 = cudaStreamEndCapture(cs, &g);
        p->graph = g;
        if (st == BSFP_OK && e3 != cudaSuccess) st = set_cuda_error(e3);
    } else {
        st = set_cuda_error(err);
    }
    for (int i = 0; i < nside; ++i) {
        if (side[i]) cudaStreamDestroy(side[i]);
        if (join[i]) cudaEventDestroy(join[i]);
    }
    if (fork) cudaEventDestroy(fork);
    cudaStreamDestroy(cs);
    if (st == BSFP_OK) {
        err = cudaGraphInstantiate(&p->exec, p->graph, 0);
        if (err != cudaSuccess) st = set_cuda_error(err);
    }
    if (st != BSFP_OK) {
        plan_destroy(p);
        return st;
    }
    *plan_out = p;
    return BSFP_OK;
}

bsfp_status bsfp_set_batch_stream_min_tiles(int32_t tiles_per_sm) {
    if (tiles_per_sm < 0 || tiles_per_sm > 1 << 20) return BSFP_ERR_SIZE;
    g_batch_stream_min_tiles.store(tiles_per_sm, std::memory_order_relaxed);
    return BSFP_OK;
}

bsfp_status bsfp_batch_run(bsfp_batch_plan plan, bsfp_stream_t s) {
    NvtxRange range("bsfp_batch_run");
    if (!plan) return BSFP_ERR_NULL;
    const cudaError_t err = cudaGraphLaunch(plan->exec, (cudaStream_t)s);
    if (err != cudaSuccess) return set_cuda_error(err);
    count_launches(plan->launches);
    return BSFP_OK;
}

int64_t bsfp_batch_launches(bsfp_batch_plan plan) { return plan ? plan->launches : -1; }

void bsfp_batch_free(bsfp_batch_plan plan) { plan_destroy(plan); }

bsfp_status bsfp_launch_jobs(const bsfp_job* jobs, int32_t njobs, bsfp_stream_t s) {
    if (njobs < 0) return BSFP_ERR_SIZE;
    if (njobs > 0 && !jobs) return BSFP_ERR_NULL;
    for (int32_t i = 0; i < njobs; ++i) {
        PreparedOp po;
        const bsfp_job& j = jobs[i];
        bsfp_status st = prepare_binop(j.f, j.op, j.a, j.b, j.c, j.out, j.n, &po);
        if (st == BSFP_OK && !po.skip) {
            st = launch_prepared(po, (cudaStream_t)s);
            if (st == BSFP_OK) count_launches(1);
        }
        if (st != BSFP_OK) return st;
    }
    return BSFP_OK;
}

}  // extern "C"
