/*
 * Batched and served forms.
 *
 * Batched (gx_batch_*): many (program, events) items run by ONE persistent kernel.  The
 * paper schedules device work with persistent workers that claim logical work units
 * (Sec. 4.3.2, Sec. 5.3); here every item is cut into chunks of block*ept events, the
 * chunk table is uploaded once, and a launch is a captured CUDA graph of
 * [reset the claim cursor, persistent kernel with one block per free SM slot].  Blocks
 * claim chunks with one atomicAdd and restage the decoded program into shared memory
 * only when the program changes (items are laid out largest first, so a block mostly
 * stays on one program).
 *
 * Served (gx_server_*): a host thread does continuous batching over the same kernel.
 * Requests are admitted in arrival order while the device-memory budget allows
 * (resident maps + event bytes of requests not yet finished); every time one of
 * `max_inflight` streams is free, all admitted, waiting requests become the next tick:
 * its chunk table is copied to the stream's table and the stream's captured graph is
 * launched.  Ticks on different streams overlap on the device; a request that arrives
 * while ticks run joins the next one.  The plain baseline issues one gx_run_batch
 * launch per admitted request on the same streams instead.
 */
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <numeric>
#include <set>
#include <thread>
#include <vector>

#include "gx_kernels.h"
#include "gx_runtime.h"
#include "gx_steal.cuh"
#include "gx_trace.h"

using namespace gx;

namespace {

uint64_t round_up(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

struct Item {
    gx_prog *prog;
    const void *events;
    uint64_t n;
    int64_t *ret_out;
};

/*
 * Cut items into chunks of `chunk_events`, largest item first; slots: program -> slot of a
 * multi-program kernel.  With `pref_bits` set (the kernel's widest combining cache), a chunk
 * of a program whose sharding was tuned carries that choice (bit 63 of pad, the
 * ExecParams.wc_bits value in bits 32..40).
 */
/* the cache width a gx_launch.shards value runs with (0: combining off) */
uint32_t bits_of(uint32_t shards, uint32_t default_bits) {
    if (shards == GX_SHARDS_OFF) return 0;
    const uint32_t w = shards & 0xFFu;
    return w ? w : default_bits;
}

/* the width a persistent kernel's combining area is sized for: its default chunks' and the widest per-chunk choice */
uint32_t area_bits(const gx::JitKernel *jk, uint32_t shards, uint32_t widest_choice) {
    if (!jk || !jk->shard_bytes) return 0;
    return std::max(bits_of(shards, gx::wc_default_bits(*jk)), std::min(widest_choice, jk->wc_max_bits));
}

void make_chunks(const std::vector<Item> &items, uint64_t chunk_events, std::vector<gx_chunk> &out,
                 const std::map<gx_prog *, uint32_t> *slots = nullptr, uint32_t pref_bits = 0,
                 uint32_t alloc_bits = 0) {
    std::vector<size_t> order(items.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return items[a].n > items[b].n; });
    out.clear();
    for (size_t k : order) {
        const Item &it = items[k];
        for (uint64_t b = 0; b < it.n; b += chunk_events) {
            gx_chunk c;
            memset(&c, 0, sizeof c);
            c.image = (const uint8_t *)it.prog->dmem;
            c.events = (const uint8_t *)it.events;
            c.ret_out = (long long *)it.ret_out;
            c.begin = b;
            c.end = std::min(it.n, b + chunk_events);
            c.idx_base = 0;
            c.image_bytes = it.prog->image_bytes;
            c.ctx_size = it.prog->opts.ctx_size;
            c.pad = slots ? slots->at(it.prog) : 0;
            if (pref_bits && it.prog->pref_tuned && it.prog->pref_shards) {
                uint32_t sh = it.prog->pref_shards;
                uint32_t wc = sh == GX_SHARDS_OFF ? 0u : shards_param(sh, pref_bits);
                if ((wc & 0xFFu) > alloc_bits) wc = (wc & ~0xFFu) | alloc_bits; /* never wider than the area */
                c.pad |= (1ull << 63) | ((uint64_t)wc << 32);
            }
            out.push_back(c);
        }
    }
}

/* a persistent launch captured into a graph: [memset cursor][kernel] */
struct Persist {
    gx_ctx *ctx = nullptr;
    uint32_t block = 256, area = 0, max_ctx = 0;
    uint64_t smem = 0;
    unsigned grid = 0;
    void *dmem = nullptr; /* [cursor 4 B | nchunks 4 B | pad][chunk table] */
    uint64_t dbytes = 0;
    uint64_t cap_chunks = 0;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    gx::JitKernel *jk = nullptr; /* set: the persistent kernel is a multi-program specialised kernel */
    /* set: this scheduling program steers stealing (mode 2: blocks own shares of the table; mode 3 below) */
    gx_prog *sched = nullptr;
    uint64_t sched_budget = 0;
    bool launch_control = false; /* mode 3: one block per chunk, stealing by cancelling blocks not yet started */
    uint64_t steal_off = 0; /* the per-share claim counters, then the per-block tallies */

    unsigned *cursor() { return (unsigned *)dmem; }
    unsigned *nchunks() { return (unsigned *)dmem + 1; }
    gx_chunk *table() { return (gx_chunk *)((uint8_t *)dmem + 256); }
    uint32_t *steal_next() { return (uint32_t *)((uint8_t *)dmem + steal_off); }
    uint32_t *steal_tally() { return steal_next() + round_up(grid, 4); }
    uint64_t steal_bytes() const { return round_up(grid, 4) * 4 + (uint64_t)grid * GX_STEAL_WORDS * 4; }

    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        dfree(ctx, dmem, dbytes);
        dmem = nullptr;
        dbytes = 0;
    }

    /*
     * shards: gx_launch.shards of chunks that carry no choice of their own (0 = the default
     * width, GX_SHARDS_OFF = none); alloc_bits: the widest cache any chunk may use, which
     * sizes the combining area.
     */
    uint32_t alloc_bits = 0;
    uint32_t variant = 0; /* the multi-program kernel's entry (GX_VARIANT_*; 0 = its default, capped) */
    int build(gx_ctx *c, uint32_t blk, uint32_t image_area, uint32_t ctx_max, uint64_t chunks, uint32_t shards = 0,
              uint32_t alloc_wc = 0) {
        release();
        ctx = c;
        block = blk;
        area = (uint32_t)round_up(image_area, 16);
        max_ctx = ctx_max;
        smem = exec_smem(area, block, max_ctx);
        uint32_t wc = 0, shard_off = 0;
        alloc_bits = area_bits(jk, shards, alloc_wc);
        if (jk && jk->shard_bytes) { /* chunks may switch combining on even when the default is off */
            wc = shards == GX_SHARDS_OFF ? 0u : shards_param(shards, gx::wc_default_bits(*jk));
            shard_off = (uint32_t)round_up(smem, 16);
            smem = shard_off + gx::wc_area_bytes(*jk, alloc_bits);
        }
        int rc = jk ? cuda_status(jit_set_smem(*jk, smem)) : ensure_smem(c, smem);
        if (rc) return rc;
        int occ = 0;
        cudaError_t oe = jk ? jit_occupancy(*jk, (int)block, smem, &occ, variant) : exec_occupancy((int)block, smem, &occ);
        if (oe != cudaSuccess || occ < 1) {
            cudaGetLastError();
            return GX_E_CUDA;
        }
        grid = (unsigned)(c->sms * occ);
        if (sched && launch_control) grid = (unsigned)std::max<uint64_t>(chunks, 1);
        cap_chunks = std::max<uint64_t>(chunks, 1);
        dbytes = 256 + cap_chunks * sizeof(gx_chunk);
        steal_off = dbytes;
        if (sched) dbytes += steal_bytes();
        rc = dalloc(c, dbytes, &dmem);
        if (rc) return rc;
        if (cudaMemset(dmem, 0, 256) != cudaSuccess) return GX_E_CUDA;
        if (sched) { /* the header of modes 2 and 3; the chunk count is written with the table */
            gx_steal_hdr h;
            memset(&h, 0, sizeof h);
            h.shares = grid;
            h.hook_ctx_size = GX_SCHED_CTX;
            h.budget_ns = sched_budget;
            h.hook = (const uint8_t *)sched->dmem;
            h.next = steal_next();
            h.tally = steal_tally();
            if (cudaMemcpy(dmem, &h, sizeof h, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemset(steal_next(), 0, steal_bytes()) != cudaSuccess)
                return GX_E_CUDA;
        }
        ExecParams P;
        memset(&P, 0, sizeof P);
        P.image_area = area;
        P.mode = sched ? (launch_control ? 3 : 2) : 1;
        P.chunks = table();
        P.cursor = cursor();
        P.nchunks_dev = nchunks();
        P.wc_bits = wc;
        P.shard_off = shard_off;
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return GX_E_CUDA;
        rc = GX_OK;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = GX_E_CUDA;
        if (rc == GX_OK) {
            cudaMemsetAsync(cursor(), 0, 4, cs);
            if (sched) cudaMemsetAsync(steal_next(), 0, steal_bytes(), cs);
            if (jk) jit_launch(*jk, P, grid, block, smem, cs, variant);
            else launch_exec(P, grid, block, smem, cs);
            if (cudaStreamEndCapture(cs, &graph) != cudaSuccess) rc = GX_E_CUDA;
        }
        if (rc == GX_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rc = GX_E_CUDA;
        cudaStreamDestroy(cs);
        if (rc) cudaGetLastError();
        return rc;
    }

    int launch(cudaStream_t s) { return cudaGraphLaunch(exec, s) == cudaSuccess ? GX_OK : GX_E_CUDA; }
};

} // namespace

struct gx_batch {
    gx_ctx *ctx = nullptr;
    std::vector<Item> items;
    std::vector<gx_chunk> chunks;
    Persist persist;
    bool planned = false;
    gx_launch shape{};
    /* all programs specialised: one kernel holding every distinct program, switched by slot */
    gx::JitKernel jk;
    std::map<gx_prog *, uint32_t> slots;
    bool jit = false;
    gx_prog *sched = nullptr; /* the scheduling program (gx_batch_set_sched) */
    uint64_t sched_budget = 0;
    uint32_t sched_flags = 0;
};

/* build the batch's multi-program kernel when every item's program is specialised */
static int batch_jit(gx_batch *b) {
    b->jit = !b->items.empty();
    for (auto &it : b->items)
        if (!it.prog->jit) b->jit = false;
    if (!b->jit) {
        for (auto &it : b->items)
            if (it.prog->jp.warp) return GX_EINVAL; /* a warp-level program exists only as specialised code */
        return b->sched ? GX_EINVAL : GX_OK; /* so does the work-stealing kernel */
    }
    std::vector<const gx::JitProgram *> progs;
    b->slots.clear();
    for (auto &it : b->items)
        if (!b->slots.count(it.prog)) {
            b->slots[it.prog] = (uint32_t)progs.size();
            progs.push_back(&it.prog->jp);
        }
    std::string log;
    int rc = gx::jit_build(progs, b->jk, log, b->sched ? &b->sched->jp : nullptr);
    if (rc) b->jit = false;
    return rc;
}

struct gx_server {
    struct Req {
        gx_prog *prog;
        const void *events;
        uint64_t n;
        int64_t *ret_out;
        uint64_t tag;
        double t_arrival;
        uint64_t bytes;
    };
    struct Slot {
        cudaStream_t stream = nullptr;
        cudaEvent_t done = nullptr;
        Persist persist;
        gx_chunk *host_table = nullptr; /* pinned */
        std::vector<Req> reqs;
        double t_start = 0;
        bool busy = false;
    };
    gx_ctx *ctx = nullptr;
    gx_server_opts opts{};
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_in, cv_out;
    bool stop = false;
    std::deque<Req> queue;
    std::deque<gx_completion> done;
    std::vector<Slot> slots;
    uint64_t inflight_bytes = 0;
    uint64_t chunk_events = 1024;
    uint64_t cap_chunks = 1 << 16;
    std::set<gx_map *> maps_seen;
    uint64_t map_bytes = 0;
    int error = GX_OK;
    /* registered specialised programs: one multi-program kernel for every tick */
    gx::JitKernel jk;
    std::map<gx_prog *, uint32_t> prog_slot;
    bool jit = false;

    void run();
};

/* ================================================================ batch */
extern "C" {

int gx_batch_create(gx_ctx *c, gx_batch **out) {
    if (!c || !out) return GX_EINVAL;
    gx_batch *b = new gx_batch();
    b->ctx = c;
    c->live++;
    *out = b;
    return GX_OK;
}

int gx_batch_add(gx_batch *b, gx_prog *p, const void *events, uint64_t n, int64_t *ret_out) {
    if (!b || !p || p->ctx != b->ctx || (!events && n) || (((uintptr_t)events) & 15)) return GX_EINVAL;
    if (b->planned || (p->opts.flags & GX_PROG_CHECKED)) return GX_EINVAL; /* checked programs: plain launches */
    b->items.push_back(Item{p, events, n, ret_out});
    return GX_OK;
}

static int batch_plan_shape(gx_batch *b, uint32_t block, uint32_t ept, uint32_t shards, uint32_t variant = 0) {
    uint32_t area = 0, max_ctx = 8;
    for (auto &it : b->items) {
        area = std::max(area, it.prog->image_bytes);
        max_ctx = std::max(max_ctx, it.prog->opts.ctx_size);
    }
    /* the default width lets every program use its own tuned sharding */
    const bool use_pref = b->jit && shards == 0;
    const uint32_t dflt = b->jit ? gx::wc_default_bits(b->jk) : 0;
    uint32_t alloc = 0;
    if (use_pref)
        for (auto &it : b->items)
            if (it.prog->pref_tuned) alloc = std::max(alloc, bits_of(it.prog->pref_shards, dflt));
    /* one kernel holds every program: a wide cache would cost all of them occupancy */
    alloc = std::min(alloc, dflt);
    b->persist.jk = b->jit ? &b->jk : nullptr;
    b->persist.variant = b->jit ? variant : 0;
    b->persist.sched = b->sched;
    b->persist.sched_budget = b->sched_budget;
    b->persist.launch_control = (b->sched_flags & GX_SCHED_F_LAUNCH_CONTROL) != 0;
    make_chunks(b->items, (uint64_t)block * ept, b->chunks, b->jit ? &b->slots : nullptr, use_pref ? dflt : 0,
                area_bits(b->persist.jk, shards, alloc));
    int rc = b->persist.build(b->ctx, block, area, max_ctx, b->chunks.size(), shards, alloc);
    if (rc) return rc;
    unsigned nch = (unsigned)b->chunks.size();
    if (cudaMemcpy(b->persist.table(), b->chunks.data(), b->chunks.size() * sizeof(gx_chunk),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->persist.nchunks(), &nch, 4, cudaMemcpyHostToDevice) != cudaSuccess)
        return GX_E_CUDA;
    b->shape = gx_launch{block, ept, b->persist.grid, shards, b->persist.variant, 0};
    return GX_OK;
}

int gx_batch_plan(gx_batch *b, const gx_launch *lp, void *stream) {
    if (!b || b->items.empty()) return GX_EINVAL;
    if (b->chunks.size() > 0x7FFFFFFF) return GX_E2BIG;
    cudaStream_t s = (cudaStream_t)stream;
    int jrc = batch_jit(b);
    if (jrc) return jrc;
    if (lp) {
        uint32_t blk = lp->block ? lp->block : 256, ept = lp->ept ? lp->ept : 4;
        if (blk < 64 || blk > GX_MAX_BLOCK || blk % 32 || ept < 1 || ept > 64) return GX_EINVAL;
        if (!shards_valid(lp->shards)) return GX_EINVAL;
        if (lp->variant > GX_VARIANT_4) return GX_EINVAL;
        int rc = batch_plan_shape(b, blk, ept, lp->shards, lp->variant);
        if (rc == GX_OK) b->planned = true;
        return rc;
    }
    /*
     * Autotune on scratch copies of every map the items touch: the tuning launches run
     * real programs over real events, so they must not change the real maps.
     */
    std::vector<gx_map *> maps;
    for (auto &it : b->items)
        for (auto *m : it.prog->maps)
            if (std::find(maps.begin(), maps.end(), m) == maps.end()) maps.push_back(m);
    if (b->sched)
        for (auto *m : b->sched->maps)
            if (std::find(maps.begin(), maps.end(), m) == maps.end()) maps.push_back(m);
    std::vector<void *> saved(maps.size(), nullptr);
    int rc = GX_OK;
    /* each program's own sharding first (on its largest item, scratch maps) */
    if (b->jit) {
        std::map<gx_prog *, const Item *> largest;
        for (auto &it : b->items)
            if (!largest.count(it.prog) || largest[it.prog]->n < it.n) largest[it.prog] = &it;
        for (auto &kv : largest)
            if (!kv.first->pref_tuned && kv.second->n && rc == GX_OK)
                rc = gx::tune_shards(kv.first, kv.second->events, kv.second->n, s);
    }
    for (size_t i = 0; i < maps.size() && rc == GX_OK; i++) {
        rc = dalloc(b->ctx, maps[i]->dbytes, &saved[i]);
        if (rc == GX_OK &&
            cudaMemcpyAsync(saved[i], maps[i]->dmem, maps[i]->dbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            rc = GX_E_CUDA;
    }
    gx_launch best = {256, 4, 0, 0};
    if (rc == GX_OK) {
        float best_ms = 1e30f;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        const uint32_t blocks[] = {128, 256};
        const uint32_t epts[] = {2, 4, 8, 16};
        std::vector<uint32_t> widths = {0}; /* per-program choices ride on the chunks */
        /* every entry the multi-program kernel has */
        std::vector<uint32_t> variants;
        for (uint32_t v = 1; b->jit && v < 5; v++)
            if (b->jk.variant[v]) variants.push_back(v);
        if (variants.empty()) variants = {0};
        for (uint32_t blk : blocks)
            for (uint32_t ept : epts) for (uint32_t w : widths) for (uint32_t v : variants) {
                if (batch_plan_shape(b, blk, ept, w, v) != GX_OK) continue;
                b->persist.launch(s); /* warm-up */
                cudaEventRecord(e0, s);
                b->persist.launch(s);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best_ms) {
                    best_ms = ms;
                    best = gx_launch{blk, ept, 0, w, v, 0};
                }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        /* put the maps back as they were before tuning */
        for (size_t i = 0; i < maps.size(); i++)
            if (cudaMemcpyAsync(maps[i]->dmem, saved[i], maps[i]->dbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                rc = GX_E_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) rc = GX_E_CUDA;
    }
    for (size_t i = 0; i < maps.size(); i++) dfree(b->ctx, saved[i], maps[i]->dbytes);
    if (rc) return rc;
    rc = batch_plan_shape(b, best.block, best.ept, best.shards, best.variant);
    if (rc == GX_OK) b->planned = true;
    return rc;
}

int gx_batch_launch(gx_batch *b, void *stream) {
    if (!b || !b->planned) return GX_EINVAL;
    if (b->persist.launch_control && b->ctx->launch_control_timed_out) return GX_E_TIMEOUT;
    TraceRange tr("gx_batch_launch");
    int rc = b->persist.launch((cudaStream_t)stream);
    if (rc == GX_OK) {
        for (auto &it : b->items) it.prog->launches++;
        if (b->sched) b->sched->launches++;
    }
    return rc;
}

int gx_batch_set_sched(gx_batch *b, gx_prog *hook, uint64_t budget_ns, const gx_simt_spec *limits, uint32_t flags,
                       char *log, size_t log_len) {
    if (!b || !hook || hook->ctx != b->ctx || b->planned || !hook->jit || hook->jp.warp) return GX_EINVAL;
    if (flags & ~GX_SCHED_F_LAUNCH_CONTROL) return GX_EINVAL;
    gx::VerifyOut v;
    const gx::JitProgram &jp = hook->jp;
    int rc = gx::check_sched_program(jp.insns.data(), (uint32_t)jp.insns.size(), jp.maps.data(),
                                     (uint32_t)jp.maps.size(), hook->opts, limits, v);
    if (log && log_len) {
        size_t k = std::min(log_len - 1, v.log.size());
        memcpy(log, v.log.data(), k);
        log[k] = 0;
    }
    if (rc) return rc;
    if ((flags & GX_SCHED_F_LAUNCH_CONTROL) && b->ctx->launch_control_timed_out) return GX_E_TIMEOUT;
    b->sched = hook;
    b->sched_budget = budget_ns;
    b->sched_flags = flags;
    if (flags & GX_SCHED_F_LAUNCH_CONTROL) hook->sched_lc = true;
    return GX_OK;
}

int gx_batch_sched_tally(gx_batch *b, uint32_t *out, uint32_t cap_blocks, uint32_t *n_blocks, void *stream) {
    if (!b || !b->sched || !b->planned || !n_blocks || (cap_blocks && !out)) return GX_EINVAL;
    const uint32_t g = b->persist.grid;
    *n_blocks = g;
    if (cap_blocks < g) return GX_ENOSPC;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess ||
        cudaMemcpy(out, b->persist.steal_tally(), (size_t)g * GX_STEAL_WORDS * 4, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
        return GX_E_CUDA;
    return GX_OK;
}

int gx_batch_destroy(gx_batch *b) {
    if (!b) return GX_EINVAL;
    cudaDeviceSynchronize();
    b->persist.release();
    b->ctx->live--;
    delete b;
    return GX_OK;
}

/* ================================================================ server */
int gx_server_create(gx_ctx *c, const gx_server_opts *o, gx_server **out) {
    if (!c || !o || !out) return GX_EINVAL;
    gx_server_opts opts = *o;
    if (opts.max_inflight == 0) opts.max_inflight = 2;
    if (opts.max_items == 0) opts.max_items = 1024;
    if (opts.block == 0) opts.block = 256;
    if (opts.ept == 0) opts.ept = 4;
    if (opts.max_inflight > 8 || opts.max_items > 4096 || opts.block < 64 || opts.block > GX_MAX_BLOCK ||
        opts.block % 32 || opts.ept > 64)
        return GX_EINVAL;
    if (opts.n_progs && !opts.progs) return GX_EINVAL;
    gx_server *s = new gx_server();
    s->ctx = c;
    s->opts = opts;
    s->chunk_events = (uint64_t)opts.block * opts.ept;
    if (opts.n_progs) {
        bool all_jit = true;
        std::vector<const gx::JitProgram *> progs;
        for (uint32_t i = 0; i < opts.n_progs; i++) {
            gx_prog *p = opts.progs[i];
            if (!p || p->ctx != c) {
                delete s;
                return GX_EINVAL;
            }
            if (!p->jit) all_jit = false;
            if (!s->prog_slot.count(p)) {
                s->prog_slot[p] = (uint32_t)progs.size();
                progs.push_back(&p->jp);
            }
        }
        if (!all_jit && !opts.plain)
            for (auto &ps : s->prog_slot)
                if (ps.first->jp.warp) { /* a warp-level program exists only as specialised code */
                    delete s;
                    return GX_EINVAL;
                }
        if (all_jit && !opts.plain) {
            std::string log;
            int rc = gx::jit_build(progs, s->jk, log);
            if (rc) {
                delete s;
                return rc;
            }
            s->jit = true;
        }
    }
    s->slots.resize(opts.max_inflight);
    for (auto &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost((void **)&sl.host_table, (s->cap_chunks + 1) * sizeof(gx_chunk)) != cudaSuccess) {
            cudaGetLastError();
            for (auto &x : s->slots) {
                if (x.stream) cudaStreamDestroy(x.stream);
                if (x.done) cudaEventDestroy(x.done);
                if (x.host_table) cudaFreeHost(x.host_table);
            }
            delete s;
            return GX_E_CUDA;
        }
    }
    c->live++;
    s->th = std::thread([s] { s->run(); });
    *out = s;
    return GX_OK;
}

int gx_server_submit(gx_server *s, gx_prog *p, const void *events, uint64_t n, int64_t *ret_out, uint64_t tag,
                     double t_arrival) {
    if (!s || !p || p->ctx != s->ctx || (!events && n) || (((uintptr_t)events) & 15)) return GX_EINVAL;
    if (s->jit && !s->prog_slot.count(p)) return GX_EINVAL; /* not part of the server's kernel */
    if (p->opts.flags & GX_PROG_CHECKED) return GX_EINVAL;   /* checked programs: plain launches */
    gx_server::Req r{p, events, n, ret_out, tag, t_arrival > 0 ? t_arrival : now_s(), n * p->opts.ctx_size};
    std::lock_guard<std::mutex> g(s->mu);
    for (auto *m : p->maps)
        if (s->maps_seen.insert(m).second) s->map_bytes += m->dbytes;
    if (s->opts.mem_budget && r.bytes + s->map_bytes > s->opts.mem_budget) return GX_E_ADMISSION;
    if (!s->opts.plain && (n + s->chunk_events - 1) / s->chunk_events > s->cap_chunks) return GX_E_ADMISSION;
    s->queue.push_back(r);
    s->cv_in.notify_one();
    return GX_OK;
}

int gx_server_replay(gx_server *s, const gx_request *reqs, uint32_t n, double t0) {
    if (!s || (!reqs && n)) return GX_EINVAL;
    if (t0 <= 0) t0 = now_s();
    int rc = GX_OK;
    for (uint32_t i = 0; i < n; i++) {
        const double t = t0 + reqs[i].t_offset;
        while (now_s() < t) {
        }
        int r = gx_server_submit(s, reqs[i].prog, reqs[i].events_dev, reqs[i].n, reqs[i].ret_out_dev, reqs[i].tag, t);
        if (r && rc == GX_OK) rc = r;
    }
    return rc;
}

int gx_server_poll(gx_server *s, gx_completion *out, uint32_t cap, uint32_t *n_out, int wait_ms) {
    if (!s || (!out && cap) || !n_out) return GX_EINVAL;
    std::unique_lock<std::mutex> g(s->mu);
    if (s->done.empty() && wait_ms > 0)
        s->cv_out.wait_for(g, std::chrono::milliseconds(wait_ms), [s] { return !s->done.empty() || s->error; });
    uint32_t k = 0;
    while (k < cap && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *n_out = k;
    return s->error;
}

int gx_server_destroy(gx_server *s) {
    if (!s) return GX_EINVAL;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        s->cv_in.notify_all();
    }
    s->th.join();
    for (auto &sl : s->slots) {
        cudaStreamSynchronize(sl.stream);
        sl.persist.release();
        cudaStreamDestroy(sl.stream);
        cudaEventDestroy(sl.done);
        cudaFreeHost(sl.host_table);
    }
    s->ctx->live--;
    delete s;
    return GX_OK;
}

} /* extern "C" */

/* the server thread: retire finished launches, admit, launch */
void gx_server::run() {
    const bool plain = opts.plain != 0;
    for (;;) {
        bool busy_any = false;
        /* 1. retire finished launches */
        for (auto &sl : slots) {
            if (!sl.busy) continue;
            cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) {
                busy_any = true;
                continue;
            }
            const double t = now_s();
            std::lock_guard<std::mutex> g(mu);
            for (auto &r : sl.reqs) {
                gx_completion c;
                memset(&c, 0, sizeof c);
                c.tag = r.tag;
                c.status = q == cudaSuccess ? GX_OK : GX_E_CUDA;
                c.t_arrival = r.t_arrival;
                c.t_start = sl.t_start;
                c.t_done = t;
                done.push_back(c);
                inflight_bytes -= r.bytes;
            }
            if (q != cudaSuccess) {
                cudaGetLastError();
                error = GX_E_CUDA;
            }
            sl.reqs.clear();
            sl.busy = false;
            cv_out.notify_all();
        }
        /* 2. form the next launch on a free stream */
        Slot *free_slot = nullptr;
        for (auto &sl : slots)
            if (!sl.busy) {
                free_slot = &sl;
                break;
            }
        std::vector<Req> take;
        {
            std::unique_lock<std::mutex> g(mu);
            if (stop && queue.empty() && !busy_any) break;
            if (!free_slot || queue.empty()) {
                if (!busy_any && queue.empty()) cv_in.wait_for(g, std::chrono::microseconds(200));
                g.unlock();
                if (busy_any) std::this_thread::yield();
                continue;
            }
            uint64_t nchunks = 0;
            while (!queue.empty() && take.size() < (plain ? 1u : opts.max_items)) {
                Req &r = queue.front();
                if (opts.mem_budget && inflight_bytes + r.bytes + map_bytes > opts.mem_budget) break;
                uint64_t c = (r.n + chunk_events - 1) / chunk_events;
                if (!plain && nchunks + c > cap_chunks) break;
                nchunks += c;
                inflight_bytes += r.bytes;
                take.push_back(r);
                queue.pop_front();
            }
        }
        if (take.empty()) {
            std::this_thread::yield();
            continue;
        }
        Slot &sl = *free_slot;
        sl.t_start = now_s();
        int rc = GX_OK;
        if (plain) {
            for (auto &r : take) {
                gx_launch l = {opts.block, opts.ept, 0, 0};
                int e = gx_run_batch_ex(r.prog, r.events, r.n, 0, r.ret_out, &l, sl.stream);
                if (e) rc = e;
            }
        } else {
            std::vector<Item> items;
            uint32_t area = 0, max_ctx = 8;
            for (auto &r : take) {
                items.push_back(Item{r.prog, r.events, r.n, r.ret_out});
                area = std::max(area, r.prog->image_bytes);
                max_ctx = std::max(max_ctx, r.prog->opts.ctx_size);
            }
            if (!sl.persist.exec || area > sl.persist.area || max_ctx > sl.persist.max_ctx) {
                cudaStreamSynchronize(sl.stream);
                sl.persist.jk = jit ? &jk : nullptr;
                /* the registered programs' tuned widths, at most the default: one kernel holds them all */
                uint32_t widest = 0;
                if (jit)
                    for (auto &kv : prog_slot)
                        if (kv.first->pref_tuned)
                            widest = std::max(widest, bits_of(kv.first->pref_shards, gx::wc_default_bits(jk)));
                if (jit) widest = std::min(widest, gx::wc_default_bits(jk));
                rc = sl.persist.build(ctx, opts.block, std::max(area, sl.persist.area),
                                      std::max(max_ctx, sl.persist.max_ctx), cap_chunks, 0, widest);
            }
            std::vector<gx_chunk> table;
            make_chunks(items, chunk_events, table, jit ? &prog_slot : nullptr, jit ? gx::wc_default_bits(jk) : 0,
                        sl.persist.alloc_bits);
            if (rc == GX_OK) {
                memcpy(sl.host_table, table.data(), table.size() * sizeof(gx_chunk));
                /* the count travels in the same pinned buffer, in the entry after the table */
                unsigned *count = (unsigned *)(sl.host_table + cap_chunks);
                *count = (unsigned)table.size();
                if (cudaMemcpyAsync(sl.persist.table(), sl.host_table, table.size() * sizeof(gx_chunk),
                                    cudaMemcpyHostToDevice, sl.stream) != cudaSuccess ||
                    cudaMemcpyAsync(sl.persist.nchunks(), count, 4, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
                    rc = GX_E_CUDA;
            }
            if (rc == GX_OK) {
                TraceRange tr("gx_server_tick");
                rc = sl.persist.launch(sl.stream);
            }
            for (auto &r : take) r.prog->launches++;
        }
        if (rc == GX_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) rc = GX_E_CUDA;
        sl.reqs = take;
        sl.busy = true;
        if (rc) {
            std::lock_guard<std::mutex> g(mu);
            error = rc;
        }
    }
}
