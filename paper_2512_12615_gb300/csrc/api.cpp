/*
 * Host runtime behind the C ABI in include/gx.h: contexts, device-memory accounting,
 * maps (create / snapshot / restore / drain), program load (verify -> decode -> upload),
 * runs, the end-to-end host-buffer path and the launch-shape autotuner.
 */
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "gx_internal.h"
#include "gx_kernels.h"
#include "gx_runtime.h"
#include "gx_trace.h"
#include "tune_cache.h"

using namespace gx;

/* ================================================================ helpers */
namespace gx {

double now_s() {
    using namespace std::chrono;
    return duration_cast<duration<double>>(steady_clock::now().time_since_epoch()).count();
}

static uint64_t round_up(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

int dalloc(gx_ctx *c, uint64_t bytes, void **out) {
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    bytes = round_up(bytes, 256);
    {
        std::lock_guard<std::mutex> g(c->mu);
        if (c->budget && c->used + bytes > c->budget) return GX_ENOMEM;
        c->used += bytes;
    }
    if (cudaMalloc(out, bytes) != cudaSuccess) {
        cudaGetLastError();
        std::lock_guard<std::mutex> g(c->mu);
        c->used -= bytes;
        *out = nullptr;
        return GX_ENOMEM;
    }
    return GX_OK;
}

void dfree(gx_ctx *c, void *p, uint64_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 16;
    bytes = round_up(bytes, 256);
    cudaFree(p);
    std::lock_guard<std::mutex> g(c->mu);
    c->used -= bytes;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return GX_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GX_ENOMEM : GX_E_CUDA;
}

/* program image bytes for a given set of map descriptors */
std::vector<uint8_t> build_image(const gx_prog *p, const std::vector<gx_dmap> &descs, unsigned long long *stats) {
    uint64_t bytes = sizeof(gx_dprog_hdr) + descs.size() * sizeof(gx_dmap) + p->uops.size() * 8;
    bytes = round_up(bytes, 16);
    std::vector<uint8_t> img(bytes, 0);
    gx_dprog_hdr h;
    memset(&h, 0, sizeof h);
    h.n_uops = (uint32_t)p->uops.size();
    h.n_maps = (uint32_t)descs.size();
    h.ctx_size = p->opts.ctx_size;
    h.image_bytes = (uint32_t)bytes;
    h.budget = p->opts.insn_budget ? p->opts.insn_budget : (1ull << 16);
    h.stats = stats;
    memcpy(img.data(), &h, sizeof h);
    if (!descs.empty()) memcpy(img.data() + sizeof h, descs.data(), descs.size() * sizeof(gx_dmap));
    memcpy(img.data() + sizeof h + descs.size() * sizeof(gx_dmap), p->uops.data(), p->uops.size() * 8);
    return img;
}

/* gx_launch.shards: OFF, or a width in 2..10 (0 = default) with an optional GX_SHARDS_AGG */
bool shards_valid(uint32_t sh) {
    if (sh == GX_SHARDS_OFF) return true;
    if (sh & ~(GX_SHARDS_AGG | 0xFFu)) return false;
    uint32_t w = sh & 0xFFu;
    return w == 0 || (w >= 2 && w <= 10);
}

/* ExecParams.wc_bits of a validated, enabled gx_launch.shards */
uint32_t shards_param(uint32_t sh, uint32_t default_bits) {
    uint32_t w = sh & 0xFFu;
    return (w ? w : default_bits) | ((sh & GX_SHARDS_AGG) ? 0x100u : 0u);
}

/* dynamic shared memory of one block: staged image(s) + transposed ctx tiles */
uint64_t exec_smem(uint32_t image_area, uint32_t block, uint32_t ctx_size) {
    const uint32_t cw = ctx_size / 8;
    return (uint64_t)image_area + (block / 32) * (uint64_t)cw * GX_CTX_ROW(cw) * 8;
}

int ensure_smem(gx_ctx *c, uint64_t smem) {
    std::lock_guard<std::mutex> g(c->mu);
    if (smem > c->smem_optin) return GX_E2BIG;
    if (smem > c->smem_attr) {
        if (exec_set_smem(smem) != cudaSuccess) {
            cudaGetLastError();
            return GX_E_CUDA;
        }
        c->smem_attr = smem;
    }
    return GX_OK;
}

int launch_plain(gx_prog *p, const uint8_t *image, uint32_t image_bytes, const void *events, uint64_t n,
                 uint64_t idx_base, int64_t *ret_out, const gx_launch &lp, cudaStream_t s) {
    uint32_t block = lp.block ? lp.block : 256, ept = lp.ept ? lp.ept : 4;
    if (block < 32 || block > GX_MAX_BLOCK || block % 32 || ept < 1 || ept > 64) return GX_EINVAL;
    if (lp.variant > GX_VARIANT_4) return GX_EINVAL;
    uint32_t area = (uint32_t)round_up(image_bytes, 16);
    uint64_t smem = exec_smem(area, block, p->opts.ctx_size);
    uint32_t wc = 0, shard_off = 0;
    if (!shards_valid(lp.shards)) return GX_EINVAL;
    const uint32_t sh = (lp.shards == 0 && p->pref_tuned) ? p->pref_shards : lp.shards; /* the program's tuned choice */
    if (p->jit && p->jk.shard_bytes && sh != GX_SHARDS_OFF) {
        wc = shards_param(sh, wc_default_bits(p->jk));
        shard_off = (uint32_t)round_up(smem, 16);
        smem = shard_off + wc_area_bytes(p->jk, wc & 0xFFu);
    }
    int rc = ensure_smem(p->ctx, smem);
    if (rc) return rc;
    const uint64_t per_block = (uint64_t)block * ept;
    const uint64_t chunks = (n + per_block - 1) / per_block;
    uint64_t grid = chunks;
    if (lp.grid != GX_GRID_PER_CHUNK) {
        uint64_t cap = lp.grid;
        if (cap == 0) { /* one wave: the blocks the device holds at once loop over the chunks */
            const bool checked = (p->opts.flags & GX_PROG_CHECKED) != 0;
            const uint64_t key = ((uint64_t)block << 40) | (smem << 4) | (checked ? 8u : 0u) | lp.variant;
            int occ = 0;
            bool known = false;
            {
                std::lock_guard<std::mutex> g(p->ctx->mu);
                auto it = p->occupancy.find(key);
                if (it != p->occupancy.end()) {
                    occ = it->second;
                    known = true;
                }
            }
            if (!known) {
                if (p->jit) rc = cuda_status(jit_set_smem(p->jk, smem));
                cudaError_t e = rc ? cudaSuccess
                                   : p->jit ? jit_occupancy(p->jk, (int)block, smem, &occ, lp.variant)
                                            : exec_occupancy((int)block, smem, &occ, checked);
                if (rc == GX_OK && e != cudaSuccess) {
                    cudaGetLastError();
                    rc = GX_E_CUDA;
                }
                if (rc) return rc;
                std::lock_guard<std::mutex> g(p->ctx->mu);
                p->occupancy[key] = occ;
            }
            cap = (uint64_t)p->ctx->sms * (uint64_t)(occ > 0 ? occ : 1);
        }
        grid = std::min<uint64_t>(chunks, cap);
    }
    if (grid > 0x7FFFFFFFull) return GX_E2BIG;
    ExecParams P;
    memset(&P, 0, sizeof P);
    P.image = image;
    P.image_bytes = image_bytes;
    P.image_area = area;
    P.ctx_size = p->opts.ctx_size;
    P.ept = ept;
    P.mode = 0;
    P.events = (const uint8_t *)events;
    P.n = n;
    P.idx_base = idx_base;
    P.ret_out = (long long *)ret_out;
    P.wc_bits = wc;
    P.shard_off = shard_off;
    if (p->jit) {
        rc = cuda_status(jit_set_smem(p->jk, smem));
        if (rc == GX_OK)
            rc = cuda_status(jit_launch(p->jk, P, (unsigned)grid, block, smem, s, lp.variant));
    } else {
        rc = cuda_status(launch_exec(P, (unsigned)grid, block, smem, s, (p->opts.flags & GX_PROG_CHECKED) != 0));
    }
    if (rc == GX_OK) p->launches++;
    return rc;
}

int tuned_launch(gx_prog *p, uint64_t n, gx_launch *out) {
    int bucket = 63 - __builtin_clzll(n | 1);
    auto it = p->tuned.find(bucket);
    if (it != p->tuned.end()) {
        *out = it->second;
        return 1;
    }
    out->block = 256;
    out->ept = n >= (1ull << 24) ? 8 : 4;
    out->grid = 0;
    out->shards = 0;
    out->variant = 0;
    out->reserved = 0;
    return 0;
}

} // namespace gx

/* ================================================================ C ABI */
extern "C" {

const char *gx_strerror(int s) {
    switch (s) {
    case GX_OK: return "ok";
    case GX_ENOENT: return "no such entry";
    case GX_E2BIG: return "too big / map full";
    case GX_EAGAIN: return "no space, try again";
    case GX_ENOMEM: return "out of (budgeted) device memory";
    case GX_EFAULT: return "bad address";
    case GX_EEXIST: return "entry exists";
    case GX_EINVAL: return "invalid argument";
    case GX_ENOSPC: return "no space";
    case GX_E_VERIFY: return "program rejected by the verifier";
    case GX_E_CUDA: return "CUDA runtime error";
    case GX_E_BUDGET: return "event exceeded its instruction budget";
    case GX_E_TIMEOUT: return "bounded device wait expired";
    case GX_E_DEVICE: return "device-side invariant violated";
    case GX_E_ADMISSION: return "request exceeds the admission budget";
    case GX_E_NODEV: return "no suitable CUDA device (compute capability 10.3 required)";
    }
    return "unknown status";
}

double gx_now(void) { return now_s(); }

int gx_init(int device, uint64_t mem_budget, gx_ctx **out) {
    if (!out) return GX_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return GX_E_NODEV;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return GX_E_NODEV;
    if (prop.major != 10 || prop.minor != 3) return GX_E_NODEV;
    if (cudaSetDevice(device) != cudaSuccess) return GX_E_NODEV;
    gx_ctx *c = new gx_ctx();
    c->device = device;
    c->budget = mem_budget;
    c->sms = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    c->l2_bytes = prop.l2CacheSize;
    *out = c;
    return GX_OK;
}

int gx_shutdown(gx_ctx *c) {
    if (!c) return GX_EINVAL;
    if (c->live.load()) return GX_EINVAL;
    cudaDeviceSynchronize();
    delete c;
    return GX_OK;
}

uint64_t gx_mem_used(const gx_ctx *c) { return c ? c->used : 0; }

/* ---------------------------------------------------------------- maps */
int gx_map_create(gx_ctx *c, uint32_t type, uint32_t key_size, uint32_t value_size, uint32_t max_entries,
                  uint32_t flags, gx_map **out) {
    if (!c || !out || (flags & ~GX_MAP_F_NO_DELETE) || (flags && type != GX_MAP_HASH)) return GX_EINVAL;
    *out = nullptr;
    gx_map_spec spec = {type, key_size, value_size, max_entries, flags, 0};
    gx_dmap d;
    memset(&d, 0, sizeof d);
    d.type = type;
    d.key_size = key_size;
    d.value_size = value_size;
    d.max_entries = max_entries;
    uint64_t ctr_bytes = 256, slot_bytes = 0, value_bytes = 0;
    if (type == GX_MAP_ARRAY) {
        if (key_size != 4 || value_size < 1 || value_size > GX_MAX_VALUE || max_entries < 1) return GX_EINVAL;
        d.vstride = (uint32_t)round_up(value_size, 8);
        value_bytes = (uint64_t)max_entries * d.vstride;
    } else if (type == GX_MAP_HASH) {
        if (key_size < 1 || key_size > GX_MAX_KEY || value_size < 1 || value_size > GX_MAX_VALUE || max_entries < 1 ||
            max_entries > (1u << 30))
            return GX_EINVAL;
        uint64_t cap = 16;
        while (cap < 2ull * max_entries) cap <<= 1;
        d.vstride = (uint32_t)round_up(value_size, 8);
        d.sstride = 8 + (uint32_t)round_up(key_size, 8);
        d.mask = cap - 1;
        slot_bytes = cap * d.sstride;
        value_bytes = cap * d.vstride;
    } else if (type == GX_MAP_RINGBUF) {
        if (key_size || value_size || max_entries < 4096 || (max_entries & (max_entries - 1))) return GX_EINVAL;
        d.mask = max_entries;
        value_bytes = max_entries;
    } else {
        return GX_EINVAL;
    }
    uint64_t off_slots = ctr_bytes, off_values = round_up(off_slots + slot_bytes, 256);
    uint64_t total = off_values + value_bytes;
    gx_map *m = new gx_map();
    m->ctx = c;
    m->spec = spec;
    int rc = dalloc(c, total, &m->dmem);
    if (rc) {
        delete m;
        return rc;
    }
    m->dbytes = total;
    uint8_t *base = (uint8_t *)m->dmem;
    d.ctr = (unsigned long long *)base;
    d.slots = slot_bytes ? base + off_slots : nullptr;
    d.values = base + off_values;
    m->d = d;
    m->off_values = off_values;
    if (cudaMemset(m->dmem, 0, total) != cudaSuccess) {
        dfree(c, m->dmem, total);
        delete m;
        return GX_E_CUDA;
    }
    m->refs = 1;
    c->live++;
    *out = m;
    return GX_OK;
}

static void map_release(gx_map *m) {
    if (--m->refs > 0) return;
    gx_ctx *c = m->ctx;
    cudaDeviceSynchronize();
    dfree(c, m->dmem, m->dbytes);
    dfree(c, m->scratch, m->scratch_bytes);
    c->live--;
    delete m;
}

int gx_map_destroy(gx_map *m) {
    if (!m) return GX_EINVAL;
    map_release(m);
    return GX_OK;
}

uint64_t gx_map_bytes(const gx_map *m) { return m ? m->dbytes + m->scratch_bytes : 0; }

static int map_scratch(gx_map *m, uint64_t bytes) {
    if (m->scratch_bytes >= bytes) return GX_OK;
    dfree(m->ctx, m->scratch, m->scratch_bytes);
    m->scratch = nullptr;
    m->scratch_bytes = 0;
    int rc = dalloc(m->ctx, bytes, &m->scratch);
    if (rc) return rc;
    m->scratch_bytes = bytes;
    return GX_OK;
}

int gx_map_read(gx_map *m, void *host_out, uint64_t cap_bytes, uint64_t *n_out, void *stream) {
    if (!m || (!host_out && cap_bytes)) return GX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const gx_dmap &d = m->d;
    if (d.type == GX_MAP_ARRAY) {
        uint64_t bytes = (uint64_t)d.max_entries * d.value_size;
        if (cap_bytes < bytes) return GX_E2BIG;
        if (d.vstride == d.value_size) {
            if (cudaMemcpyAsync(host_out, d.values, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return GX_E_CUDA;
        } else {
            if (cudaMemcpy2DAsync(host_out, d.value_size, d.values, d.vstride, d.value_size, d.max_entries,
                                  cudaMemcpyDeviceToHost, s) != cudaSuccess)
                return GX_E_CUDA;
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) return GX_E_CUDA;
        if (n_out) *n_out = d.max_entries;
        return GX_OK;
    }
    if (d.type != GX_MAP_HASH) return GX_EINVAL;
    uint64_t pair = d.key_size + d.value_size;
    uint64_t cap_pairs = d.max_entries;
    int rc = map_scratch(m, 256 + cap_pairs * pair);
    if (rc) return rc;
    unsigned long long *count = (unsigned long long *)m->scratch;
    uint8_t *pairs = (uint8_t *)m->scratch + 256;
    if (cudaMemsetAsync(count, 0, 8, s) != cudaSuccess) return GX_E_CUDA;
    if (launch_hash_compact(d, pairs, count, cap_pairs, s) != cudaSuccess) return GX_E_CUDA;
    unsigned long long cnt = 0;
    if (cudaMemcpyAsync(&cnt, count, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) return GX_E_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GX_E_CUDA;
    if (cnt > cap_pairs) return GX_E_DEVICE;
    if (cnt * pair > cap_bytes) {
        if (n_out) *n_out = cnt;
        return GX_E2BIG;
    }
    if (cnt && cudaMemcpy(host_out, pairs, cnt * pair, cudaMemcpyDeviceToHost) != cudaSuccess) return GX_E_CUDA;
    if (n_out) *n_out = cnt;
    return GX_OK;
}

int gx_map_write(gx_map *m, const void *host_in, uint64_t bytes, void *stream) {
    if (!m || (!host_in && bytes)) return GX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const gx_dmap &d = m->d;
    if (d.type == GX_MAP_ARRAY) {
        if (bytes != (uint64_t)d.max_entries * d.value_size) return GX_EINVAL;
        cudaError_t e = d.vstride == d.value_size
                            ? cudaMemcpyAsync(d.values, host_in, bytes, cudaMemcpyHostToDevice, s)
                            : cudaMemcpy2DAsync(d.values, d.vstride, host_in, d.value_size, d.value_size,
                                                d.max_entries, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return GX_E_CUDA;
        return cudaStreamSynchronize(s) == cudaSuccess ? GX_OK : GX_E_CUDA;
    }
    if (d.type != GX_MAP_HASH) return GX_EINVAL;
    uint64_t pair = d.key_size + d.value_size;
    if (bytes % pair) return GX_EINVAL;
    uint64_t np = bytes / pair;
    int rc = map_scratch(m, 256 + std::max<uint64_t>(np, d.max_entries) * pair);
    if (rc) return rc;
    int *err = (int *)m->scratch;
    uint8_t *buf = (uint8_t *)m->scratch + 256;
    if (cudaMemsetAsync(err, 0, 16, s) != cudaSuccess) return GX_E_CUDA;
    if (np && cudaMemcpyAsync(buf, host_in, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return GX_E_CUDA;
    unsigned long long *stats = (unsigned long long *)((uint8_t *)m->scratch + 64);
    if (cudaMemsetAsync(stats, 0, 64, s) != cudaSuccess) return GX_E_CUDA;
    if (launch_hash_insert(d, buf, np, stats, err, s) != cudaSuccess) return GX_E_CUDA;
    int herr = 0;
    if (cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return GX_E_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GX_E_CUDA;
    return herr;
}

int gx_map_clear(gx_map *m, void *stream) {
    if (!m) return GX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t bytes = m->d.type == GX_MAP_RINGBUF ? 256 : m->dbytes;
    return cudaMemsetAsync(m->dmem, 0, bytes, s) == cudaSuccess ? GX_OK : GX_E_CUDA;
}

int gx_ringbuf_drain(gx_map *rb, void *host_out, uint64_t cap, uint64_t *bytes_out, uint64_t *dropped, void *stream) {
    if (!rb || rb->d.type != GX_MAP_RINGBUF || (!host_out && cap)) return GX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long ctr[2] = {0, 0};
    if (cudaMemcpyAsync(ctr, rb->d.ctr, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess) return GX_E_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GX_E_CUDA;
    uint64_t used = std::min<uint64_t>(ctr[0], rb->d.mask);
    std::vector<uint8_t> raw(used);
    if (used && cudaMemcpy(raw.data(), rb->d.values, used, cudaMemcpyDeviceToHost) != cudaSuccess) return GX_E_CUDA;
    /* pack committed records; a PAD record marks where the reservations stopped fitting */
    uint64_t w = 0;
    for (uint64_t pos = 0; pos + GX_RB_HDR <= used;) {
        uint32_t len, flags;
        memcpy(&len, &raw[pos], 4);
        memcpy(&flags, &raw[pos + 4], 4);
        if (flags & GX_RB_PAD) break;
        uint64_t rec = GX_RB_HDR + round_up(len, 8);
        if (pos + rec > used) break;
        if (!(flags & GX_RB_DISCARDED)) {
            if (w + rec > cap) {
                if (bytes_out) *bytes_out = w;
                return GX_E2BIG;
            }
            memcpy((uint8_t *)host_out + w, &raw[pos], rec);
            w += rec;
        }
        pos += rec;
    }
    if (cudaMemsetAsync(rb->d.ctr, 0, 16, s) != cudaSuccess) return GX_E_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GX_E_CUDA;
    if (bytes_out) *bytes_out = w;
    if (dropped) *dropped = ctr[1];
    return GX_OK;
}

/* ---------------------------------------------------------------- programs */
int gx_verify(const uint64_t *insns, uint32_t n, const gx_map_spec *maps, uint32_t n_maps, const gx_prog_opts *opts,
              char *log, size_t log_len) {
    if (!insns || !opts || (n_maps && !maps)) return GX_EINVAL;
    VerifyOut v;
    int rc = verify_program(insns, n, maps, n_maps, *opts, v);
    if (log && log_len) {
        size_t k = std::min(log_len - 1, v.log.size());
        memcpy(log, v.log.data(), k);
        log[k] = 0;
    }
    return rc;
}

int gx_analyze(const uint64_t *insns, uint32_t n, const gx_map_spec *maps, uint32_t n_maps, const gx_prog_opts *opts,
               gx_analysis *out, char *log, size_t log_len) {
    if (!insns || !opts || !out || (n_maps && !maps)) return GX_EINVAL;
    VerifyOut v;
    int rc = verify_program(insns, n, maps, n_maps, *opts, v);
    memset(out, 0, sizeof *out);
    if (rc == GX_OK) {
        out->insns_processed = v.insns_processed;
        out->stack_depth = v.stack_depth;
        for (uint32_t m = 0; m < n_maps && m < v.map_use.size(); m++)
            if (v.map_use[m].combinable() && maps[m].type != GX_MAP_RINGBUF) out->combinable_maps |= 1u << m;
    }
    if (log && log_len) {
        size_t k = std::min(log_len - 1, v.log.size());
        memcpy(log, v.log.data(), k);
        log[k] = 0;
    }
    return rc;
}

int gx_merge_ops(const uint64_t *insns, uint32_t n, const gx_map_spec *maps, uint32_t n_maps,
                 const gx_prog_opts *opts, uint32_t map_index, uint8_t *word_ops, uint8_t *insert_value,
                 uint32_t *has_insert, char *log, size_t log_len) {
    if (!insns || !opts || !word_ops || (n_maps && !maps) || map_index >= n_maps) return GX_EINVAL;
    static_assert(GX_MAP_HASH_T == GX_MAP_HASH && GX_MAP_RINGBUF_T == GX_MAP_RINGBUF, "map types of gx_layout.h");
    static_assert(UC_ADD == GX_MERGE_ADD && UC_OR == GX_MERGE_OR && UC_AND == GX_MERGE_AND && UC_XOR == GX_MERGE_XOR &&
                      UC_MAX == GX_MERGE_MAX && UC_MIN == GX_MERGE_MIN && UC_W8 == GX_MERGE_W8,
                  "the ABI's merge codes are the verifier's update classes");
    gx_prog_opts det = *opts;
    det.deterministic = 1;
    VerifyOut v;
    int rc = verify_program(insns, n, maps, n_maps, det, v);
    std::string msg = v.log;
    const uint32_t words = (maps[map_index].value_size + 3) / 4;
    if (rc == GX_OK && maps[map_index].type != GX_MAP_RINGBUF) {
        const MapUse &u = v.map_use[map_index];
        if (u.merge_mixed) {
            rc = GX_EINVAL;
            msg = "map " + std::to_string(map_index) + ": a word is updated at two widths; its copies cannot be merged";
        } else if (u.insert_conflict) {
            rc = GX_EINVAL;
            msg = "map " + std::to_string(map_index) + ": inserts of different constants; its copies cannot be merged";
        } else {
            memcpy(word_ops, u.merge_op.data(), words);
            if (insert_value) {
                memset(insert_value, 0, maps[map_index].value_size);
                if (u.insert_seen) memcpy(insert_value, u.insert.data(), maps[map_index].value_size);
            }
            if (has_insert) *has_insert = u.insert_seen ? 1u : 0u;
        }
    } else if (rc == GX_OK) {
        memset(word_ops, 0, words);
        if (has_insert) *has_insert = 0;
    }
    if (log && log_len) {
        size_t k = std::min(log_len - 1, msg.size());
        memcpy(log, msg.data(), k);
        log[k] = 0;
    }
    return rc;
}

int gx_verify_simt(const uint64_t *insns, uint32_t n, const gx_map_spec *maps, uint32_t n_maps,
                   const gx_prog_opts *opts, const gx_simt_spec *simt, gx_simt_report *out, char *log, size_t log_len) {
    if (out) {
        memset(out, 0, sizeof *out);
        out->violation_pc = -1;
    }
    if (!insns || !opts || !simt || (n_maps && !maps) || simt->reserved) return GX_EINVAL;
    if (opts->ctx_size < 8 || opts->ctx_size > GX_MAX_CTX) return GX_EINVAL;
    const SimtIn in = simt_in(*simt, opts->ctx_size);
    VerifyOut v;
    int rc = verify_program(insns, n, maps, n_maps, *opts, v, &in);
    if (rc == GX_E_VERIFY && v.simt.violation == GX_SIMT_V_NONE) {
        v.simt.violation = GX_SIMT_V_VERIFY;
        v.simt.pc = v.fail_pc;
    }
    if (out) {
        out->max_insns = v.simt.max_insns;
        out->max_helper_calls = v.simt.max_helpers;
        out->max_mem_ops = v.simt.max_mem;
        out->uniform_branches = v.simt.uniform_branches;
        out->varying_insns = v.simt.varying_insns;
        out->violation_pc = rc == GX_OK ? -1 : v.simt.pc;
        out->violation = rc == GX_OK ? GX_SIMT_V_NONE : v.simt.violation;
    }
    if (log && log_len) {
        size_t k = std::min(log_len - 1, v.log.size());
        memcpy(log, v.log.data(), k);
        log[k] = 0;
    }
    return rc;
}

int gx_verify_load(gx_ctx *c, const uint64_t *insns, uint32_t n, gx_map *const *maps, uint32_t n_maps,
                   const gx_prog_opts *opts, gx_prog **out, char *log, size_t log_len) {
    if (!c || !insns || !opts || !out || (n_maps && !maps)) return GX_EINVAL;
    if (opts->flags & ~(GX_PROG_JIT | GX_PROG_CHECKED)) return GX_EINVAL;
    if ((opts->flags & GX_PROG_JIT) && (opts->flags & GX_PROG_CHECKED)) return GX_EINVAL; /* checks: interpreter only */
    *out = nullptr;
    std::vector<gx_map_spec> specs(n_maps);
    for (uint32_t i = 0; i < n_maps; i++) {
        if (!maps[i] || maps[i]->ctx != c) return GX_EINVAL;
        specs[i] = maps[i]->spec;
    }
    VerifyOut v;
    std::string msg;
    int rc = verify_program(insns, n, specs.data(), n_maps, *opts, v);
    msg = v.log;
    gx_prog *p = nullptr;
    if (rc == GX_OK) {
        p = new gx_prog();
        p->ctx = c;
        p->opts = *opts;
        rc = decode_program(insns, n, v, p->uops, msg);
        if (rc == GX_OK) {
            p->jp.insns.assign(insns, insns + n);
            p->jp.info = v.info;
            p->jp.maps = specs;
            p->jp.use = v.map_use;
            p->jp.ctx_size = opts->ctx_size;
            p->jp.budget = opts->insn_budget ? opts->insn_budget : (1ull << 16);
            if (opts->flags & GX_PROG_JIT) {
                p->jp.max_path = path_bound(insns, n, specs.data(), n_maps, *opts);
                rc = jit_build({&p->jp}, p->jk, msg);
                p->jit = rc == GX_OK;
            }
        }
    }
    if (log && log_len) {
        size_t k = std::min(log_len - 1, msg.size());
        memcpy(log, msg.data(), k);
        log[k] = 0;
    }
    if (rc) {
        delete p;
        return rc;
    }
    for (uint32_t i = 0; i < n_maps; i++) {
        p->maps.push_back(maps[i]);
        maps[i]->refs++;
    }
    std::vector<gx_dmap> descs;
    for (auto *m : p->maps) descs.push_back(m->d);
    uint64_t img_guess = round_up(sizeof(gx_dprog_hdr) + descs.size() * sizeof(gx_dmap) + p->uops.size() * 8, 16);
    uint64_t stats_off = round_up(img_guess, 256);
    p->dbytes = stats_off + 256;
    rc = dalloc(c, p->dbytes, &p->dmem);
    if (rc) {
        for (auto *m : p->maps) map_release(m);
        delete p;
        return rc;
    }
    p->dstats = (unsigned long long *)((uint8_t *)p->dmem + stats_off);
    std::vector<uint8_t> img = build_image(p, descs, p->dstats);
    p->image_bytes = (uint32_t)img.size();
    if (cudaMemcpy(p->dmem, img.data(), img.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(p->dstats, 0, 256) != cudaSuccess) {
        dfree(c, p->dmem, p->dbytes);
        for (auto *m : p->maps) map_release(m);
        delete p;
        return GX_E_CUDA;
    }
    if (p->image_bytes > GX_MAX_IMAGE) {
        dfree(c, p->dmem, p->dbytes);
        for (auto *m : p->maps) map_release(m);
        delete p;
        return GX_E2BIG;
    }
    c->live++;
    *out = p;
    return GX_OK;
}

int gx_prog_destroy(gx_prog *p) {
    if (!p) return GX_EINVAL;
    gx_ctx *c = p->ctx;
    cudaDeviceSynchronize();
    dfree(c, p->dmem, p->dbytes);
    for (int i = 0; i < 2; i++) dfree(c, p->stage[i], p->stage_bytes);
    dfree(c, p->ret_stage[0], p->ret_stage_bytes);
    dfree(c, p->ret_stage[1], p->ret_stage_bytes);
    for (int i = 0; i < 2; i++)
        if (p->streams[i]) cudaStreamDestroy(p->streams[i]);
    for (auto *m : p->maps) map_release(m);
    c->live--;
    delete p;
    return GX_OK;
}

/* upload a verified program's image (header, map table, micro-ops) and take its map references */
static int upload_program(gx_ctx *c, gx_prog *p, gx_map *const *maps, uint32_t n_maps) {
    for (uint32_t i = 0; i < n_maps; i++) {
        p->maps.push_back(maps[i]);
        maps[i]->refs++;
    }
    std::vector<gx_dmap> descs;
    for (auto *m : p->maps) descs.push_back(m->d);
    uint64_t img_guess = round_up(sizeof(gx_dprog_hdr) + descs.size() * sizeof(gx_dmap) + p->uops.size() * 8, 16);
    uint64_t stats_off = round_up(img_guess, 256);
    p->dbytes = stats_off + 256;
    int rc = dalloc(c, p->dbytes, &p->dmem);
    if (rc) {
        for (auto *m : p->maps) map_release(m);
        return rc;
    }
    p->dstats = (unsigned long long *)((uint8_t *)p->dmem + stats_off);
    std::vector<uint8_t> img = build_image(p, descs, p->dstats);
    p->image_bytes = (uint32_t)img.size();
    if (p->image_bytes > GX_MAX_IMAGE) rc = GX_E2BIG;
    else if (cudaMemcpy(p->dmem, img.data(), img.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemset(p->dstats, 0, 256) != cudaSuccess)
        rc = GX_E_CUDA;
    if (rc) {
        dfree(c, p->dmem, p->dbytes);
        for (auto *m : p->maps) map_release(m);
        return rc;
    }
    c->live++;
    return GX_OK;
}

int gx_verify_load_simt(gx_ctx *c, const uint64_t *insns, uint32_t n, gx_map *const *maps, uint32_t n_maps,
                        const gx_prog_opts *opts, const gx_simt_spec *simt, gx_prog **out, char *log,
                        size_t log_len) {
    if (!c || !insns || !opts || !simt || !out || (n_maps && !maps) || simt->reserved) return GX_EINVAL;
    if (opts->flags != GX_PROG_JIT) return GX_EINVAL; /* the warp-level form exists only as specialised code */
    if (opts->ctx_size < 8 || opts->ctx_size > GX_MAX_CTX) return GX_EINVAL;
    *out = nullptr;
    std::vector<gx_map_spec> specs(n_maps);
    for (uint32_t i = 0; i < n_maps; i++) {
        if (!maps[i] || maps[i]->ctx != c) return GX_EINVAL;
        specs[i] = maps[i]->spec;
    }
    const SimtIn in = simt_in(*simt, opts->ctx_size);
    VerifyOut v;
    int rc = verify_program(insns, n, specs.data(), n_maps, *opts, v, &in);
    std::string msg = v.log;
    gx_prog *p = nullptr;
    if (rc == GX_OK) {
        p = new gx_prog();
        p->ctx = c;
        p->opts = *opts;
        /* no micro-ops: the interpreter never runs this form (batches and servers refuse to) */
        p->jp.insns.assign(insns, insns + n);
        p->jp.info = v.info;
        p->jp.maps = specs;
        p->jp.use = v.map_use;
        p->jp.ctx_size = opts->ctx_size;
        p->jp.budget = opts->insn_budget ? opts->insn_budget : (1ull << 16);
        p->jp.max_path = v.simt.max_insns; /* the SIMT pass counted every path */
        p->jp.warp = true;
        rc = jit_build({&p->jp}, p->jk, msg);
        p->jit = rc == GX_OK;
    }
    if (log && log_len) {
        size_t k = std::min(log_len - 1, msg.size());
        memcpy(log, msg.data(), k);
        log[k] = 0;
    }
    if (rc == GX_OK) rc = upload_program(c, p, maps, n_maps);
    if (rc) {
        delete p;
        return rc;
    }
    *out = p;
    return GX_OK;
}

uint32_t gx_prog_uops(const gx_prog *p) { return p ? (uint32_t)(p->uops.size() / 2) : 0; } /* two words each */

/* ---------------------------------------------------------------- runs */
int gx_run_batch_ex(gx_prog *p, const void *events, uint64_t n, uint64_t idx_base, int64_t *ret_out,
                    const gx_launch *lp, void *stream) {
    TraceRange tr("gx_run_batch");
    if (!p || (!events && n)) return GX_EINVAL;
    if (((uintptr_t)events) & 15) return GX_EINVAL;
    if (n == 0) return GX_OK;
    gx_launch l{};
    if (lp) l = *lp;
    else tuned_launch(p, n, &l);
    return launch_plain(p, (const uint8_t *)p->dmem, p->image_bytes, events, n, idx_base, ret_out, l,
                        (cudaStream_t)stream);
}

int gx_run_batch(gx_prog *p, const void *events, uint64_t n, void *stream) {
    return gx_run_batch_ex(p, events, n, 0, nullptr, nullptr, stream);
}

int gx_run_batch_host(gx_prog *p, const void *events_host, uint64_t n, int64_t *ret_out_host) {
    TraceRange tr("gx_run_batch_host");
    if (!p || (!events_host && n)) return GX_EINVAL;
    if (n == 0) return GX_OK;
    const uint64_t cs = p->opts.ctx_size;
    const uint64_t chunk = std::min<uint64_t>(n, GX_HOST_CHUNK_EVENTS);
    if (p->stage_bytes < chunk * cs) {
        for (int i = 0; i < 2; i++) {
            dfree(p->ctx, p->stage[i], p->stage_bytes);
            p->stage[i] = nullptr;
        }
        p->stage_bytes = 0;
        for (int i = 0; i < 2; i++) {
            int rc = dalloc(p->ctx, chunk * cs, &p->stage[i]);
            if (rc) return rc;
        }
        p->stage_bytes = chunk * cs;
    }
    if (ret_out_host && p->ret_stage_bytes < chunk * 8) {
        for (int i = 0; i < 2; i++) {
            dfree(p->ctx, p->ret_stage[i], p->ret_stage_bytes);
            p->ret_stage[i] = nullptr;
        }
        p->ret_stage_bytes = 0;
        for (int i = 0; i < 2; i++) {
            int rc = dalloc(p->ctx, chunk * 8, &p->ret_stage[i]);
            if (rc) return rc;
        }
        p->ret_stage_bytes = chunk * 8;
    }
    for (int i = 0; i < 2; i++)
        if (!p->streams[i] && cudaStreamCreateWithFlags(&p->streams[i], cudaStreamNonBlocking) != cudaSuccess)
            return GX_E_CUDA;
    gx_launch l{};
    tuned_launch(p, chunk, &l);
    int rc = GX_OK;
    for (uint64_t off = 0, k = 0; off < n; off += chunk, k++) {
        const int b = (int)(k & 1);
        cudaStream_t s = p->streams[b];
        uint64_t cnt = std::min(chunk, n - off);
        if (cudaMemcpyAsync(p->stage[b], (const uint8_t *)events_host + off * cs, cnt * cs, cudaMemcpyHostToDevice,
                            s) != cudaSuccess) {
            rc = GX_E_CUDA;
            break;
        }
        int64_t *rdev = ret_out_host ? (int64_t *)p->ret_stage[b] : nullptr;
        rc = launch_plain(p, (const uint8_t *)p->dmem, p->image_bytes, p->stage[b], cnt, off, rdev, l, s);
        if (rc) break;
        if (ret_out_host &&
            cudaMemcpyAsync(ret_out_host + off, rdev, cnt * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            rc = GX_E_CUDA;
            break;
        }
    }
    for (int i = 0; i < 2; i++)
        if (cudaStreamSynchronize(p->streams[i]) != cudaSuccess) rc = rc ? rc : GX_E_CUDA;
    return rc;
}

int gx_last_status(gx_prog *p, gx_run_stats *out, int reset, void *stream) {
    if (!p || !out) return GX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long st[GX_STAT_WORDS];
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_status(cudaGetLastError());
    if (cudaMemcpy(st, p->dstats, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess) return GX_E_CUDA;
    memset(out, 0, sizeof *out);
    out->status = (int32_t)(uint32_t)st[GX_STAT_STATUS];
    out->fault_pc = (uint32_t)st[GX_STAT_FAULT];
    if (out->status == GX_E_TIMEOUT && p->sched_lc) p->ctx->launch_control_timed_out = true;
    out->budget_trips = st[GX_STAT_BUDGET];
    out->waits_expired = st[GX_STAT_WAITS];
    out->launches = p->launches;
    if (reset && cudaMemset(p->dstats, 0, sizeof st) != cudaSuccess) return GX_E_CUDA;
    return GX_OK;
}

static int autotune_impl(gx_prog *p, const void *events, uint64_t n, cudaStream_t s, gx_launch *best, bool policy_only);

/*
 * What a cached choice is valid for: the program (its micro-ops, and for a specialised
 * program its kernel key, which covers the generated source and the device headers), its
 * maps and options, the device (name and SM count) and this engine build.
 */
static uint64_t tune_identity(gx_prog *p) {
    uint64_t h = tune_fnv(p->uops.data(), p->uops.size() * 8);
    const uint32_t o[3] = {p->opts.ctx_size, p->opts.deterministic, p->opts.flags};
    h = tune_fnv(o, sizeof o, h);
    for (auto *m : p->maps) h = tune_fnv(&m->spec, sizeof m->spec, h);
    if (p->jit) h = tune_fnv(p->jk.key.data(), p->jk.key.size(), h);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, p->ctx->device) == cudaSuccess) {
        h = tune_fnv(prop.name, strnlen(prop.name, sizeof prop.name), h);
        h = tune_fnv(&prop.multiProcessorCount, sizeof prop.multiProcessorCount, h);
    } else {
        cudaGetLastError();
    }
    static const char build[] = __DATE__ " " __TIME__;
    return tune_fnv(build, sizeof build, h);
}

/* the autotuner behind the on-disk cache (GX_TUNE_CACHE): a stored choice is used as is */
static int autotune_cached(gx_prog *p, const void *events, uint64_t n, cudaStream_t s, gx_launch *best,
                           bool policy_only) {
    if (!p || !events || n == 0) return GX_EINVAL;
    const char *dir = getenv("GX_TUNE_CACHE");
    const int bucket = 63 - __builtin_clzll(n | 1);
    std::string path;
    if (dir && *dir) {
        path = tune_cache_path(dir, tune_identity(p), bucket, policy_only);
        gx_launch l;
        if (tune_cache_load(path, &l)) {
            if (!policy_only) p->tuned[bucket] = l;
            p->pref_shards = l.shards;
            p->pref_tuned = true;
            if (best) *best = l;
            return GX_OK;
        }
    }
    gx_launch chosen{};
    const int rc = autotune_impl(p, events, n, s, &chosen, policy_only);
    if (rc == GX_OK && !path.empty()) {
        mkdir(dir, 0755);
        tune_cache_store(path, chosen);
    }
    if (best) *best = chosen;
    return rc;
}

static int autotune_impl(gx_prog *p, const void *events, uint64_t n, cudaStream_t s, gx_launch *best, bool policy_only) {
    if (!p || (!events && n)) return GX_EINVAL;
    if (n == 0) return GX_EINVAL;
    gx_ctx *c = p->ctx;
    /* scratch copies of every map, so tuning runs leave the real maps untouched */
    std::vector<void *> clones;
    std::vector<uint64_t> clone_bytes;
    std::vector<gx_dmap> descs;
    /* ring buffers restart from the real ring's head before every tuning launch: a ring that
       fills up during tuning would make the configurations tried last look cheap */
    std::vector<std::pair<void *, const void *>> rings;
    int rc = GX_OK;
    for (auto *m : p->maps) {
        void *cl = nullptr;
        rc = dalloc(c, m->dbytes, &cl);
        if (rc) break;
        clones.push_back(cl);
        clone_bytes.push_back(m->dbytes);
        if (cudaMemcpyAsync(cl, m->dmem, m->dbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            rc = GX_E_CUDA;
            break;
        }
        gx_dmap d = m->d;
        uint8_t *base = (uint8_t *)cl;
        d.ctr = (unsigned long long *)base;
        if (m->d.type == GX_MAP_RINGBUF) rings.push_back({base, m->dmem});
        if (d.slots) d.slots = base + ((uint8_t *)m->d.slots - (uint8_t *)m->dmem);
        d.values = base + m->off_values;
        descs.push_back(d);
    }
    void *timg = nullptr;
    uint64_t timg_bytes = 0;
    if (rc == GX_OK) {
        std::vector<uint8_t> img0 = build_image(p, descs, nullptr);
        timg_bytes = round_up(img0.size(), 256) + 256;
        rc = dalloc(c, timg_bytes, &timg);
        if (rc == GX_OK) {
            unsigned long long *tstats = (unsigned long long *)((uint8_t *)timg + round_up(img0.size(), 256));
            std::vector<uint8_t> img = build_image(p, descs, tstats);
            if (cudaMemcpyAsync(timg, img.data(), img.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaMemsetAsync(tstats, 0, 256, s) != cudaSuccess)
                rc = GX_E_CUDA;
            cudaStreamSynchronize(s);
        }
    }
    gx_launch chosen{};
    tuned_launch(p, n, &chosen);
    if (rc == GX_OK) {
        /* policy only: the sharding choice at one shape on a smaller sample (batch planning) */
        const uint64_t sample = std::min<uint64_t>(n, policy_only ? (1ull << 21) : (1ull << 26));
        const std::vector<uint32_t> blocks = policy_only ? std::vector<uint32_t>{256} : std::vector<uint32_t>{128, 256};
        /* (events per thread, grid): one wave of blocks looping over chunks of every size, and
           one block per chunk at two sizes */
        const std::vector<std::pair<uint32_t, uint32_t>> epts =
            policy_only ? std::vector<std::pair<uint32_t, uint32_t>>{{8, 0}}
                        : std::vector<std::pair<uint32_t, uint32_t>>{{1, 0}, {2, 0}, {4, 0}, {8, 0}, {16, 0}, {32, 0},
                                                                     {64, 0}, {8, GX_GRID_PER_CHUNK},
                                                                     {32, GX_GRID_PER_CHUNK}};
        /* specialised single programs: every compiled entry, wide to register-capped */
        std::vector<uint32_t> variants = {0};
        if (!policy_only && p->jit) {
            variants.clear();
            for (uint32_t v = 1; v < 5; v++)
                if (p->jk.variant[v]) variants.push_back(v);
            if (variants.empty()) variants = {0};
        }
        float best_ms = 1e30f;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        uint32_t img_bytes = (uint32_t)round_up(sizeof(gx_dprog_hdr) + descs.size() * sizeof(gx_dmap) + p->uops.size() * 8, 16);
        /* map-sharding width: off, and the combining caches at 64 and at their widest */
        std::vector<uint32_t> widths = {0};
        if (p->jit && p->jk.shard_bytes) {
            widths = {GX_SHARDS_OFF, 0};
            if (p->jk.wc_max_bits > 1) widths.push_back(GX_SHARDS_AGG); /* programs with a cache */
            if (p->jk.wc_max_bits > WC_DEFAULT_BITS) widths.push_back(p->jk.wc_max_bits); /* the widest cache */
        }
        auto rewind = [&] {
            for (auto &r : rings) cudaMemcpyAsync(r.first, r.second, 16, cudaMemcpyDeviceToDevice, s);
        };
        /* the median of `reps` timed launches of l over m events (after one untimed launch):
           one slow launch (a clock step, another stream) does not rank a shape down, and a
           shape whose launches are only sometimes fast is not ranked up; < 0 if it cannot
           launch */
        auto timed = [&](const gx_launch &l, uint64_t m, int reps) -> float {
            rewind();
            if (launch_plain(p, (const uint8_t *)timg, img_bytes, events, m, 0, nullptr, l, s)) return -1.0f;
            std::vector<float> t;
            for (int r = 0; r < reps; r++) {
                rewind();
                cudaEventRecord(e0, s);
                launch_plain(p, (const uint8_t *)timg, img_bytes, events, m, 0, nullptr, l, s);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                t.push_back(ms);
            }
            std::sort(t.begin(), t.end());
            return t[t.size() / 2];
        };
        std::vector<std::pair<float, gx_launch>> ranked;
        for (uint32_t b : blocks)
            for (const auto &eg : epts) for (uint32_t w : widths) for (uint32_t v : variants) {
                const gx_launch l = {b, eg.first, eg.second, w, v, 0};
                const float ms = timed(l, sample, 3);
                if (ms >= 0) ranked.push_back({ms, l});
            }
        std::stable_sort(ranked.begin(), ranked.end(),
                         [](const std::pair<float, gx_launch> &a, const std::pair<float, gx_launch> &b) {
                             return a.first < b.first;
                         });
        /* close shapes can swap places in one pass (and a sample smaller than the batch can rank
           them wrongly): the best three race again over the whole batch */
        if (!ranked.empty()) chosen = ranked[0].second;
        if (ranked.size() > 1 && (!policy_only || n > sample)) {
            for (size_t k = 0; k < ranked.size() && k < 3; k++) {
                const float ms = timed(ranked[k].second, n, policy_only ? 2 : 5);
                if (ms >= 0 && ms < best_ms) {
                    best_ms = ms;
                    chosen = ranked[k].second;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (!policy_only) p->tuned[63 - __builtin_clzll(n | 1)] = chosen;
        p->pref_shards = chosen.shards;
        p->pref_tuned = true;
        if (cudaGetLastError() != cudaSuccess) rc = GX_E_CUDA;
    }
    cudaStreamSynchronize(s);
    for (size_t i = 0; i < clones.size(); i++) dfree(c, clones[i], clone_bytes[i]);
    dfree(c, timg, timg_bytes);
    if (best) *best = chosen;
    return rc;
}

int gx_autotune(gx_prog *p, const void *events, uint64_t n, void *stream, gx_launch *best) {
    TraceRange tr("gx_autotune");
    return autotune_cached(p, events, n, (cudaStream_t)stream, best, false);
}

} /* extern "C" */

namespace gx {
int tune_shards(gx_prog *p, const void *events, uint64_t n, cudaStream_t s) {
    if (!p->jit || !p->jk.shard_bytes) {
        p->pref_tuned = true;
        p->pref_shards = 0;
        return GX_OK;
    }
    return autotune_cached(p, events, n, s, nullptr, true);
}
} // namespace gx
