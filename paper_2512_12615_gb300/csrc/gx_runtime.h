/* Host-side object definitions behind the opaque handles of include/gx.h. */
#ifndef GX_RUNTIME_H
#define GX_RUNTIME_H

#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "gx_internal.h"
#include "gx_jit.h"

#define GX_MAX_BLOCK 256                   /* the exec kernel's launch bound */
#define GX_MAX_IMAGE (160u * 1024u)        /* decoded image must fit in shared memory */
#define GX_HOST_CHUNK_EVENTS (8ull << 20)  /* events per staged chunk of gx_run_batch_host */

struct gx_ctx {
    int device = 0;
    uint64_t budget = 0;
    uint64_t used = 0;
    int sms = 0;
    uint64_t smem_optin = 0;
    uint64_t smem_attr = 0;
    uint64_t l2_bytes = 0;
    std::atomic<int> live{0};
    std::mutex mu;
    /* a cancel response of cluster launch control did not arrive in time: launch control
       stays refused on this context (a late response may still land in a block's shared
       memory, so the results of that launch and of its SMs' later blocks are suspect) */
    std::atomic<bool> launch_control_timed_out{false};
};

struct gx_map {
    gx_ctx *ctx = nullptr;
    gx_map_spec spec{};
    int refs = 0;
    void *dmem = nullptr; /* [counters 256 B][hash slots][values] */
    uint64_t dbytes = 0;
    uint64_t off_values = 0;
    gx_dmap d{};
    void *scratch = nullptr; /* snapshot / restore staging */
    uint64_t scratch_bytes = 0;
};

struct gx_prog {
    gx_ctx *ctx = nullptr;
    gx_prog_opts opts{};
    std::vector<gx_map *> maps;
    std::vector<uint64_t> uops;
    void *dmem = nullptr; /* [image][stats] */
    uint64_t dbytes = 0;
    uint32_t image_bytes = 0;
    unsigned long long *dstats = nullptr;
    uint64_t launches = 0;
    std::map<int, gx_launch> tuned; /* log2(n) bucket -> shape */
    std::map<uint64_t, int> occupancy; /* (block, shared bytes, variant) -> resident blocks per SM */
    bool sched_lc = false; /* steers a batch under cluster launch control (gx_batch_set_sched) */
    uint32_t pref_shards = 0;       /* tuned gx_launch.shards of this program in batches and ticks */
    bool pref_tuned = false;
    /* load-time specialisation (GX_PROG_JIT) */
    gx::JitProgram jp;
    gx::JitKernel jk;
    bool jit = false;
    /* gx_run_batch_host staging */
    void *stage[2] = {nullptr, nullptr};
    uint64_t stage_bytes = 0;
    void *ret_stage[2] = {nullptr, nullptr};
    uint64_t ret_stage_bytes = 0;
    cudaStream_t streams[2] = {nullptr, nullptr};
};

namespace gx {
double now_s();
int dalloc(gx_ctx *c, uint64_t bytes, void **out);
void dfree(gx_ctx *c, void *p, uint64_t bytes);
int cuda_status(cudaError_t e);
uint64_t exec_smem(uint32_t image_area, uint32_t block, uint32_t ctx_size);
bool shards_valid(uint32_t shards);
uint32_t shards_param(uint32_t shards, uint32_t default_bits);
/* choose p->pref_shards by timing OFF / default / aggregated misses on a sample (scratch maps) */
int tune_shards(gx_prog *p, const void *events, uint64_t n, cudaStream_t s);
int ensure_smem(gx_ctx *c, uint64_t smem);
int tuned_launch(gx_prog *p, uint64_t n, gx_launch *out);
} // namespace gx

#endif
