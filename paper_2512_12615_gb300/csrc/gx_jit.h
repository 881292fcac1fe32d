/* Load-time specialisation of programs (jit.cpp). */
#ifndef GX_JIT_H
#define GX_JIT_H

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "gx_internal.h"
#include "gx_kernels.h"

namespace gx {

/* what the code generator needs from a verified program */
struct JitProgram {
    std::vector<uint64_t> insns;
    std::vector<InsnInfo> info;
    std::vector<gx_map_spec> maps; /* layouts become compile-time constants */
    std::vector<MapUse> use;       /* per map: may its updates be combined per block? */
    uint32_t ctx_size = 8;         /* bytes per event record */
    uint64_t budget = 1ull << 16;
    /* the longest path's instruction count, from the verifier (0: unknown); when it is
       within `budget`, no event can reach the back-jump budget and the check is left out */
    uint64_t max_path = 0;
    bool warp = false; /* a SIMT-verified warp-level handler: shared effects once per warp, by its leader lane */
};

struct JitKernel {
    cudaKernel_t kernel = nullptr;      /* the default entry (GX_VARIANT_4 for one program, capped for several) */
    cudaKernel_t variant[5] = {};       /* entries by GX_VARIANT_* (index 0 unused); null where not compiled */
    std::string key;
    size_t smem_attr = 0;
    uint32_t shard_bytes = 0; /* shared memory of the block-private combining area at its widest (0: none) */
    uint32_t wc_max_bits = 0; /* widest combining cache (0: no combinable map; 1: private arrays only) */
    uint32_t shard_bytes_for[11] = {}; /* the area's bytes when caches are 2^b entries wide (max over programs) */
};

/* combining-cache width when a launch leaves it to the default: 256 entries */
const uint32_t WC_DEFAULT_BITS = 8;
inline uint32_t wc_default_bits(const JitKernel &k) { return k.wc_max_bits < WC_DEFAULT_BITS ? k.wc_max_bits : WC_DEFAULT_BITS; }
inline uint32_t wc_area_bytes(const JitKernel &k, uint32_t bits) { return k.shard_bytes_for[bits > 10 ? 10 : bits]; }

/*
 * The block-private combining layout of one program (shared memory): private copies of
 * small array maps at fixed offsets, then one cache per other map whose 2^b entries of
 * {u64 tag, accumulators} follow each other; b = min(runtime width, the cache's max), so
 * the caches' offsets and the area's size follow the width chosen at launch.
 */
struct ShardMap {
    int map = -1;
    bool full = false;       /* whole private copy of an array map, else a tagged cache */
    uint32_t acc_off = 0;    /* full: offset of the copy (values laid out with the map's stride) */
    uint32_t stride = 0;     /* value stride (bytes, multiple of 8) */
    uint32_t max_bits = 0;   /* cache: log2 entries at most */
    uint32_t n_values = 0;   /* full: max_entries */
    std::vector<uint8_t> op; /* per 4-byte word of a value: UpdClass | UC_W8 */
    uint32_t sites = 0;      /* update instructions that reach it at a known offset */
};
struct ShardPlan {
    std::vector<ShardMap> maps; /* private copies first, then caches */
    uint32_t full_bytes = 0;    /* bytes of the private copies */
    uint32_t max_bits = 0;
    uint32_t bytes_for[11] = {}; /* area bytes at each width */
    uint32_t bytes_at(uint32_t bits) const;
    const ShardMap *find(int m) const {
        for (const ShardMap &s : maps)
            if (s.map == m) return &s;
        return nullptr;
    }
};
ShardPlan plan_shards(const JitProgram &p);
/* the verifier's bound on any path's instruction count (0 if it cannot give one) */
uint64_t path_bound(const uint64_t *insns, uint32_t n, const gx_map_spec *maps, uint32_t n_maps,
                    const gx_prog_opts &opts);

/*
 * compile (or fetch from the caches) one kernel running progs[slot] for chunk slot `slot`;
 * with `sched`, the kernel is the work-stealing form steered by that scheduling program
 */
int jit_build(const std::vector<const JitProgram *> &progs, JitKernel &out, std::string &log,
              const JitProgram *sched = nullptr);
/*
 * Is this program fit to steer a batch (gx_batch_set_sched)?  ctx_size GX_SCHED_CTX and a
 * warp-uniform handler within `limits` (nullable: the GX_SCHED_MAX_* budget).  GX_OK,
 * GX_EINVAL or GX_E_VERIFY; `v` gets the verifier's findings.
 */
int check_sched_program(const uint64_t *insns, uint32_t n, const gx_map_spec *maps, uint32_t n_maps,
                        const gx_prog_opts &opts, const gx_simt_spec *limits, VerifyOut &v);
/* the entry of a GX_VARIANT_* (0 or one not compiled: the default entry) */
inline cudaKernel_t jit_entry(const JitKernel &k, uint32_t variant) {
    return variant < 5 && k.variant[variant] ? k.variant[variant] : k.kernel;
}
cudaError_t jit_launch(const JitKernel &k, const ExecParams &p, unsigned grid, unsigned block, size_t smem,
                       cudaStream_t s, uint32_t variant = 0);
cudaError_t jit_set_smem(JitKernel &k, size_t bytes);
cudaError_t jit_occupancy(const JitKernel &k, int block, size_t smem, int *blocks_per_sm, uint32_t variant = 0);

} // namespace gx

#endif
