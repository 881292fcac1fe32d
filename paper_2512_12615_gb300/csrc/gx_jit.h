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
    uint64_t budget = 1ull << 16;
};

struct JitKernel {
    cudaKernel_t kernel = nullptr;
    std::string key;
    size_t smem_attr = 0;
};

/* compile (or fetch from the caches) one kernel running progs[slot] for chunk slot `slot` */
int jit_build(const std::vector<const JitProgram *> &progs, JitKernel &out, std::string &log);
cudaError_t jit_launch(const JitKernel &k, const ExecParams &p, unsigned grid, unsigned block, size_t smem,
                       cudaStream_t s);
cudaError_t jit_set_smem(JitKernel &k, size_t bytes);
cudaError_t jit_occupancy(const JitKernel &k, int block, size_t smem, int *blocks_per_sm);

} // namespace gx

#endif
