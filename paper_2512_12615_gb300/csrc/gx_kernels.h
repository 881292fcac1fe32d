/* Launch interface between the host runtime and the device kernels (engine.cu). */
#ifndef GX_KERNELS_H
#define GX_KERNELS_H

#include <cuda_runtime.h>
#include <stdint.h>

#include "gx_layout.h"

namespace gx {

typedef gx_exec_params ExecParams;

cudaError_t exec_set_smem(size_t bytes);
cudaError_t exec_occupancy(int block, size_t smem, int *blocks_per_sm, bool checked = false);
cudaError_t launch_exec(const ExecParams &p, unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                        bool checked = false);
cudaError_t launch_hash_compact(const gx_dmap &m, uint8_t *out, unsigned long long *count, uint64_t cap_pairs,
                                cudaStream_t s);
cudaError_t launch_hash_insert(const gx_dmap &m, const uint8_t *in, uint64_t npairs, unsigned long long *stats,
                               int *err, cudaStream_t s);

} // namespace gx

#endif
