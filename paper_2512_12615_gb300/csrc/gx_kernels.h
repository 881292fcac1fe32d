/* Launch interface between the host runtime and the device kernels (engine.cu). */
#ifndef GX_KERNELS_H
#define GX_KERNELS_H

#include <cuda_runtime.h>
#include <stdint.h>

#include "gx_layout.h"

namespace gx {

struct ExecParams {
    const uint8_t *image;  /* plain mode: the program image */
    uint32_t image_bytes;  /* plain mode: its size (multiple of 16) */
    uint32_t image_area;   /* shared-memory bytes reserved for images; ctx tiles follow */
    uint32_t ctx_size;     /* plain mode: bytes per record */
    uint32_t ept;          /* plain mode: tiles of blockDim events per block */
    uint32_t mode;         /* 0 = plain, 1 = persistent chunk table */
    uint32_t nchunks;
    const uint8_t *events; /* plain mode */
    uint64_t n;
    uint64_t idx_base;
    long long *ret_out;
    const gx_chunk *chunks; /* persistent mode */
    unsigned int *cursor;   /* persistent mode: next chunk to claim */
    const unsigned int *nchunks_dev; /* persistent mode: if set, the chunk count is read here */
};

cudaError_t exec_set_smem(size_t bytes);
cudaError_t exec_occupancy(int block, size_t smem, int *blocks_per_sm);
cudaError_t launch_exec(const ExecParams &p, unsigned grid, unsigned block, size_t smem, cudaStream_t s);
cudaError_t launch_hash_compact(const gx_dmap &m, uint8_t *out, unsigned long long *count, uint64_t cap_pairs,
                                cudaStream_t s);
cudaError_t launch_hash_insert(const gx_dmap &m, const uint8_t *in, uint64_t npairs, unsigned long long *stats,
                               int *err, cudaStream_t s);

} // namespace gx

#endif
