/*
 * Layouts shared by the host side (decoder, map management) and the device kernels.
 *
 * Decoded program ("micro-ops"): one 16-byte micro-op per eBPF instruction (the second
 * slot of a 64-bit immediate becomes a NOP).  The verifier annotates every instruction
 * with the memory region it touches, so ctx and stack accesses carry their proven
 * absolute offsets and map / ring-buffer accesses their region.  The interpreter keeps
 * R0..R10 in a per-thread array indexed by the dst / src fields.
 *   word 0  bits  0..7   operation (enum gx_op)
 *           bits  8..11  dst register, bits 12..15 src register
 *           bits 16..31  aux: jump target (micro-op index), or absolute ctx / stack offset
 *           bits 32..63  imm: signed 32-bit immediate, or memory offset
 *   word 1  the 64-bit value of a 64-bit immediate (map references: the map's index)
 *
 * Device program image (16-byte aligned, staged whole into shared memory):
 *   gx_dprog_hdr | gx_dmap[n_maps] | u64 uops[2 * n_uops]
 */
#ifndef GX_LAYOUT_H
#define GX_LAYOUT_H

#ifndef __CUDACC_RTC__
#include <stdint.h>
#endif

/*
 * Operations.  ALU: width (64, 32) x operand (K immediate, X register) x the 14 RFC 9669
 * operations, in enum order (O_ADD .. O_MOV of the device header); jumps: the 11
 * conditions x (64 K, 64 X, 32 K, 32 X); loads: region (C ctx, S stack, M memory) x size
 * (1, 2, 4, 8, then sign-extending 1, 2, 4); stores: region (S, M) x size, immediate or
 * register; atomics: region (S, M) x the 20 forms; then the helper calls.  F64K_*: a
 * register copy fused with the 64-bit immediate operation on its destination that
 * follows it ("mov d, s; op d, imm" as d = op(s, imm)), which then skips that second
 * instruction's micro-op (left in place for jumps to it).
 */
#define GX_ALU_OPS(X, P) X(P##ADD) X(P##SUB) X(P##MUL) X(P##DIV) X(P##SDIV) X(P##MOD) X(P##SMOD) \
    X(P##OR) X(P##AND) X(P##XOR) X(P##LSH) X(P##RSH) X(P##ARSH) X(P##MOV)
#define GX_JMP_OPS(X, P) X(P##JEQ) X(P##JNE) X(P##JGT) X(P##JGE) X(P##JLT) X(P##JLE) X(P##JSGT) \
    X(P##JSGE) X(P##JSLT) X(P##JSLE) X(P##JSET)
#define GX_LD_OPS(X, P) X(P##1) X(P##2) X(P##4) X(P##8) X(P##S1) X(P##S2) X(P##S4)
#define GX_SZ_OPS(X, P) X(P##1) X(P##2) X(P##4) X(P##8)
#define GX_ATOM_OPS(X, P) X(P##ADD4) X(P##OR4) X(P##AND4) X(P##XOR4) X(P##ADD8) X(P##OR8) X(P##AND8) \
    X(P##XOR8) X(P##FADD4) X(P##FOR4) X(P##FAND4) X(P##FXOR4) X(P##FADD8) X(P##FOR8) X(P##FAND8) \
    X(P##FXOR8) X(P##XCHG4) X(P##XCHG8) X(P##CMPX4) X(P##CMPX8)

#define GX_OPS(X)                                                                                \
    GX_ALU_OPS(X, A64K_) GX_ALU_OPS(X, A64X_) GX_ALU_OPS(X, A32K_) GX_ALU_OPS(X, A32X_)          \
    X(NEG64) X(NEG32) X(MOVSX64_8) X(MOVSX64_16) X(MOVSX64_32) X(MOVSX32_8) X(MOVSX32_16)        \
    X(LE16) X(LE32) X(BSWAP16) X(BSWAP32) X(BSWAP64) X(LDIMM64)                                   \
    GX_ALU_OPS(X, F64K_)                                                                         \
    GX_JMP_OPS(X, J64K_) GX_JMP_OPS(X, J64X_) GX_JMP_OPS(X, J32K_) GX_JMP_OPS(X, J32X_)          \
    X(JA) X(EXIT) X(NOP)                                                                         \
    GX_LD_OPS(X, LDC) GX_LD_OPS(X, LDS) GX_LD_OPS(X, LDM)                                        \
    GX_SZ_OPS(X, STIS) GX_SZ_OPS(X, STIM) GX_SZ_OPS(X, STXS) GX_SZ_OPS(X, STXM)                  \
    GX_ATOM_OPS(X, AS_) GX_ATOM_OPS(X, AM_)                                                      \
    X(CALL_LOOKUP) X(CALL_UPDATE) X(CALL_DELETE) X(CALL_RB_OUTPUT) X(CALL_RB_RESERVE)             \
    X(CALL_RB_SUBMIT) X(CALL_RB_DISCARD) X(CALL_AMAX) X(CALL_AMIN)

#define GX_ENUM_OP(n) GXO_##n,
enum gx_op { GX_OPS(GX_ENUM_OP) GX_NUM_OPS };

#ifndef __CUDACC_RTC__
static inline uint64_t gx_uop(uint32_t op, uint32_t dst, uint32_t src, uint32_t aux, int32_t imm) {
    return (uint64_t)(op & 0xFFu) | ((uint64_t)(dst & 0xFu) << 8) | ((uint64_t)(src & 0xFu) << 12) |
           ((uint64_t)(aux & 0xFFFFu) << 16) | ((uint64_t)(uint32_t)imm << 32);
}
#endif

/*
 * Transposed event tiles: a warp's 32 records of cw words are kept as cw rows of
 * GX_CTX_ROW(cw) words (word w of record r at w * row + r).  The padding (16 / cw words
 * for cw = 4, 8, 16) spreads the tile's 8-byte stores over all banks; reads of one word
 * across the warp are consecutive either way.
 */
#define GX_CTX_ROW(cw) (32u + (((cw) == 4u || (cw) == 8u || (cw) == 16u) ? 16u / (cw) : 0u))

/* ---------------------------------------------------------------- device map descriptor */
#define GX_SLOT_EMPTY 0u
#define GX_SLOT_BUSY 1u
#define GX_SLOT_FULL 2u
#define GX_SLOT_TOMB 3u

#define GX_RB_HDR 16u
#define GX_RB_DISCARDED 1u
#define GX_RB_PAD 2u

typedef struct gx_dmap {
    uint32_t type;        /* GX_MAP_* */
    uint32_t key_size;
    uint32_t value_size;
    uint32_t max_entries;
    uint32_t vstride;     /* bytes between values (value_size rounded up to 8) */
    uint32_t sstride;     /* hash: bytes per slot = 8 (state word + pad) + key rounded to 8 */
    uint64_t mask;        /* hash: slots - 1; ringbuf: buffer bytes */
    uint8_t *values;      /* array / hash values; ringbuf data */
    uint8_t *slots;       /* hash slots */
    unsigned long long *ctr; /* hash: [0] live keys [1] refused inserts; ringbuf: [0] head [1] drops */
    uint64_t pad;
} gx_dmap;

typedef struct gx_dprog_hdr {
    uint32_t n_uops;
    uint32_t n_maps;
    uint32_t ctx_size;
    uint32_t image_bytes;      /* whole image, multiple of 16 */
    uint64_t budget;           /* taken backward jumps allowed per event */
    unsigned long long *stats; /* [0] sticky status (int32 in low bits) [1] budget trips [2] waits expired */
    uint64_t pad[4];
} gx_dprog_hdr;

#define GX_STAT_STATUS 0
#define GX_STAT_BUDGET 1
#define GX_STAT_WAITS 2
#define GX_STAT_FAULT 3 /* checked programs: 1 + the pc of the first stopped access */
#define GX_STAT_WORDS 4

/* persistent-kernel work item: events [begin, end) of one program */
typedef struct gx_chunk {
    const uint8_t *image;      /* device program image */
    const uint8_t *events;     /* record 0 of the item */
    long long *ret_out;        /* nullable, indexed by event index within the item */
    uint64_t begin, end;       /* event range within the item */
    uint64_t idx_base;         /* added to ring-buffer event indices */
    uint32_t image_bytes;
    uint32_t ctx_size;
    uint64_t pad;
} gx_chunk;

/* kernel parameters of the interpreter and of specialised programs */
typedef struct gx_exec_params {
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
    uint32_t wc_bits;      /* specialised programs: bits 0-7 log2 entries of each map's combining cache,
                              0 = no block-private combining (updates go to device memory); bit 8:
                              updates that miss the cache are warp-aggregated */
    uint32_t shard_off;    /* byte offset of the combining area in dynamic shared memory */
} gx_exec_params;

/*
 * Checked programs (GX_PROG_CHECKED): the regions an event may touch through a pointer.
 * Written once for the device's checked interpreter and for host tests of the bounds.
 */
#if defined(__CUDACC__)
#define GX_HD __host__ __device__ __forceinline__
#else
#define GX_HD static inline
#endif
#define GX_MAP_HASH_T 1u    /* GX_MAP_HASH of gx.h */
#define GX_MAP_RINGBUF_T 27u /* GX_MAP_RINGBUF of gx.h */

/* bytes of a map's value memory (a ring buffer: its data area) */
GX_HD uint64_t gx_value_bytes(const gx_dmap *m) {
    if (m->type == GX_MAP_RINGBUF_T) return m->mask;
    if (m->type == GX_MAP_HASH_T) return (m->mask + 1) * (uint64_t)m->vstride;
    return (uint64_t)m->max_entries * m->vstride;
}

/* [a, a + bytes) lies within the lane's stack or within one map's value memory (a ring
   buffer's data): bytes >= 1, no wrap-around */
GX_HD int gx_range_ok(const gx_dmap *maps, uint32_t n_maps, uint64_t stack_lo, uint32_t stack_bytes, uint64_t a,
                      uint64_t bytes) {
    if (bytes == 0 || a + bytes < a) return 0;
    if (a >= stack_lo && a + bytes <= stack_lo + stack_bytes) return 1;
    for (uint32_t i = 0; i < n_maps; i++) {
        const uint64_t lo = (uint64_t)maps[i].values;
        if (a >= lo && a + bytes <= lo + gx_value_bytes(&maps[i])) return 1;
    }
    return 0;
}

/* a load, store or atomic of `size` bytes (1, 2, 4, 8) at a: in range and naturally aligned */
GX_HD int gx_access_ok(const gx_dmap *maps, uint32_t n_maps, uint64_t stack_lo, uint32_t stack_bytes, uint64_t a,
                       uint32_t size) {
    return (a & (uint64_t)(size - 1)) == 0 && gx_range_ok(maps, n_maps, stack_lo, stack_bytes, a, size);
}

#ifdef __cplusplus
static_assert(sizeof(gx_dmap) == 64, "descriptor size");
static_assert(sizeof(gx_dprog_hdr) == 64, "header size");
static_assert(sizeof(gx_chunk) == 64, "chunk size");
#endif

#endif /* GX_LAYOUT_H */
