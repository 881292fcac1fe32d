/*
 * Layouts shared by the host side (decoder, map management) and the device kernels.
 *
 * Decoded program ("micro-ops").  The verifier annotates every instruction with the
 * memory region it touches; the decoder then turns each eBPF instruction into one or
 * two 64-bit micro-ops whose handler is specialised on the eBPF register it writes (or
 * reads), so the interpreter keeps R0..R10 in GPU registers and never indexes a
 * register file at run time.  Operands that would need a second register go through two
 * temporaries: T (second operand / value) and B (memory base address).
 *
 *   bits  0..15  handler id  = family * 11 + register   (families below)
 *                             or GX_SINGLE_BASE + k      (register-free handlers)
 *   bits 16..31  aux         jump target (micro-op index), or absolute ctx / stack offset
 *   bits 32..63  imm         signed 32-bit immediate / memory offset
 *
 * Device program image (16-byte aligned, staged whole into shared memory):
 *   gx_dprog_hdr | gx_dmap[n_maps] | u64 uops[n_uops]
 */
#ifndef GX_LAYOUT_H
#define GX_LAYOUT_H

#ifndef __CUDACC_RTC__
#include <stdint.h>
#endif

/*
 * Register-specialised families: the handler id carries the eBPF register (11 slots per
 * family; R0..R9, plus R10 for the three temp loads MOVT/MOVA/MOVB).  Rare operations
 * are "singles" that work on the temporaries only: A (accumulator), T (operand),
 * B (base address); the decoder wraps them in MOVA/MOVT and MOVRA/MOVR.
 */
#define GX_FAST_ALU(X, W, F) \
    X(ADD##W##F) X(SUB##W##F) X(MUL##W##F) X(OR##W##F) X(AND##W##F) X(XOR##W##F) X(LSH##W##F) X(RSH##W##F) \
    X(MOV##W##F)
#define GX_FAST_JMP(X, W, F) \
    X(JEQ##W##F) X(JNE##W##F) X(JGT##W##F) X(JGE##W##F) X(JLT##W##F) X(JLE##W##F) X(JSGT##W##F) X(JSGE##W##F) \
    X(JSLT##W##F) X(JSLE##W##F) X(JSET##W##F)

#define GX_FAMILIES(X)                                                                           \
    X(MOVT) X(MOVA) X(MOVB) X(MOVR) X(MOVRA) X(LDIMM64)                                          \
    GX_FAST_ALU(X, 64, K) GX_FAST_ALU(X, 64, T) GX_FAST_ALU(X, 32, K) GX_FAST_ALU(X, 32, T)      \
    GX_FAST_JMP(X, 64, K) GX_FAST_JMP(X, 64, T) GX_FAST_JMP(X, 32, K)                            \
    X(LDXC1) X(LDXC2) X(LDXC4) X(LDXC8) X(LDXCS1) X(LDXCS2) X(LDXCS4)                            \
    X(LDXS1) X(LDXS2) X(LDXS4) X(LDXS8) X(LDXSS1) X(LDXSS2) X(LDXSS4)                            \
    X(LDXM1) X(LDXM2) X(LDXM4) X(LDXM8) X(LDXMS1) X(LDXMS2) X(LDXMS4)                            \
    X(STXS1) X(STXS2) X(STXS4) X(STXS8)

#define GX_SLOW_ALU(X, W, F) X(DIV##W##F) X(SDIV##W##F) X(MOD##W##F) X(SMOD##W##F) X(ARSH##W##F)

#define GX_SINGLES(X)                                                                            \
    GX_SLOW_ALU(X, 64, K) GX_SLOW_ALU(X, 64, T) GX_SLOW_ALU(X, 32, K) GX_SLOW_ALU(X, 32, T)      \
    X(NEG64) X(NEG32) X(MOVSX64_8) X(MOVSX64_16) X(MOVSX64_32) X(MOVSX32_8) X(MOVSX32_16)        \
    X(LE16) X(LE32) X(BSWAP16) X(BSWAP32) X(BSWAP64)                                             \
    GX_FAST_JMP(X, 32, A)                                                                        \
    X(ST_S1) X(ST_S2) X(ST_S4) X(ST_S8) X(ST_M1) X(ST_M2) X(ST_M4) X(ST_M8)                      \
    X(STT_S1) X(STT_S2) X(STT_S4) X(STT_S8) X(STT_M1) X(STT_M2) X(STT_M4) X(STT_M8)              \
    X(AADD4) X(AOR4) X(AAND4) X(AXOR4) X(AADD8) X(AOR8) X(AAND8) X(AXOR8)                        \
    X(AFADD4) X(AFOR4) X(AFAND4) X(AFXOR4) X(AFADD8) X(AFOR8) X(AFAND8) X(AFXOR8)                \
    X(AXCHG4) X(AXCHG8) X(ACMPX4) X(ACMPX8)                                                      \
    X(JA) X(EXIT) X(NOP) X(MOVB_STK)                                                             \
    X(CALL_LOOKUP) X(CALL_UPDATE) X(CALL_DELETE) X(CALL_RB_OUTPUT) X(CALL_RB_RESERVE)             \
    X(CALL_RB_SUBMIT) X(CALL_RB_DISCARD) X(CALL_AMAX) X(CALL_AMIN)

#define GX_ENUM_FAM(n) GXF_##n,
enum gx_family { GX_FAMILIES(GX_ENUM_FAM) GX_NUM_FAMILIES };
/* handler ids are dense (family * 11 + register), so the interpreter's dispatch is one
   indexed jump over contiguous cases rather than a search */
#define GX_HSTRIDE 11
#define GX_SINGLE_BASE (GX_NUM_FAMILIES * GX_HSTRIDE)
#define GX_ENUM_SINGLE(n) GXS_##n,
enum gx_single { GX_SINGLES(GX_ENUM_SINGLE) GX_NUM_SINGLES };
#define GX_NUM_HANDLERS (GX_SINGLE_BASE + GX_NUM_SINGLES)

#ifndef __CUDACC_RTC__
static inline uint64_t gx_uop(uint32_t handler, uint32_t aux, int32_t imm) {
    return (uint64_t)(handler & 0xFFFFu) | ((uint64_t)(aux & 0xFFFFu) << 16) | ((uint64_t)(uint32_t)imm << 32);
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

#ifdef __cplusplus
static_assert(sizeof(gx_dmap) == 64, "descriptor size");
static_assert(sizeof(gx_dprog_hdr) == 64, "header size");
static_assert(sizeof(gx_chunk) == 64, "chunk size");
#endif

#endif /* GX_LAYOUT_H */
