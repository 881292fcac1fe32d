/*
 * Device side of the engine: the eBPF interpreter kernel and the map kernels (sm_103a).
 *
 * Execution model (the paper's device runtime, Sec. 4.4.2 and Sec. 5.3, re-designed for
 * a batch engine):
 *   - one event per thread; a warp interprets 32 events in lock-step from the same
 *     decoded program held in shared memory (staged with cp.async);
 *   - the 32-byte (or ctx_size-byte) records of a warp are read with coalesced 16-byte
 *     streaming loads and transposed into shared memory, so ctx field loads are
 *     bank-conflict free;
 *   - R0..R10 live in GPU registers: every micro-op handler is specialised on the
 *     register it touches (see gx_layout.h), the dispatch index is warp-uniform;
 *   - divergence: while all 32 lanes sit at the same pc the warp runs in uniform mode;
 *     after a split branch it runs "min-pc" mode (only lanes at the smallest pc
 *     advance), which re-converges forward-branching code at its join points;
 *   - the 512-byte eBPF stack lives in local memory;
 *   - map value atomics are warp-aggregated: lanes hitting the same address are
 *     grouped with __match_any_sync, reduced with __reduce_*_sync, and one lane issues
 *     the atomic (the paper's per-warp leader update, Sec. 4.4.2);
 *   - ring-buffer space is reserved once per warp: ballot of the reserving lanes, an
 *     exclusive prefix sum of their record sizes, one atomicAdd on the head;
 *   - hash maps are lock-free open addressing (linear probing, slot claim by CAS,
 *     acquire/release publication of keys); every wait on another lane is bounded and
 *     records GX_E_TIMEOUT instead of hanging.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "gx_device.cuh"
#include "gx_kernels.h"
#include "gx_runtime.h"

namespace gx {

/* ------------------------------------------------------------------ the interpreter */

/* handler-case generators: one case per eBPF register */
#define RC10(FAM, M, A, B)                                                                  \
    case (FAM)*GX_HSTRIDE + 0: { M(r0, A, B) } break;                                               \
    case (FAM)*GX_HSTRIDE + 1: { M(r1, A, B) } break;                                               \
    case (FAM)*GX_HSTRIDE + 2: { M(r2, A, B) } break;                                               \
    case (FAM)*GX_HSTRIDE + 3: { M(r3, A, B) } break;                                               \
    case (FAM)*GX_HSTRIDE + 4: { M(r4, A, B) } break;                                               \
    case (FAM)*GX_HSTRIDE + 5: { M(r5, A, B) } break;                                               \
    case (FAM)*GX_HSTRIDE + 6: { M(r6, A, B) } break;                                               \
    case (FAM)*GX_HSTRIDE + 7: { M(r7, A, B) } break;                                               \
    case (FAM)*GX_HSTRIDE + 8: { M(r8, A, B) } break;                                               \
    case (FAM)*GX_HSTRIDE + 9: { M(r9, A, B) } break;
#define RC11(FAM, M, A, B) RC10(FAM, M, A, B) case (FAM)*GX_HSTRIDE + 10: { M(r10, A, B) } break;

#define IMM ((int32_t)(u >> 32))
#define AUX ((u32)(u >> 16) & 0xFFFFu)
#define SGL(k) (GX_SINGLE_BASE + (k))

#define H_A64K(R, O, _) R = a64<O>(R, sx32(IMM)); pc++;
#define H_A64T(R, O, _) R = a64<O>(R, T); pc++;
#define H_A32K(R, O, _) R = a32<O>(R, (u64)(u32)IMM); pc++;
#define H_A32T(R, O, _) R = a32<O>(R, T); pc++;
#define ALU_GROUP(OPNAME, O)                        \
    RC10(GXF_##OPNAME##64K, H_A64K, O, 0)           \
    RC10(GXF_##OPNAME##64T, H_A64T, O, 0)           \
    RC10(GXF_##OPNAME##32K, H_A32K, O, 0)           \
    RC10(GXF_##OPNAME##32T, H_A32T, O, 0)

/* accumulator forms of the rare ALU operations */
#define SLOW_GROUP(OPNAME, O)                                                                 \
    case SGL(GXS_##OPNAME##64K): A = a64<O>(A, sx32(IMM)); pc++; break;                       \
    case SGL(GXS_##OPNAME##64T): A = a64<O>(A, T); pc++; break;                               \
    case SGL(GXS_##OPNAME##32K): A = a32<O>(A, (u64)(u32)IMM); pc++; break;                   \
    case SGL(GXS_##OPNAME##32T): A = a32<O>(A, T); pc++; break;

#define JUMP_TO(TK)                                                                          \
    {                                                                                        \
        const bool tk_ = (TK);                                                               \
        const u32 np_ = tk_ ? AUX : pc + 1;                                                  \
        if (!div) {                                                                          \
            const u32 b_ = __ballot_sync(FULLM, tk_);                                        \
            if (b_ != 0 && b_ != FULLM) div = true;                                          \
        }                                                                                    \
        if (np_ <= pc && ++back > env.budget) goto budget_trip;                              \
        pc = np_;                                                                            \
    }

#define H_J64K(R, C, _) JUMP_TO(c64<C>(R, sx32(IMM)))
#define H_J64T(R, C, _) JUMP_TO(c64<C>(R, T))
#define H_J32K(R, C, _) JUMP_TO(c32<C>(R, (u64)(u32)IMM))
#define JMP_GROUP(OPNAME, C)                        \
    RC10(GXF_##OPNAME##64K, H_J64K, C, 0)           \
    RC10(GXF_##OPNAME##64T, H_J64T, C, 0)           \
    RC10(GXF_##OPNAME##32K, H_J32K, C, 0)           \
    case SGL(GXS_##OPNAME##32A): JUMP_TO(c32<C>(A, T)) break;

/* ctx word w of this lane lives at ctxw[w * env.ctx_row + lane]; AUX is the byte offset */
#define CTX_PTR ((const uint8_t *)(ctxw + (AUX >> 3) * env.ctx_row + lane) + (AUX & 7))
#define H_LDC(R, SZ, SG) R = load_sz<SZ, SG>(CTX_PTR); pc++;
#define H_LDS(R, SZ, SG) R = load_sz<SZ, SG>((const uint8_t *)stack + AUX); pc++;
#define H_LDM(R, SZ, SG) R = load_sz<SZ, SG>((const uint8_t *)B + IMM); pc++;
#define H_STS(R, SZ, _) store_sz<SZ>((uint8_t *)stack + AUX, R); pc++;
#define H_MOVT(R, _a, _b) T = R; pc++;
#define H_MOVA(R, _a, _b) A = R; pc++;
#define H_MOVB(R, _a, _b) B = R; pc++;
#define H_MOVR(R, _a, _b) R = T; pc++;
#define H_MOVRA(R, _a, _b) R = A; pc++;
#define H_LDIMM(R, _a, _b) R = (u64)(u32)IMM | ((u64)(u32)(env.uops[pc + 1] >> 32) << 32); pc += 2;

#define ST_IMM(SZ, ADDR) store_sz<SZ>((uint8_t *)(ADDR), sx32(IMM)); pc++; break;
#define ATOM(OP, SZ) agg_update<OP, SZ>(B + (u64)(s64)IMM, T, exec); pc++; break;
#define ATOMF(OP, SZ) T = fetch_update<OP, SZ>(B + (u64)(s64)IMM, T); pc++; break;

/*
 * Interpret one event per lane.  All 32 lanes of the warp call this together; lanes
 * without an event pass valid = false.  Returns R0.
 */
__device__ __noinline__ u64 interp(const ExecEnv env, const u64 *ctxw, bool valid, u64 ev_idx) {
    const u32 lane = lane_id();
    u64 stack[GX_STACK_BYTES / 8];
    u64 r0 = 0, r1 = 0, r2 = 0, r3 = 0, r4 = 0, r5 = 0, r6 = 0, r7 = 0, r8 = 0, r9 = 0;
    u64 r10 = (u64)(stack + GX_STACK_BYTES / 8);
    u64 T = 0, A = 0, B = 0;
    u32 pc = valid ? 0u : PC_DONE;
    u32 exec = __ballot_sync(FULLM, valid);
    bool div = exec != FULLM;
    u64 back = 0;
    for (;;) {
        if (div) {
            const u32 mpc = __reduce_min_sync(FULLM, pc);
            if (mpc == PC_DONE) break;
            exec = __ballot_sync(FULLM, pc == mpc);
            if (exec == FULLM) div = false;
            if (pc != mpc) continue;
        }
        const u64 u = env.uops[pc];
        switch ((u32)u & 0xFFFFu) {
            RC11(GXF_MOVT, H_MOVT, 0, 0)
            RC11(GXF_MOVA, H_MOVA, 0, 0)
            RC11(GXF_MOVB, H_MOVB, 0, 0)
            RC10(GXF_MOVR, H_MOVR, 0, 0)
            RC10(GXF_MOVRA, H_MOVRA, 0, 0)
            RC10(GXF_LDIMM64, H_LDIMM, 0, 0)
            ALU_GROUP(ADD, O_ADD)
            ALU_GROUP(SUB, O_SUB)
            ALU_GROUP(MUL, O_MUL)
            ALU_GROUP(OR, O_OR)
            ALU_GROUP(AND, O_AND)
            ALU_GROUP(XOR, O_XOR)
            ALU_GROUP(LSH, O_LSH)
            ALU_GROUP(RSH, O_RSH)
            ALU_GROUP(MOV, O_MOV)
            JMP_GROUP(JEQ, C_EQ)
            JMP_GROUP(JNE, C_NE)
            JMP_GROUP(JGT, C_GT)
            JMP_GROUP(JGE, C_GE)
            JMP_GROUP(JLT, C_LT)
            JMP_GROUP(JLE, C_LE)
            JMP_GROUP(JSGT, C_SGT)
            JMP_GROUP(JSGE, C_SGE)
            JMP_GROUP(JSLT, C_SLT)
            JMP_GROUP(JSLE, C_SLE)
            JMP_GROUP(JSET, C_SET)
            RC10(GXF_LDXC1, H_LDC, 1, false)
            RC10(GXF_LDXC2, H_LDC, 2, false)
            RC10(GXF_LDXC4, H_LDC, 4, false)
            RC10(GXF_LDXC8, H_LDC, 8, false)
            RC10(GXF_LDXCS1, H_LDC, 1, true)
            RC10(GXF_LDXCS2, H_LDC, 2, true)
            RC10(GXF_LDXCS4, H_LDC, 4, true)
            RC10(GXF_LDXS1, H_LDS, 1, false)
            RC10(GXF_LDXS2, H_LDS, 2, false)
            RC10(GXF_LDXS4, H_LDS, 4, false)
            RC10(GXF_LDXS8, H_LDS, 8, false)
            RC10(GXF_LDXSS1, H_LDS, 1, true)
            RC10(GXF_LDXSS2, H_LDS, 2, true)
            RC10(GXF_LDXSS4, H_LDS, 4, true)
            RC10(GXF_LDXM1, H_LDM, 1, false)
            RC10(GXF_LDXM2, H_LDM, 2, false)
            RC10(GXF_LDXM4, H_LDM, 4, false)
            RC10(GXF_LDXM8, H_LDM, 8, false)
            RC10(GXF_LDXMS1, H_LDM, 1, true)
            RC10(GXF_LDXMS2, H_LDM, 2, true)
            RC10(GXF_LDXMS4, H_LDM, 4, true)
            RC10(GXF_STXS1, H_STS, 1, 0)
            RC10(GXF_STXS2, H_STS, 2, 0)
            RC10(GXF_STXS4, H_STS, 4, 0)
            RC10(GXF_STXS8, H_STS, 8, 0)

            SLOW_GROUP(DIV, O_DIV)
            SLOW_GROUP(SDIV, O_SDIV)
            SLOW_GROUP(MOD, O_MOD)
            SLOW_GROUP(SMOD, O_SMOD)
            SLOW_GROUP(ARSH, O_ARSH)
        case SGL(GXS_NEG64): A = (u64)0 - A; pc++; break;
        case SGL(GXS_NEG32): A = (u64)(u32)(0u - (u32)A); pc++; break;
        case SGL(GXS_MOVSX64_8): A = (u64)(s64)(int8_t)T; pc++; break;
        case SGL(GXS_MOVSX64_16): A = (u64)(s64)(int16_t)T; pc++; break;
        case SGL(GXS_MOVSX64_32): A = (u64)(s64)(int32_t)T; pc++; break;
        case SGL(GXS_MOVSX32_8): A = (u64)(u32)(int32_t)(int8_t)T; pc++; break;
        case SGL(GXS_MOVSX32_16): A = (u64)(u32)(int32_t)(int16_t)T; pc++; break;
        case SGL(GXS_LE16): A &= 0xFFFFull; pc++; break;
        case SGL(GXS_LE32): A &= 0xFFFFFFFFull; pc++; break;
        case SGL(GXS_BSWAP16): A = (u64)__byte_perm((u32)A, 0u, 0x4401u); pc++; break;
        case SGL(GXS_BSWAP32): A = (u64)__byte_perm((u32)A, 0u, 0x0123u); pc++; break;
        case SGL(GXS_BSWAP64):
            A = ((u64)__byte_perm((u32)A, 0u, 0x0123u) << 32) | (u64)__byte_perm((u32)(A >> 32), 0u, 0x0123u);
            pc++;
            break;
        case SGL(GXS_ST_S1): ST_IMM(1, (uint8_t *)stack + AUX)
        case SGL(GXS_ST_S2): ST_IMM(2, (uint8_t *)stack + AUX)
        case SGL(GXS_ST_S4): ST_IMM(4, (uint8_t *)stack + AUX)
        case SGL(GXS_ST_S8): ST_IMM(8, (uint8_t *)stack + AUX)
        case SGL(GXS_ST_M1): ST_IMM(1, B + (s64)(int16_t)AUX)
        case SGL(GXS_ST_M2): ST_IMM(2, B + (s64)(int16_t)AUX)
        case SGL(GXS_ST_M4): ST_IMM(4, B + (s64)(int16_t)AUX)
        case SGL(GXS_ST_M8): ST_IMM(8, B + (s64)(int16_t)AUX)
        case SGL(GXS_STT_S1): store_sz<1>((uint8_t *)stack + AUX, T); pc++; break;
        case SGL(GXS_STT_S2): store_sz<2>((uint8_t *)stack + AUX, T); pc++; break;
        case SGL(GXS_STT_S4): store_sz<4>((uint8_t *)stack + AUX, T); pc++; break;
        case SGL(GXS_STT_S8): store_sz<8>((uint8_t *)stack + AUX, T); pc++; break;
        case SGL(GXS_STT_M1): store_sz<1>((uint8_t *)(B + (u64)(s64)IMM), T); pc++; break;
        case SGL(GXS_STT_M2): store_sz<2>((uint8_t *)(B + (u64)(s64)IMM), T); pc++; break;
        case SGL(GXS_STT_M4): store_sz<4>((uint8_t *)(B + (u64)(s64)IMM), T); pc++; break;
        case SGL(GXS_STT_M8): store_sz<8>((uint8_t *)(B + (u64)(s64)IMM), T); pc++; break;
        case SGL(GXS_AADD4): ATOM(AG_ADD, 4)
        case SGL(GXS_AOR4): ATOM(AG_OR, 4)
        case SGL(GXS_AAND4): ATOM(AG_AND, 4)
        case SGL(GXS_AXOR4): ATOM(AG_XOR, 4)
        case SGL(GXS_AADD8): ATOM(AG_ADD, 8)
        case SGL(GXS_AOR8): ATOM(AG_OR, 8)
        case SGL(GXS_AAND8): ATOM(AG_AND, 8)
        case SGL(GXS_AXOR8): ATOM(AG_XOR, 8)
        case SGL(GXS_AFADD4): ATOMF(AG_ADD, 4)
        case SGL(GXS_AFOR4): ATOMF(AG_OR, 4)
        case SGL(GXS_AFAND4): ATOMF(AG_AND, 4)
        case SGL(GXS_AFXOR4): ATOMF(AG_XOR, 4)
        case SGL(GXS_AFADD8): ATOMF(AG_ADD, 8)
        case SGL(GXS_AFOR8): ATOMF(AG_OR, 8)
        case SGL(GXS_AFAND8): ATOMF(AG_AND, 8)
        case SGL(GXS_AFXOR8): ATOMF(AG_XOR, 8)
        case SGL(GXS_AXCHG4): T = xchg<4>(B + (u64)(s64)IMM, T); pc++; break;
        case SGL(GXS_AXCHG8): T = xchg<8>(B + (u64)(s64)IMM, T); pc++; break;
        case SGL(GXS_ACMPX4): r0 = cmpxchg<4>(B + (u64)(s64)IMM, r0, T); pc++; break;
        case SGL(GXS_ACMPX8): r0 = cmpxchg<8>(B + (u64)(s64)IMM, r0, T); pc++; break;
        case SGL(GXS_JA): JUMP_TO(true) break;
        case SGL(GXS_NOP): pc++; break;
        case SGL(GXS_MOVB_STK): B = (u64)((uint8_t *)stack + AUX); pc++; break;
        case SGL(GXS_EXIT):
            if (!div) goto finished;
            pc = PC_DONE;
            break;
        case SGL(GXS_CALL_LOOKUP):
            r0 = map_lookup(env.maps[r1], (const uint8_t *)r2, exec, env.stats);
            pc++;
            break;
        case SGL(GXS_CALL_UPDATE):
            r0 = (u64)(s64)map_update(env.maps[r1], (const uint8_t *)r2, (const uint8_t *)r3, r4, exec, env.stats);
            pc++;
            break;
        case SGL(GXS_CALL_DELETE): {
            const gx_dmap &m = env.maps[r1];
            r0 = (u64)(s64)(m.type == GX_MAP_HASH ? hash_delete(m, (const uint8_t *)r2, env.stats) : GX_EINVAL);
            pc++;
            break;
        }
        case SGL(GXS_CALL_RB_RESERVE):
            r0 = rb_reserve(env.maps[r1], r2, exec, ev_idx);
            pc++;
            break;
        case SGL(GXS_CALL_RB_OUTPUT): {
            const u64 p = rb_reserve(env.maps[r1], r3, exec, ev_idx);
            if (p) copy_bytes((uint8_t *)p, (const uint8_t *)r2, (u32)r3);
            r0 = p ? 0 : (u64)(s64)GX_EAGAIN;
            pc++;
            break;
        }
        case SGL(GXS_CALL_RB_SUBMIT): pc++; break; /* records are committed when reserved */
        case SGL(GXS_CALL_RB_DISCARD):
            ((u32 *)(r1 - GX_RB_HDR))[1] = GX_RB_DISCARDED;
            pc++;
            break;
        case SGL(GXS_CALL_AMAX): agg_update<AG_MAX, 8>(r1, r2, exec); pc++; break;
        case SGL(GXS_CALL_AMIN): agg_update<AG_MIN, 8>(r1, r2, exec); pc++; break;
        default:
            set_status(env.stats, GX_E_DEVICE);
            r0 = 0;
            pc = PC_DONE;
            if (!div) goto finished;
            break;
        }
        continue;
    budget_trip:
        atomicAdd(&env.stats[GX_STAT_BUDGET], 1ull);
        set_status(env.stats, GX_E_BUDGET);
        r0 = 0;
        pc = PC_DONE;
        if (!div) break;
    }
finished:
    return r0;
}

/* ------------------------------------------------------------------ kernels */
__global__ void __launch_bounds__(256, 3) gx_exec_kernel(ExecParams P) {
    exec_tiles(P, [](const ExecEnv &env, const u64 *ctxw, bool valid, u64 ev_idx) {
        return interp(env, ctxw, valid, ev_idx);
    });
}

/* hash map snapshot: FULL slots -> packed {key, value} pairs */
__global__ void gx_hash_compact_kernel(gx_dmap m, uint8_t *out, u64 *count, u64 cap_pairs) {
    const u64 stride = (u64)gridDim.x * blockDim.x;
    const u32 pair = m.key_size + m.value_size;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i <= m.mask; i += stride) {
        const uint8_t *slot = m.slots + i * m.sstride;
        if (*(const volatile u32 *)slot != GX_SLOT_FULL) continue;
        u64 k = atomicAdd(count, 1ull);
        if (k >= cap_pairs) continue;
        uint8_t *o = out + k * pair;
        for (u32 b = 0; b < m.key_size; b++) o[b] = slot[8 + b];
        const uint8_t *v = m.values + i * m.vstride;
        for (u32 b = 0; b < m.value_size; b++) o[m.key_size + b] = v[b];
    }
}

/* hash map restore: insert / overwrite packed pairs (one thread per pair) */
__global__ void gx_hash_insert_kernel(gx_dmap m, const uint8_t *in, u64 npairs, u64 *stats, int *err) {
    const u32 pair = m.key_size + m.value_size;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < npairs; i += (u64)gridDim.x * blockDim.x) {
        int r = hash_update(m, in + i * pair, in + i * pair + m.key_size, GX_ANY, stats);
        if (r) atomicCAS(err, 0, r);
    }
}

/* ------------------------------------------------------------------ host launchers */
cudaError_t exec_set_smem(size_t bytes) {
    return cudaFuncSetAttribute(gx_exec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t exec_occupancy(int block, size_t smem, int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, gx_exec_kernel, block, smem);
}

cudaError_t launch_exec(const ExecParams &p, unsigned grid, unsigned block, size_t smem, cudaStream_t s) {
    gx_exec_kernel<<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_hash_compact(const gx_dmap &m, uint8_t *out, unsigned long long *count, uint64_t cap_pairs,
                                cudaStream_t s) {
    u64 slots = m.mask + 1;
    unsigned grid = (unsigned)((slots + 255) / 256);
    if (grid > 4096) grid = 4096;
    gx_hash_compact_kernel<<<grid, 256, 0, s>>>(m, out, count, cap_pairs);
    return cudaGetLastError();
}

cudaError_t launch_hash_insert(const gx_dmap &m, const uint8_t *in, uint64_t npairs, unsigned long long *stats,
                               int *err, cudaStream_t s) {
    unsigned grid = (unsigned)((npairs + 255) / 256);
    if (grid > 4096) grid = 4096;
    if (grid == 0) return cudaSuccess;
    gx_hash_insert_kernel<<<grid, 256, 0, s>>>(m, in, npairs, stats, err);
    return cudaGetLastError();
}

} // namespace gx

/* ------------------------------------------------------------------ snapshot without allocation */
/*
 * Scratch for gx_map_read_noalloc, fixed at GX_NOALLOC_SCRATCH_BYTES: bytes [0, 256) hold the
 * pair counter, the packed {key, value} pairs follow.  Every device that loads the library
 * keeps this array until the process exits.  All calls share it, so calls whose GPU work
 * overlaps (other streams, other host threads) race on it.
 */
static __device__ __align__(256) unsigned char gx_noalloc_scratch[GX_NOALLOC_SCRATCH_BYTES];

namespace gx {
namespace {
std::mutex noalloc_mu;
void *noalloc_ptr[64];
bool noalloc_ready[64];
} // namespace
} // namespace gx

extern "C" int gx_map_read_noalloc(gx_map *m, void *host_out, uint64_t cap_bytes, uint64_t *n_out, void *stream) {
    using namespace gx;
    if (!m || (!host_out && cap_bytes)) return GX_EINVAL;
    if (m->d.type != GX_MAP_HASH) return GX_EINVAL;
    const uint64_t pair = (uint64_t)m->d.key_size + m->d.value_size;
    const uint64_t cap_pairs = (GX_NOALLOC_SCRATCH_BYTES - 256) / pair;
    if (cap_pairs == 0) return GX_E2BIG;
    const int dev = m->ctx->device;
    if (dev < 0 || dev >= 64) return GX_EINVAL;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return GX_E_CUDA;
    if (cur != dev && cudaSetDevice(dev) != cudaSuccess) return GX_E_CUDA;
    int rc = GX_OK;
    void *base = nullptr;
    {
        /* one-time set-up per device, with that device current: the array's device address */
        std::lock_guard<std::mutex> g(noalloc_mu);
        if (!noalloc_ready[dev]) {
            if (cudaGetSymbolAddress(&noalloc_ptr[dev], gx_noalloc_scratch) != cudaSuccess) {
                cudaGetLastError();
                rc = GX_E_CUDA;
            } else {
                noalloc_ready[dev] = true;
            }
        }
        base = noalloc_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long cnt = 0;
    if (rc == GX_OK) {
        unsigned long long *count = (unsigned long long *)base;
        uint8_t *pairs = (uint8_t *)base + 256;
        if (cudaMemsetAsync(count, 0, 8, s) != cudaSuccess ||
            launch_hash_compact(m->d, pairs, count, cap_pairs, s) != cudaSuccess ||
            cudaMemcpyAsync(&cnt, count, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            rc = GX_E_CUDA;
        } else if (cnt > cap_pairs) {
            rc = GX_E2BIG; /* the live pairs do not fit the fixed scratch: nothing copied */
        } else if (cnt * pair > cap_bytes) {
            rc = GX_E2BIG;
        } else if (cnt && (cudaMemcpyAsync(host_out, pairs, cnt * pair, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                           cudaStreamSynchronize(s) != cudaSuccess)) {
            cudaGetLastError();
            rc = GX_E_CUDA;
        }
    }
    if (n_out) *n_out = cnt;
    if (cur != dev) cudaSetDevice(cur);
    return rc;
}
