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
 *   - one 16-byte micro-op per eBPF instruction, dispatched on a dense operation id
 *     (warp-uniform while the lanes agree); R0..R10 in a per-thread array indexed by
 *     the micro-op's register fields (local memory, held in L1);
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

/* case generators over the operation lists of gx_layout.h */
#define ALU_CASE(P, NAME, O, W, OPND) \
    case GXO_##P##NAME: R[d] = W<O>(R[d], OPND); break;
#define ALU_FORM(P, W, OPND)                                                                     \
    ALU_CASE(P, ADD, O_ADD, W, OPND) ALU_CASE(P, SUB, O_SUB, W, OPND) ALU_CASE(P, MUL, O_MUL, W, OPND) \
    ALU_CASE(P, DIV, O_DIV, W, OPND) ALU_CASE(P, SDIV, O_SDIV, W, OPND)                          \
    ALU_CASE(P, MOD, O_MOD, W, OPND) ALU_CASE(P, SMOD, O_SMOD, W, OPND)                          \
    ALU_CASE(P, OR, O_OR, W, OPND) ALU_CASE(P, AND, O_AND, W, OPND) ALU_CASE(P, XOR, O_XOR, W, OPND) \
    ALU_CASE(P, LSH, O_LSH, W, OPND) ALU_CASE(P, RSH, O_RSH, W, OPND) ALU_CASE(P, ARSH, O_ARSH, W, OPND) \
    ALU_CASE(P, MOV, O_MOV, W, OPND)

/* a conditional jump: the taken lanes go to aux; a split of the warp switches to min-pc mode */
#define JMP_CASE(P, NAME, C, W, OPND) \
    case GXO_##P##NAME: taken = W<C>(R[d], OPND); goto jump;
#define JMP_FORM(P, W, OPND)                                                                     \
    JMP_CASE(P, JEQ, C_EQ, W, OPND) JMP_CASE(P, JNE, C_NE, W, OPND) JMP_CASE(P, JGT, C_GT, W, OPND) \
    JMP_CASE(P, JGE, C_GE, W, OPND) JMP_CASE(P, JLT, C_LT, W, OPND) JMP_CASE(P, JLE, C_LE, W, OPND) \
    JMP_CASE(P, JSGT, C_SGT, W, OPND) JMP_CASE(P, JSGE, C_SGE, W, OPND)                          \
    JMP_CASE(P, JSLT, C_SLT, W, OPND) JMP_CASE(P, JSLE, C_SLE, W, OPND) JMP_CASE(P, JSET, C_SET, W, OPND)

/* checked programs: stop the event before an access that fails its check */
#define CHK(OK)                     \
    if (CHECKED && !(OK)) goto fault;
#define CTX_OK(SZ) ((aux & ((SZ) - 1u)) == 0 && aux + (SZ) <= env.ctx_size)
#define STK_OK(SZ) ((aux & ((SZ) - 1u)) == 0 && aux + (SZ) <= GX_STACK_BYTES)
#define MEM_OK(A, SZ) gx_access_ok(env.maps, env.n_maps, (u64)stack, GX_STACK_BYTES, (u64)(A), (SZ))
#define RANGE_OK(A, N) gx_range_ok(env.maps, env.n_maps, (u64)stack, GX_STACK_BYTES, (u64)(A), (N))
#define LDM_OK(SZ) MEM_OK(R[s] + (u64)(s64)imm, SZ)
#define STIM_OK(SZ) MEM_OK(R[d] + (u64)(s64)(int16_t)aux, SZ)
#define DIMM_OK(SZ) MEM_OK(R[d] + (u64)(s64)imm, SZ)
/* a helper's map argument: a map of the program, of the kind the helper takes */
#define MAP_OK(IDX) ((IDX) < env.n_maps && env.maps[IDX].type != GX_MAP_RINGBUF)
#define RING_OK(IDX) ((IDX) < env.n_maps && env.maps[IDX].type == GX_MAP_RINGBUF)

#define LD_FORM(P, ADDR, OK)                                                                     \
    case GXO_##P##1: CHK(OK(1)) R[d] = load_sz<1, false>(ADDR); break;                           \
    case GXO_##P##2: CHK(OK(2)) R[d] = load_sz<2, false>(ADDR); break;                           \
    case GXO_##P##4: CHK(OK(4)) R[d] = load_sz<4, false>(ADDR); break;                           \
    case GXO_##P##8: CHK(OK(8)) R[d] = load_sz<8, false>(ADDR); break;                           \
    case GXO_##P##S1: CHK(OK(1)) R[d] = load_sz<1, true>(ADDR); break;                           \
    case GXO_##P##S2: CHK(OK(2)) R[d] = load_sz<2, true>(ADDR); break;                           \
    case GXO_##P##S4: CHK(OK(4)) R[d] = load_sz<4, true>(ADDR); break;

#define ST_FORM(P, ADDR, VAL, OK)                                                                \
    case GXO_##P##1: CHK(OK(1)) store_sz<1>(ADDR, VAL); break;                                   \
    case GXO_##P##2: CHK(OK(2)) store_sz<2>(ADDR, VAL); break;                                   \
    case GXO_##P##4: CHK(OK(4)) store_sz<4>(ADDR, VAL); break;                                   \
    case GXO_##P##8: CHK(OK(8)) store_sz<8>(ADDR, VAL); break;

/* atomics at ADDR with the value in R[s]: plain (warp-aggregated), fetching, xchg, cmpxchg */
#define ATOM_FORM(P, ADDR, OK)                                                                       \
    case GXO_##P##ADD4: CHK(OK(4)) agg_update<AG_ADD, 4>(ADDR, R[s], exec); break;                          \
    case GXO_##P##OR4: CHK(OK(4)) agg_update<AG_OR, 4>(ADDR, R[s], exec); break;                            \
    case GXO_##P##AND4: CHK(OK(4)) agg_update<AG_AND, 4>(ADDR, R[s], exec); break;                          \
    case GXO_##P##XOR4: CHK(OK(4)) agg_update<AG_XOR, 4>(ADDR, R[s], exec); break;                          \
    case GXO_##P##ADD8: CHK(OK(8)) agg_update<AG_ADD, 8>(ADDR, R[s], exec); break;                          \
    case GXO_##P##OR8: CHK(OK(8)) agg_update<AG_OR, 8>(ADDR, R[s], exec); break;                            \
    case GXO_##P##AND8: CHK(OK(8)) agg_update<AG_AND, 8>(ADDR, R[s], exec); break;                          \
    case GXO_##P##XOR8: CHK(OK(8)) agg_update<AG_XOR, 8>(ADDR, R[s], exec); break;                          \
    case GXO_##P##FADD4: CHK(OK(4)) R[s] = fetch_update<AG_ADD, 4>(ADDR, R[s]); break;                      \
    case GXO_##P##FOR4: CHK(OK(4)) R[s] = fetch_update<AG_OR, 4>(ADDR, R[s]); break;                        \
    case GXO_##P##FAND4: CHK(OK(4)) R[s] = fetch_update<AG_AND, 4>(ADDR, R[s]); break;                      \
    case GXO_##P##FXOR4: CHK(OK(4)) R[s] = fetch_update<AG_XOR, 4>(ADDR, R[s]); break;                      \
    case GXO_##P##FADD8: CHK(OK(8)) R[s] = fetch_update<AG_ADD, 8>(ADDR, R[s]); break;                      \
    case GXO_##P##FOR8: CHK(OK(8)) R[s] = fetch_update<AG_OR, 8>(ADDR, R[s]); break;                        \
    case GXO_##P##FAND8: CHK(OK(8)) R[s] = fetch_update<AG_AND, 8>(ADDR, R[s]); break;                      \
    case GXO_##P##FXOR8: CHK(OK(8)) R[s] = fetch_update<AG_XOR, 8>(ADDR, R[s]); break;                      \
    case GXO_##P##XCHG4: CHK(OK(4)) R[s] = xchg<4>(ADDR, R[s]); break;                                      \
    case GXO_##P##XCHG8: CHK(OK(8)) R[s] = xchg<8>(ADDR, R[s]); break;                                      \
    case GXO_##P##CMPX4: CHK(OK(4)) R[0] = cmpxchg<4>(ADDR, R[0], R[s]); break;                             \
    case GXO_##P##CMPX8: CHK(OK(8)) R[0] = cmpxchg<8>(ADDR, R[0], R[s]); break;

/*
 * Interpret one event per lane.  All 32 lanes of the warp call this together; lanes
 * without an event pass valid = false.  Returns R0.
 *
 * Each micro-op is one 16-byte shared-memory load (the same address for every lane at the
 * same pc) and one dispatch over the dense operation ids; R0..R10 sit in a per-thread
 * array indexed by the micro-op's register fields (local memory, served by L1).  While all
 * lanes sit at the same pc the warp runs in uniform mode; after a split branch it runs
 * "min-pc" mode (only lanes at the smallest pc advance), which re-converges
 * forward-branching code at its join points.
 */
template <bool CHECKED>
__device__ __noinline__ u64 interp(const ExecEnv env, const u64 *ctxw, bool valid, u64 ev_idx) {
    const u32 lane = lane_id();
    u64 stack[GX_STACK_BYTES / 8];
    u64 R[11];
#pragma unroll
    for (int k = 0; k < 10; k++) R[k] = 0;
    R[10] = (u64)(stack + GX_STACK_BYTES / 8);
    const ulonglong2 *uops = (const ulonglong2 *)env.uops;
    u32 pc = valid ? 0u : PC_DONE;
    u32 exec = __ballot_sync(FULLM, valid);
    /* the checked build stays in min-pc mode: a lane may stop on its own at any access */
    bool div = CHECKED || exec != FULLM;
    u64 back = 0;
    for (;;) {
        if (div) {
            const u32 mpc = __reduce_min_sync(FULLM, pc);
            if (mpc == PC_DONE) break;
            exec = __ballot_sync(FULLM, pc == mpc);
            if (!CHECKED && exec == FULLM) div = false;
            if (pc != mpc) continue;
        }
        const ulonglong2 u = uops[pc];
        const u32 w = (u32)u.x;
        const u32 d = (w >> 8) & 0xFu, s = (w >> 12) & 0xFu, aux = w >> 16;
        const int32_t imm = (int32_t)(u.x >> 32);
        bool taken;
        switch (w & 0xFFu) {
            ALU_FORM(A64K_, a64, (u64)(s64)imm)
            ALU_FORM(A64X_, a64, R[s])
            ALU_FORM(A32K_, a32, (u64)(u32)imm)
            ALU_FORM(A32X_, a32, R[s])
        case GXO_NEG64: R[d] = (u64)0 - R[d]; break;
        case GXO_NEG32: R[d] = (u64)(u32)(0u - (u32)R[d]); break;
        case GXO_MOVSX64_8: R[d] = (u64)(s64)(int8_t)R[s]; break;
        case GXO_MOVSX64_16: R[d] = (u64)(s64)(int16_t)R[s]; break;
        case GXO_MOVSX64_32: R[d] = (u64)(s64)(int32_t)R[s]; break;
        case GXO_MOVSX32_8: R[d] = (u64)(u32)(int32_t)(int8_t)R[s]; break;
        case GXO_MOVSX32_16: R[d] = (u64)(u32)(int32_t)(int16_t)R[s]; break;
        case GXO_LE16: R[d] &= 0xFFFFull; break;
        case GXO_LE32: R[d] &= 0xFFFFFFFFull; break;
        case GXO_BSWAP16: R[d] = (u64)__byte_perm((u32)R[d], 0u, 0x4401u); break;
        case GXO_BSWAP32: R[d] = (u64)__byte_perm((u32)R[d], 0u, 0x0123u); break;
        case GXO_BSWAP64: {
            const u64 x = R[d];
            R[d] = ((u64)__byte_perm((u32)x, 0u, 0x0123u) << 32) | (u64)__byte_perm((u32)(x >> 32), 0u, 0x0123u);
            break;
        }
        case GXO_LDIMM64: R[d] = u.y; break;
            /* "mov d, s; op d, imm": d = op(s, imm), then past the second instruction */
#define FUSED_CASE(NAME, O) \
    case GXO_F64K_##NAME: R[d] = a64<O>(R[s], (u64)(s64)imm); pc += 2; continue;
            FUSED_CASE(ADD, O_ADD) FUSED_CASE(SUB, O_SUB) FUSED_CASE(MUL, O_MUL) FUSED_CASE(DIV, O_DIV)
            FUSED_CASE(SDIV, O_SDIV) FUSED_CASE(MOD, O_MOD) FUSED_CASE(SMOD, O_SMOD) FUSED_CASE(OR, O_OR)
            FUSED_CASE(AND, O_AND) FUSED_CASE(XOR, O_XOR) FUSED_CASE(LSH, O_LSH) FUSED_CASE(RSH, O_RSH)
            FUSED_CASE(ARSH, O_ARSH) FUSED_CASE(MOV, O_MOV)
            JMP_FORM(J64K_, c64, (u64)(s64)imm)
            JMP_FORM(J64X_, c64, R[s])
            JMP_FORM(J32K_, c32, (u64)(u32)imm)
            JMP_FORM(J32X_, c32, R[s])
        case GXO_JA: taken = true; goto jump;
        case GXO_EXIT:
            if (!div) goto finished;
            pc = PC_DONE;
            continue;
        case GXO_NOP: break;
            /* ctx word k of this lane lives at ctxw[k * env.ctx_row + lane]; aux is the byte offset */
            LD_FORM(LDC, (const uint8_t *)(ctxw + (aux >> 3) * env.ctx_row + lane) + (aux & 7), CTX_OK)
            LD_FORM(LDS, (const uint8_t *)stack + aux, STK_OK)
            LD_FORM(LDM, (const uint8_t *)(R[s] + (u64)(s64)imm), LDM_OK)
            ST_FORM(STIS, (uint8_t *)stack + aux, (u64)(s64)imm, STK_OK)
            ST_FORM(STIM, (uint8_t *)(R[d] + (u64)(s64)(int16_t)aux), (u64)(s64)imm, STIM_OK)
            ST_FORM(STXS, (uint8_t *)stack + aux, R[s], STK_OK)
            ST_FORM(STXM, (uint8_t *)(R[d] + (u64)(s64)imm), R[s], DIMM_OK)
            ATOM_FORM(AS_, (u64)((uint8_t *)stack + aux), STK_OK)
            ATOM_FORM(AM_, R[d] + (u64)(s64)imm, DIMM_OK)
        case GXO_CALL_LOOKUP:
            CHK(MAP_OK(R[1]) && RANGE_OK(R[2], env.maps[R[1]].key_size))
            R[0] = map_lookup(env.maps[R[1]], (const uint8_t *)R[2], exec, env.stats);
            break;
        case GXO_CALL_UPDATE:
            CHK(MAP_OK(R[1]) && RANGE_OK(R[2], env.maps[R[1]].key_size) && RANGE_OK(R[3], env.maps[R[1]].value_size))
            R[0] = (u64)(s64)map_update(env.maps[R[1]], (const uint8_t *)R[2], (const uint8_t *)R[3], R[4], exec,
                                        env.stats);
            break;
        case GXO_CALL_DELETE: {
            CHK(MAP_OK(R[1]) && RANGE_OK(R[2], env.maps[R[1]].key_size))
            const gx_dmap &m = env.maps[R[1]];
            R[0] = (u64)(s64)(m.type == GX_MAP_HASH ? hash_delete(m, (const uint8_t *)R[2], env.stats) : GX_EINVAL);
            break;
        }
        case GXO_CALL_RB_RESERVE:
            CHK(RING_OK(R[1]))
            R[0] = rb_reserve(env.maps[R[1]], R[2], exec, ev_idx);
            break;
        case GXO_CALL_RB_OUTPUT: {
            CHK(RING_OK(R[1]) && RANGE_OK(R[2], R[3]))
            const u64 p = rb_reserve(env.maps[R[1]], R[3], exec, ev_idx);
            if (p) copy_bytes((uint8_t *)p, (const uint8_t *)R[2], (u32)R[3]);
            R[0] = p ? 0 : (u64)(s64)GX_EAGAIN;
            break;
        }
        case GXO_CALL_RB_SUBMIT: break; /* records are committed when reserved */
        case GXO_CALL_RB_DISCARD:
            CHK(MEM_OK(R[1] - GX_RB_HDR + 4, 4))
            ((u32 *)(R[1] - GX_RB_HDR))[1] = GX_RB_DISCARDED;
            break;
        case GXO_CALL_AMAX:
            CHK(MEM_OK(R[1], 8))
            agg_update<AG_MAX, 8>(R[1], R[2], exec);
            break;
        case GXO_CALL_AMIN:
            CHK(MEM_OK(R[1], 8))
            agg_update<AG_MIN, 8>(R[1], R[2], exec);
            break;
        default:
            set_status(env.stats, GX_E_DEVICE);
            R[0] = 0;
            pc = PC_DONE;
            if (!div) goto finished;
            continue;
        }
        pc++;
        continue;
    jump: {
        const u32 np = taken ? aux : pc + 1;
        if (!div) {
            const u32 b = __ballot_sync(FULLM, taken);
            if (b != 0 && b != FULLM) div = true;
        }
        if (np <= pc && ++back > env.budget) goto budget_trip;
        pc = np;
        continue;
    }
    budget_trip:
        atomicAdd(&env.stats[GX_STAT_BUDGET], 1ull);
        set_status(env.stats, GX_E_BUDGET);
        R[0] = 0;
        pc = PC_DONE;
        if (!div) break;
        continue;
    fault: /* checked build only (div is always set there): this lane's event stops */
        atomicCAS(&env.stats[GX_STAT_FAULT], 0ull, (u64)pc + 1);
        set_status(env.stats, GX_E_FAULT);
        R[0] = 0;
        pc = PC_DONE;
    }
finished:
    return R[0];
}

/* ------------------------------------------------------------------ kernels */
/*
 * Five blocks of 256 per SM (48 registers): the interpreter waits on its micro-op, register
 * and stack loads more than it computes, so more resident warps pay for the spills the
 * cap brings (three blocks ran page-heat 1.2 times and latency 1.3 times slower; eight
 * blocks, at 32 registers, 2 to 3 times slower).
 */
__global__ void __launch_bounds__(256, 5) gx_exec_kernel(ExecParams P) {
    exec_tiles(P, [](const ExecEnv &env, const u64 *ctxw, bool valid, u64 ev_idx) {
        return interp<false>(env, ctxw, valid, ev_idx);
    });
}

/* the checked build (GX_PROG_CHECKED): every access tested against the event's regions */
__global__ void __launch_bounds__(256, 3) gx_exec_kernel_checked(ExecParams P) {
    exec_tiles(P, [](const ExecEnv &env, const u64 *ctxw, bool valid, u64 ev_idx) {
        return interp<true>(env, ctxw, valid, ev_idx);
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
    cudaError_t e = cudaFuncSetAttribute(gx_exec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gx_exec_kernel_checked, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return e;
}

cudaError_t exec_occupancy(int block, size_t smem, int *blocks_per_sm, bool checked) {
    if (checked) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, gx_exec_kernel_checked, block, smem);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, gx_exec_kernel, block, smem);
}

cudaError_t launch_exec(const ExecParams &p, unsigned grid, unsigned block, size_t smem, cudaStream_t s, bool checked) {
    if (checked) gx_exec_kernel_checked<<<grid, block, smem, s>>>(p);
    else gx_exec_kernel<<<grid, block, smem, s>>>(p);
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
