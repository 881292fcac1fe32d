/*
 * Decoder: verified eBPF -> device micro-ops (layout in gx_layout.h).
 *
 * The paper specialises device handlers and inlines their helpers when it compiles them
 * (Sec. 4.4.2, Sec. 5.3); the engine's counterpart is done once at load time:
 * every instruction becomes one 16-byte micro-op that names its operation, registers,
 * the memory region (ctx / stack / global) and, for ctx and stack accesses, the absolute
 * offset proven by the verifier.  Jump offsets become absolute micro-op indices.
 */
#include <string>
#include <vector>

#include "gx_internal.h"

namespace gx {
namespace {

int size_index(int size) { return size == 1 ? 0 : size == 2 ? 1 : size == 4 ? 2 : 3; }
int size_of(int op) { return (op & 0x18) == 0x00 ? 4 : (op & 0x18) == 0x08 ? 2 : (op & 0x18) == 0x10 ? 1 : 8; }

/* index of an ALU operation in the O_* order of the device header (ADD .. MOV), -1 if none */
int alu_index(int code, int off) {
    switch (code) {
    case 0x00: return 0;            /* ADD */
    case 0x10: return 1;            /* SUB */
    case 0x20: return 2;            /* MUL */
    case 0x30: return off ? 4 : 3;  /* SDIV / DIV */
    case 0x90: return off ? 6 : 5;  /* SMOD / MOD */
    case 0x40: return 7;            /* OR */
    case 0x50: return 8;            /* AND */
    case 0xA0: return 9;            /* XOR */
    case 0x60: return 10;           /* LSH */
    case 0x70: return 11;           /* RSH */
    case 0xC0: return 12;           /* ARSH */
    case 0xB0: return 13;           /* MOV */
    }
    return -1;
}

int cond_index(int code) {
    switch (code) {
    case 0x10: return 0;  /* JEQ */
    case 0x50: return 1;  /* JNE */
    case 0x20: return 2;  /* JGT */
    case 0x30: return 3;  /* JGE */
    case 0xA0: return 4;  /* JLT */
    case 0xB0: return 5;  /* JLE */
    case 0x60: return 6;  /* JSGT */
    case 0x70: return 7;  /* JSGE */
    case 0xC0: return 8;  /* JSLT */
    case 0xD0: return 9;  /* JSLE */
    case 0x40: return 10; /* JSET */
    }
    return -1;
}

/* the atomic form index in GX_ATOM_OPS order: ADD/OR/AND/XOR x (4, 8) x (plain, fetch), XCHG, CMPXCHG */
int atom_index(int32_t imm, int size) {
    const int w8 = size == 8 ? 1 : 0;
    if (imm == 0xE1) return 16 + w8;
    if (imm == 0xF1) return 18 + w8;
    const int b = imm & ~1;
    const int o = b == 0x00 ? 0 : b == 0x40 ? 1 : b == 0x50 ? 2 : b == 0xA0 ? 3 : -1;
    if (o < 0) return -1;
    return ((imm & 1) ? 8 : 0) + w8 * 4 + o;
}

} // namespace

int decode_program(const uint64_t *insns, uint32_t n, const VerifyOut &v, std::vector<uint64_t> &uops,
                   std::string &log) {
    static_assert(GXO_A64X_ADD - GXO_A64K_ADD == 14 && GXO_A32K_ADD - GXO_A64K_ADD == 28, "ALU op order");
    static_assert(GXO_J64X_JEQ - GXO_J64K_JEQ == 11 && GXO_J32X_JEQ - GXO_J64K_JEQ == 33, "jump op order");
    static_assert(GXO_LDSS4 - GXO_LDS1 == 6 && GXO_AM_ADD4 - GXO_AS_ADD4 == 20, "memory op order");
    static_assert(GX_NUM_OPS <= 256, "operation field");
    static_assert(GXO_F64K_MOV - GXO_F64K_ADD == 13, "fused op order");
    uops.assign((size_t)n * 2, 0);
    /* instructions some jump lands on: a fused pair may not have its second one among them */
    std::vector<uint8_t> landed(n + 1, 0);
    for (uint32_t pc = 0; pc < n; pc++) {
        const uint64_t w = insns[pc];
        const int op = (int)(w & 0xFF), cls = op & 7, code = op & 0xF0;
        if (op == 0x18) {
            pc++;
            continue;
        }
        if ((cls == 5 || cls == 6) && code != 0x80 && code != 0x90) {
            const int64_t t = (int64_t)pc + 1 + ((cls == 6 && code == 0) ? (int32_t)(uint32_t)(w >> 32)
                                                                           : (int)(int16_t)(uint16_t)((w >> 16) & 0xFFFF));
            if (t >= 0 && t <= (int64_t)n) landed[t] = 1;
        }
    }
    /* one micro-op per instruction slot: micro-op k is instruction k, so jump targets stay */
    for (uint32_t pc = 0; pc < n; pc++) {
        const uint64_t w = insns[pc];
        const int op = (int)(w & 0xFF), cls = op & 7;
        const int dst = (int)((w >> 8) & 0xF), src = (int)((w >> 12) & 0xF);
        const int off = (int)(int16_t)(uint16_t)((w >> 16) & 0xFFFF);
        const int32_t imm = (int32_t)(uint32_t)(w >> 32);
        const InsnInfo &ii = v.info[pc];
        auto emit = [&](uint32_t o, uint32_t aux, int32_t im, uint64_t wide = 0) {
            uops[2 * pc] = gx_uop(o, (uint32_t)dst, (uint32_t)src, aux, im);
            uops[2 * pc + 1] = wide;
        };
        auto bad = [&](const char *what) {
            log = std::string("decoder: ") + what + " at insn " + std::to_string(pc);
            return GX_EINVAL;
        };
        if (!ii.visited) { /* never reached */
            emit(GXO_NOP, 0, 0);
            if (op == 0x18 && pc + 1 < n) {
                pc++;
                uops[2 * pc] = gx_uop(GXO_NOP, 0, 0, 0, 0);
            }
            continue;
        }
        switch (cls) {
        case 4: case 7: { /* ALU / ALU64 */
            const bool w32 = cls == 4, x = op & 8;
            const int code = op & 0xF0;
            if (code == 0xD0) {
                if (w32 && !x) emit(imm == 16 ? GXO_LE16 : imm == 32 ? GXO_LE32 : GXO_NOP, 0, 0);
                else emit(imm == 16 ? GXO_BSWAP16 : imm == 32 ? GXO_BSWAP32 : GXO_BSWAP64, 0, 0);
                break;
            }
            if (code == 0x80) {
                emit(w32 ? GXO_NEG32 : GXO_NEG64, 0, 0);
                break;
            }
            if (code == 0xB0 && off) { /* MOVSX */
                emit(w32 ? (off == 8 ? GXO_MOVSX32_8 : GXO_MOVSX32_16)
                         : (off == 8 ? GXO_MOVSX64_8 : off == 16 ? GXO_MOVSX64_16 : GXO_MOVSX64_32),
                     0, 0);
                break;
            }
            const int a = alu_index(code, (code == 0x30 || code == 0x90) ? off : 0);
            if (a < 0) return bad("unknown ALU operation");
            /* "mov d, s" then a 64-bit immediate operation on d, nothing jumping between them:
               one micro-op d = op(s, imm) that skips the second */
            if (op == 0xBF && !off && pc + 1 < n && !landed[pc + 1] && v.info[pc + 1].visited) {
                const uint64_t w2 = insns[pc + 1];
                const int op2 = (int)(w2 & 0xFF), code2 = op2 & 0xF0;
                const int off2 = (int)(int16_t)(uint16_t)((w2 >> 16) & 0xFFFF);
                const int a2 = (op2 & 0x0F) == 0x07 && code2 != 0xD0 && code2 != 0x80
                                   ? alu_index(code2, (code2 == 0x30 || code2 == 0x90) ? off2 : 0)
                                   : -1;
                if (a2 >= 0 && a2 != 13 && (int)((w2 >> 8) & 0xF) == dst && !(code2 == 0xB0 && off2)) {
                    emit(GXO_F64K_ADD + a2, 0, (int32_t)(uint32_t)(w2 >> 32));
                    break;
                }
            }
            emit(GXO_A64K_ADD + ((w32 ? 2 : 0) + (x ? 1 : 0)) * 14 + a, 0, imm);
            break;
        }
        case 5: case 6: { /* JMP / JMP32 */
            const int code = op & 0xF0;
            if (code == 0x00) {
                emit(GXO_JA, (uint32_t)((int64_t)pc + 1 + (cls == 6 ? imm : off)), 0);
                break;
            }
            if (code == 0x90) {
                emit(GXO_EXIT, 0, 0);
                break;
            }
            if (code == 0x80) {
                int o;
                switch (imm) {
                case GX_HELPER_MAP_LOOKUP: o = GXO_CALL_LOOKUP; break;
                case GX_HELPER_MAP_UPDATE: o = GXO_CALL_UPDATE; break;
                case GX_HELPER_MAP_DELETE: o = GXO_CALL_DELETE; break;
                case GX_HELPER_RINGBUF_OUTPUT: o = GXO_CALL_RB_OUTPUT; break;
                case GX_HELPER_RINGBUF_RESERVE: o = GXO_CALL_RB_RESERVE; break;
                case GX_HELPER_RINGBUF_SUBMIT: o = GXO_CALL_RB_SUBMIT; break;
                case GX_HELPER_RINGBUF_DISCARD: o = GXO_CALL_RB_DISCARD; break;
                case GX_HELPER_ATOMIC_MAX_U64: o = GXO_CALL_AMAX; break;
                case GX_HELPER_ATOMIC_MIN_U64: o = GXO_CALL_AMIN; break;
                default: return bad("unknown helper");
                }
                emit(o, 0, 0);
                break;
            }
            const int ci = cond_index(code);
            if (ci < 0) return bad("unknown jump");
            const int form = (cls == 6 ? 2 : 0) + ((op & 8) ? 1 : 0);
            emit(GXO_J64K_JEQ + form * 11 + ci, (uint32_t)((int64_t)pc + 1 + off), imm);
            break;
        }
        case 0: { /* 64-bit immediate; a map reference becomes the map's index */
            const uint64_t wide = src == 1 ? (uint64_t)(uint32_t)imm
                                           : ((uint64_t)(uint32_t)imm | ((insns[pc + 1] >> 32) << 32));
            emit(GXO_LDIMM64, 0, 0, wide);
            pc++;
            uops[2 * pc] = gx_uop(GXO_NOP, 0, 0, 0, 0);
            break;
        }
        case 1: { /* LDX: ctx and stack at the proven absolute offset, else through the register */
            const int size = size_of(op);
            const bool sign = (op & 0xE0) == 0x80;
            const int k = sign ? 4 + size_index(size) : size_index(size);
            if (ii.kind == MK_CTX) emit(GXO_LDC1 + k, (uint32_t)ii.off, 0);
            else if (ii.kind == MK_STACK) emit(GXO_LDS1 + k, (uint32_t)(ii.off + GX_STACK_BYTES), 0);
            else emit(GXO_LDM1 + k, 0, off);
            break;
        }
        case 2: case 3: { /* ST / STX / atomics */
            const int size = size_of(op), si = size_index(size);
            const bool stk = ii.kind == MK_STACK;
            const uint32_t aux = stk ? (uint32_t)(ii.off + GX_STACK_BYTES) : 0;
            if ((op & 0xE0) == 0xC0) {
                const int a = atom_index(imm, size);
                if (a < 0) return bad("unknown atomic");
                emit((stk ? GXO_AS_ADD4 : GXO_AM_ADD4) + a, aux, stk ? 0 : off);
                break;
            }
            if (cls == 2) emit((stk ? GXO_STIS1 : GXO_STIM1) + si, stk ? aux : (uint32_t)(uint16_t)(int16_t)off, imm);
            else emit((stk ? GXO_STXS1 : GXO_STXM1) + si, aux, stk ? 0 : off);
            break;
        }
        default: return bad("unknown instruction class");
        }
    }
    if (n >= 0xFFFF) {
        log = "decoded program too long";
        return GX_E2BIG;
    }
    return GX_OK;
}

} // namespace gx
