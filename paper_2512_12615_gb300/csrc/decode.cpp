/*
 * Decoder: verified eBPF -> device micro-ops (layout in gx_layout.h).
 *
 * The paper specialises device handlers and inlines their helpers when it compiles them
 * (Sec. 4.4.2, Sec. 5.3); the engine's counterpart is done once at load time:
 * every instruction becomes one to four micro-ops whose handler already names the
 * eBPF register, the memory region (ctx / stack / global) and, for ctx and stack
 * accesses, the absolute offset proven by the verifier.  Jump offsets become absolute
 * micro-op indices.
 */
#include <string>
#include <vector>

#include "gx_internal.h"

namespace gx {
namespace {

uint32_t H(int fam, int reg) { return (uint32_t)(fam * GX_HSTRIDE + reg); }
uint32_t S(int single) { return (uint32_t)(GX_SINGLE_BASE + single); }
int size_index(int size) { return size == 1 ? 0 : size == 2 ? 1 : size == 4 ? 2 : 3; }
int size_of(int op) { return (op & 0x18) == 0x00 ? 4 : (op & 0x18) == 0x08 ? 2 : (op & 0x18) == 0x10 ? 1 : 8; }

/* fast ALU family for (code, width, form), or -1 for the ops that go through A */
int fast_alu(int code, bool w32, bool x) {
    int base;
    switch (code) {
    case 0x00: base = 0; break; /* ADD */
    case 0x10: base = 1; break; /* SUB */
    case 0x20: base = 2; break; /* MUL */
    case 0x40: base = 3; break; /* OR */
    case 0x50: base = 4; break; /* AND */
    case 0xA0: base = 5; break; /* XOR */
    case 0x60: base = 6; break; /* LSH */
    case 0x70: base = 7; break; /* RSH */
    case 0xB0: base = 8; break; /* MOV */
    default: return -1;
    }
    return GXF_ADD64K + ((w32 ? 2 : 0) + (x ? 1 : 0)) * 9 + base;
}

/* accumulator form of DIV / SDIV / MOD / SMOD / ARSH */
int slow_alu(int code, int off, bool w32, bool x) {
    int base;
    switch (code) {
    case 0x30: base = off ? 1 : 0; break;
    case 0x90: base = off ? 3 : 2; break;
    case 0xC0: base = 4; break;
    default: return -1;
    }
    return GXS_DIV64K + ((w32 ? 2 : 0) + (x ? 1 : 0)) * 5 + base;
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

} // namespace

int decode_program(const uint64_t *insns, uint32_t n, const VerifyOut &v, std::vector<uint64_t> &uops,
                   std::string &log) {
    static_assert(GXF_MOV64K - GXF_ADD64K == 8 && GXF_ADD64T - GXF_ADD64K == 9 && GXF_ADD32T - GXF_ADD64K == 27,
                  "fast ALU family order");
    static_assert(GXF_JEQ64T - GXF_JEQ64K == 11 && GXF_JEQ32K - GXF_JEQ64K == 22, "fast jump family order");
    static_assert(GXS_ARSH64K - GXS_DIV64K == 4 && GXS_DIV64T - GXS_DIV64K == 5 && GXS_DIV32T - GXS_DIV64K == 15,
                  "slow ALU order");
    std::vector<uint32_t> first(n + 1, 0);
    /* pass 0 sizes the output, pass 1 emits with resolved jump targets */
    for (int pass = 0; pass < 2; pass++) {
        uops.clear();
        for (uint32_t pc = 0; pc < n; pc++) {
            first[pc] = (uint32_t)uops.size();
            const uint64_t w = insns[pc];
            const int op = (int)(w & 0xFF), cls = op & 7;
            const int dst = (int)((w >> 8) & 0xF), src = (int)((w >> 12) & 0xF);
            const int off = (int)(int16_t)(uint16_t)((w >> 16) & 0xFFFF);
            const int32_t imm = (int32_t)(uint32_t)(w >> 32);
            const InsnInfo &ii = v.info[pc];
            auto target = [&](int64_t rel) -> uint32_t { return pass ? first[(uint32_t)((int64_t)pc + 1 + rel)] : 0; };
            auto emit = [&](uint32_t h, uint32_t aux, int32_t im) { uops.push_back(gx_uop(h, aux, im)); };
            if (!ii.visited) { /* never reached: keep the index map simple */
                emit(S(GXS_NOP), 0, 0);
                if (op == 0x18 && pc + 1 < n) {
                    pc++;
                    first[pc] = (uint32_t)uops.size();
                    emit(S(GXS_NOP), 0, 0);
                }
                continue;
            }
            switch (cls) {
            case 4: case 7: { /* ALU / ALU64 */
                const bool w32 = cls == 4, x = op & 8;
                const int code = op & 0xF0;
                if (code == 0xD0) { /* byte swaps through A */
                    int sgl;
                    if (w32 && !x) {
                        if (imm == 64) {
                            emit(S(GXS_NOP), 0, 0);
                            break;
                        }
                        sgl = imm == 16 ? GXS_LE16 : GXS_LE32;
                    } else {
                        sgl = imm == 16 ? GXS_BSWAP16 : imm == 32 ? GXS_BSWAP32 : GXS_BSWAP64;
                    }
                    emit(H(GXF_MOVA, dst), 0, 0);
                    emit(S(sgl), 0, 0);
                    emit(H(GXF_MOVRA, dst), 0, 0);
                    break;
                }
                if (code == 0x80) {
                    emit(H(GXF_MOVA, dst), 0, 0);
                    emit(S(w32 ? GXS_NEG32 : GXS_NEG64), 0, 0);
                    emit(H(GXF_MOVRA, dst), 0, 0);
                    break;
                }
                if (code == 0xB0 && off) { /* MOVSX: A = sign-extend(T) */
                    int sgl = w32 ? (off == 8 ? GXS_MOVSX32_8 : GXS_MOVSX32_16)
                                  : (off == 8 ? GXS_MOVSX64_8 : off == 16 ? GXS_MOVSX64_16 : GXS_MOVSX64_32);
                    emit(H(GXF_MOVT, src), 0, 0);
                    emit(S(sgl), 0, 0);
                    emit(H(GXF_MOVRA, dst), 0, 0);
                    break;
                }
                int f = fast_alu(code, w32, x);
                if (f >= 0 && !(code == 0x30 || code == 0x90)) {
                    if (x) emit(H(GXF_MOVT, src), 0, 0);
                    emit(H(f, dst), 0, imm);
                    break;
                }
                int sgl = slow_alu(code, off, w32, x);
                if (sgl < 0) {
                    log = "decoder: unknown ALU operation at insn " + std::to_string(pc);
                    return GX_EINVAL;
                }
                if (x) emit(H(GXF_MOVT, src), 0, 0);
                emit(H(GXF_MOVA, dst), 0, 0);
                emit(S(sgl), 0, imm);
                emit(H(GXF_MOVRA, dst), 0, 0);
                break;
            }
            case 5: case 6: { /* JMP / JMP32 */
                const int code = op & 0xF0;
                if (code == 0x00) {
                    emit(S(GXS_JA), target(cls == 6 ? imm : off), 0);
                    break;
                }
                if (code == 0x90) {
                    emit(S(GXS_EXIT), 0, 0);
                    break;
                }
                if (code == 0x80) {
                    int sgl;
                    switch (imm) {
                    case GX_HELPER_MAP_LOOKUP: sgl = GXS_CALL_LOOKUP; break;
                    case GX_HELPER_MAP_UPDATE: sgl = GXS_CALL_UPDATE; break;
                    case GX_HELPER_MAP_DELETE: sgl = GXS_CALL_DELETE; break;
                    case GX_HELPER_RINGBUF_OUTPUT: sgl = GXS_CALL_RB_OUTPUT; break;
                    case GX_HELPER_RINGBUF_RESERVE: sgl = GXS_CALL_RB_RESERVE; break;
                    case GX_HELPER_RINGBUF_SUBMIT: sgl = GXS_CALL_RB_SUBMIT; break;
                    case GX_HELPER_RINGBUF_DISCARD: sgl = GXS_CALL_RB_DISCARD; break;
                    case GX_HELPER_ATOMIC_MAX_U64: sgl = GXS_CALL_AMAX; break;
                    case GX_HELPER_ATOMIC_MIN_U64: sgl = GXS_CALL_AMIN; break;
                    default: log = "decoder: unknown helper"; return GX_EINVAL;
                    }
                    emit(S(sgl), 0, 0);
                    break;
                }
                const bool x = op & 8, w32 = cls == 6;
                const int ci = cond_index(code);
                if (ci < 0) {
                    log = "decoder: unknown jump at insn " + std::to_string(pc);
                    return GX_EINVAL;
                }
                if (w32 && x) { /* 32-bit register compare: A (dst) against T (src) */
                    emit(H(GXF_MOVA, dst), 0, 0);
                    emit(H(GXF_MOVT, src), 0, 0);
                    emit(S(GXS_JEQ32A + ci), target(off), 0);
                    break;
                }
                const int f = GXF_JEQ64K + (w32 ? 22 : x ? 11 : 0) + ci;
                if (x) emit(H(GXF_MOVT, src), 0, 0);
                emit(H(f, dst), target(off), imm);
                break;
            }
            case 0: { /* 64-bit immediate; a map reference becomes the map index */
                if (src == 1) emit(H(GXF_MOV64K, dst), 0, imm);
                else emit(H(GXF_LDIMM64, dst), 0, imm);
                pc++;
                first[pc] = (uint32_t)uops.size();
                emit(S(GXS_NOP), 0, (int32_t)(uint32_t)(insns[pc] >> 32));
                break;
            }
            case 1: { /* LDX */
                const int size = size_of(op);
                const bool sign = (op & 0xE0) == 0x80;
                const int k = sign ? 4 + size_index(size) : size_index(size);
                if (ii.kind == MK_CTX) {
                    emit(H(GXF_LDXC1 + k, dst), (uint32_t)ii.off, 0);
                } else if (ii.kind == MK_STACK) {
                    emit(H(GXF_LDXS1 + k, dst), (uint32_t)(ii.off + GX_STACK_BYTES), 0);
                } else {
                    emit(H(GXF_MOVB, src), 0, 0);
                    emit(H(GXF_LDXM1 + k, dst), 0, off);
                }
                break;
            }
            case 2: case 3: { /* ST / STX / atomics */
                const int size = size_of(op), si = size_index(size);
                if ((op & 0xE0) == 0xC0) {
                    if (ii.kind == MK_STACK) emit(S(GXS_MOVB_STK), (uint32_t)(ii.off + GX_STACK_BYTES), 0);
                    else emit(H(GXF_MOVB, dst), 0, 0);
                    const int32_t moff = ii.kind == MK_STACK ? 0 : off;
                    const bool w8 = size == 8;
                    emit(H(GXF_MOVT, src), 0, 0);
                    if (imm == 0xF1) {
                        emit(S(w8 ? GXS_ACMPX8 : GXS_ACMPX4), 0, moff);
                    } else if (imm == 0xE1) {
                        emit(S(w8 ? GXS_AXCHG8 : GXS_AXCHG4), 0, moff);
                        emit(H(GXF_MOVR, src), 0, 0);
                    } else {
                        const int o = (imm & ~1) == 0x00 ? 0 : (imm & ~1) == 0x40 ? 1 : (imm & ~1) == 0x50 ? 2 : 3;
                        emit(S((imm & 1 ? GXS_AFADD4 : GXS_AADD4) + (w8 ? 4 : 0) + o), 0, moff);
                        if (imm & 1) emit(H(GXF_MOVR, src), 0, 0);
                    }
                    break;
                }
                if (ii.kind == MK_STACK) {
                    const uint32_t a = (uint32_t)(ii.off + GX_STACK_BYTES);
                    if (cls == 2) {
                        emit(S(GXS_ST_S1 + si), a, imm);
                    } else if (src <= 9) {
                        emit(H(GXF_STXS1 + si, src), a, 0);
                    } else {
                        emit(H(GXF_MOVT, src), 0, 0);
                        emit(S(GXS_STT_S1 + si), a, 0);
                    }
                } else {
                    emit(H(GXF_MOVB, dst), 0, 0);
                    if (cls == 2) {
                        emit(S(GXS_ST_M1 + si), (uint32_t)(uint16_t)(int16_t)off, imm);
                    } else {
                        emit(H(GXF_MOVT, src), 0, 0);
                        emit(S(GXS_STT_M1 + si), 0, off);
                    }
                }
                break;
            }
            }
        }
        first[n] = (uint32_t)uops.size();
        if (uops.size() >= 0xFFFF) {
            log = "decoded program too long";
            return GX_E2BIG;
        }
    }
    return GX_OK;
}

} // namespace gx
