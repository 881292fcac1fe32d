/*
 * Program verifier and decoder.
 *
 * The paper verifies every device program before it runs: standard eBPF typing,
 * bounded loops and memory safety, plus per-hook resource budgets (Sec. 4.4, Sec. 5.3).
 * This verifier is written from scratch for the engine: a path-sensitive abstract
 * interpreter over the standard eBPF ISA (RFC 9669).
 *
 *   Register types: uninitialised, scalar (unsigned and signed ranges, known trailing
 *   zero bits, an order-dependence taint), ctx pointer, stack pointer, map handle, map
 *   value pointer (+ maybe-NULL form), ring-buffer record pointer (+ maybe-NULL form).
 *   Pointers carry an offset range; ctx and stack offsets must be constants.
 *   Stack: 512 bytes tracked per byte (invalid / written / spilled register).
 *   Memory: every access in bounds of its region and naturally aligned; ctx read-only;
 *   pointers never leak into scalars, memory or maps.
 *   Control flow: jumps stay inside the program, never into the second slot of a 64-bit
 *   immediate, execution never falls off the end.  Loops are allowed when exploration
 *   finishes within GX_VERIFY_BUDGET processed instructions; a state that repeats an
 *   ancestor state exactly is an infinite loop.  States at jump targets are kept, and a
 *   new state that lies inside a kept one (ignoring dead registers) is pruned.
 *   Ring-buffer reservations must be submitted or discarded on every path.
 *   Deterministic mode (an engine reading of the paper's relaxed map consistency,
 *   Sec. 4.4.3): values read back from maps, fetched by atomics or returned by updates
 *   are tainted and may not reach branch conditions, R0 at exit, map keys, stored map
 *   values, ring-buffer payloads or pointer offsets; map values change only through
 *   ADD/OR/AND/XOR atomics without fetch or the atomic max/min helpers, adds to the same
 *   bytes at one width (a 32-bit add drops the carry a 64-bit add keeps); updates must be
 *   NOEXIST inserts of constant bytes, one constant per map; deletes, XCHG and CMPXCHG on
 *   map memory are refused.  Under these rules the final map state, the set of ring-buffer
 *   records and every R0 are the same for every order in which the events run.
 *   SIMT mode (gx_verify_simt; the warp-uniformity pass and per-hook budgets of Sec. 4.4.1
 *   and Sec. 5.3): a second mark, lane-varying, starts at the ctx bytes not declared
 *   warp-uniform and flows like the taint through registers, spills and stack bytes.  A
 *   value the abstract state pins to one constant is uniform whatever its mark: control
 *   flow is uniform, so every lane holds that constant.  Lane-varying values may not reach
 *   branch conditions, map keys, helper arguments, R0 at exit, or the address or operand
 *   of a store or atomic into map or ring-buffer memory; the warp helpers turn them into
 *   uniform values.  Each path also counts its instructions, helper calls and memory
 *   operations against the hook's budgets; a state is pruned only by a kept state whose
 *   counts are at least as large, so the maxima found are the maxima over all paths.
 */
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "gx_internal.h"

namespace gx {
namespace {

typedef uint64_t u64;
typedef int64_t s64;
typedef uint32_t u32;

const u64 GX_VERIFY_BUDGET = 1000000;
const int MAX_STATES_PER_PC = 64;
const size_t MAX_STATES_TOTAL = 16384;

enum RT : uint8_t { NI = 0, SC, CTX, STK, CMAP, MV, MVN, RB, RBN };
const uint8_t ST_LV = 0x40, ST_TAINT = 0x80;

const char *rt_name(int t) {
    static const char *n[] = {"uninit", "scalar", "ctx", "stack", "map", "map_value", "map_value_or_null",
                              "ringbuf_mem", "ringbuf_mem_or_null"};
    return n[t];
}

struct Reg {
    uint8_t t = NI;
    uint8_t taint = 0;
    uint8_t lv = 0; /* SIMT mode: lane-varying */
    uint8_t map = 0;
    uint8_t tz = 0; /* known zero low bits of the value (scalar) or offset (pointer) */
    u32 id = 0;     /* maybe-NULL group / ring-buffer reference */
    u32 size = 0;   /* ring-buffer record size */
    u64 umin = 0, umax = 0;
    s64 smin = 0, smax = 0;
};

bool same(const Reg &a, const Reg &b) {
    return a.t == b.t && a.taint == b.taint && a.lv == b.lv && a.map == b.map && a.tz == b.tz && a.id == b.id && a.size == b.size &&
           a.umin == b.umin && a.umax == b.umax && a.smin == b.smin && a.smax == b.smax;
}

int ctz64(u64 v) { return v ? __builtin_ctzll(v) : 64; }

/* a value that may differ between the lanes of a warp (a constant cannot) */
bool varies(const Reg &r) { return r.lv && !(r.umin == r.umax); }

Reg sc_const(u64 v) {
    Reg r;
    r.t = SC;
    r.umin = r.umax = v;
    r.smin = r.smax = (s64)v;
    r.tz = (uint8_t)ctz64(v);
    return r;
}

Reg sc_unknown() {
    Reg r;
    r.t = SC;
    r.umin = 0;
    r.umax = ~0ULL;
    r.smin = INT64_MIN;
    r.smax = INT64_MAX;
    r.tz = 0;
    return r;
}

Reg sc_range(u64 lo, u64 hi) {
    Reg r = sc_unknown();
    r.umin = lo;
    r.umax = hi;
    return r;
}

bool is_const(const Reg &r) { return r.umin == r.umax; }

/* tighten the unsigned and signed views against each other; false if empty */
bool sync(Reg &r) {
    for (int it = 0; it < 2; it++) {
        if (r.smin >= 0 || r.smax < 0) { /* signed range does not cross the sign boundary */
            r.umin = std::max(r.umin, (u64)r.smin);
            r.umax = std::min(r.umax, (u64)r.smax);
        }
        if ((s64)r.umin >= 0 && (s64)r.umax >= 0) {
            r.smin = std::max(r.smin, (s64)r.umin);
            r.smax = std::min(r.smax, (s64)r.umax);
        } else if ((s64)r.umin < 0 && (s64)r.umax < 0) {
            r.smin = std::max(r.smin, (s64)r.umin);
            r.smax = std::min(r.smax, (s64)r.umax);
        }
    }
    if (r.umin > r.umax || r.smin > r.smax) return false;
    if (r.umin == r.umax) r.tz = (uint8_t)ctz64(r.umin);
    return true;
}

/* ------------------------------------------------------------ concrete ALU (RFC 9669 Sec. 4.1) */
u64 bswap_n(u64 v, int bits) {
    u64 r = 0;
    for (int i = 0; i < bits / 8; i++) r = (r << 8) | ((v >> (8 * i)) & 0xFF);
    return r;
}

u64 sx(u64 v, int bits) {
    if (bits >= 64) return v;
    u64 m = 1ULL << (bits - 1);
    v &= (1ULL << bits) - 1;
    return (v ^ m) - m;
}

u64 eval_alu(int code, bool w32, int off, u64 d, u64 s) {
    if (w32) {
        d &= 0xFFFFFFFFULL;
        s &= 0xFFFFFFFFULL;
    }
    u64 r = 0;
    int sh = w32 ? 31 : 63;
    switch (code) {
    case 0x00: r = d + s; break;
    case 0x10: r = d - s; break;
    case 0x20: r = d * s; break;
    case 0x30:
        if (off == 0) r = s ? d / s : 0;
        else if (w32) {
            int32_t a = (int32_t)d, b = (int32_t)s;
            r = b == 0 ? 0 : (a == INT32_MIN && b == -1) ? (u64)(uint32_t)a : (u64)(uint32_t)(a / b);
        } else {
            s64 a = (s64)d, b = (s64)s;
            r = b == 0 ? 0 : (a == INT64_MIN && b == -1) ? (u64)a : (u64)(a / b);
        }
        break;
    case 0x40: r = d | s; break;
    case 0x50: r = d & s; break;
    case 0x60: r = d << (s & sh); break;
    case 0x70: r = d >> (s & sh); break;
    case 0x80: r = 0 - d; break;
    case 0x90:
        if (off == 0) r = s ? d % s : d;
        else if (w32) {
            int32_t a = (int32_t)d, b = (int32_t)s;
            r = b == 0 ? (u64)(uint32_t)a : b == -1 ? 0 : (u64)(uint32_t)(a % b);
        } else {
            s64 a = (s64)d, b = (s64)s;
            r = b == 0 ? (u64)a : b == -1 ? 0 : (u64)(a % b);
        }
        break;
    case 0xA0: r = d ^ s; break;
    case 0xB0: r = off ? sx(s, off) : s; break;
    case 0xC0:
        r = w32 ? (u64)(uint32_t)((int32_t)d >> (s & 31)) : (u64)((s64)d >> (s & 63));
        break;
    }
    return w32 ? (r & 0xFFFFFFFFULL) : r;
}

bool eval_cond(int code, bool w32, u64 d, u64 s) {
    if (w32) {
        d &= 0xFFFFFFFFULL;
        s &= 0xFFFFFFFFULL;
    }
    s64 sd = w32 ? (s64)(int32_t)d : (s64)d, ss = w32 ? (s64)(int32_t)s : (s64)s;
    switch (code) {
    case 0x10: return d == s;
    case 0x20: return d > s;
    case 0x30: return d >= s;
    case 0x40: return (d & s) != 0;
    case 0x50: return d != s;
    case 0x60: return sd > ss;
    case 0x70: return sd >= ss;
    case 0xA0: return d < s;
    case 0xB0: return d <= s;
    case 0xC0: return sd < ss;
    case 0xD0: return sd <= ss;
    }
    return false;
}

/* ------------------------------------------------------------ abstract ALU */
u64 ones_below(u64 m) { return m ? (~0ULL >> __builtin_clzll(m)) : 0; }

Reg trunc32(const Reg &a) {
    if (a.umax <= 0xFFFFFFFFULL) return a;
    if (is_const(a)) {
        Reg c = sc_const(a.umin & 0xFFFFFFFFULL);
        c.taint = a.taint;
        c.lv = a.lv;
        return c;
    }
    Reg r = sc_range(0, 0xFFFFFFFFULL);
    r.tz = std::min<int>(a.tz, 32);
    r.taint = a.taint;
    r.lv = a.lv;
    sync(r);
    return r;
}

Reg abs_alu64(int code, int off, const Reg &a, const Reg &b) {
    Reg r = sc_unknown();
    switch (code) {
    case 0x00:
        if (a.umax <= ~b.umax) {
            r.umin = a.umin + b.umin;
            r.umax = a.umax + b.umax;
        }
        {
            s64 lo, hi;
            if (!__builtin_add_overflow(a.smin, b.smin, &lo) && !__builtin_add_overflow(a.smax, b.smax, &hi)) {
                r.smin = lo;
                r.smax = hi;
            }
        }
        r.tz = std::min(a.tz, b.tz);
        break;
    case 0x10:
        if (a.umin >= b.umax) {
            r.umin = a.umin - b.umax;
            r.umax = a.umax - b.umin;
        }
        {
            s64 lo, hi;
            if (!__builtin_sub_overflow(a.smin, b.smax, &lo) && !__builtin_sub_overflow(a.smax, b.smin, &hi)) {
                r.smin = lo;
                r.smax = hi;
            }
        }
        r.tz = std::min(a.tz, b.tz);
        break;
    case 0x20: {
        u64 hi;
        if (!__builtin_mul_overflow(a.umax, b.umax, &hi)) {
            r.umin = a.umin * b.umin;
            r.umax = hi;
        }
        r.tz = (uint8_t)std::min(64, a.tz + b.tz);
        break;
    }
    case 0x30:
        if (off == 0) {
            if (is_const(b) && b.umin) {
                r.umin = a.umin / b.umin;
                r.umax = a.umax / b.umin;
            } else {
                r.umax = a.umax;
            }
        }
        break;
    case 0x90:
        if (off == 0) {
            if (is_const(b) && b.umin && a.umax >= b.umin) r.umax = b.umin - 1;
            else r.umax = a.umax;
        }
        break;
    case 0x40:
        r.umin = std::max(a.umin, b.umin);
        r.umax = ones_below(std::max(a.umax, b.umax));
        r.tz = std::min(a.tz, b.tz);
        break;
    case 0x50:
        r.umax = std::min(a.umax, b.umax);
        r.tz = std::max(a.tz, b.tz);
        break;
    case 0xA0:
        r.umax = ones_below(std::max(a.umax, b.umax));
        r.tz = std::min(a.tz, b.tz);
        break;
    case 0x60:
        if (is_const(b)) {
            int k = (int)(b.umin & 63);
            if (a.umax <= (~0ULL >> k)) {
                r.umin = a.umin << k;
                r.umax = a.umax << k;
            }
            r.tz = (uint8_t)std::min(64, a.tz + k);
        }
        break;
    case 0x70:
        if (is_const(b)) {
            int k = (int)(b.umin & 63);
            r.umin = a.umin >> k;
            r.umax = a.umax >> k;
            r.tz = (uint8_t)(a.tz > k ? a.tz - k : 0);
        } else {
            r.umax = a.umax;
        }
        break;
    case 0xC0:
        if (is_const(b)) {
            int k = (int)(b.umin & 63);
            r.smin = a.smin >> k;
            r.smax = a.smax >> k;
        }
        break;
    case 0xB0:
        if (off == 0) r = b;
        else {
            s64 lim = (s64)1 << (off - 1);
            r.smin = -lim;
            r.smax = lim - 1;
        }
        break;
    default: break; /* SDIV, SMOD, NEG: unknown */
    }
    if (!sync(r)) r = sc_unknown();
    return r;
}

Reg abs_alu(int code, bool w32, int off, const Reg &a, const Reg &b) {
    Reg r;
    if (is_const(a) && is_const(b)) {
        r = sc_const(eval_alu(code, w32, off, a.umin, b.umin));
    } else if (!w32) {
        r = abs_alu64(code, off, a, b);
    } else {
        Reg a32 = trunc32(a), b32 = trunc32(b);
        if (code == 0x60 || code == 0x70) { /* 32-bit shift counts are masked to 31 */
            if (is_const(b32)) b32 = sc_const(b32.umin & 31);
        }
        bool exact32 = code != 0x30 && code != 0x90 ? true : off == 0;
        if (code == 0xC0 || code == 0x80 || (code == 0xB0 && off) || !exact32) {
            r = sc_range(0, 0xFFFFFFFFULL);
        } else {
            r = abs_alu64(code, off, a32, b32);
            if (r.umax > 0xFFFFFFFFULL) {
                uint8_t tz = std::min<uint8_t>(r.tz, 32);
                r = sc_range(0, 0xFFFFFFFFULL);
                r.tz = tz;
            }
        }
        r.smin = (s64)r.umin;
        r.smax = (s64)r.umax;
        if (!sync(r)) r = sc_range(0, 0xFFFFFFFFULL);
    }
    r.taint = a.taint | b.taint;
    r.lv = a.lv | b.lv;
    return r;
}

/* ------------------------------------------------------------ verifier state */
enum SB : uint8_t { S_INV = 0, S_MISC = 1, S_SPILL = 2 };

struct State {
    Reg r[11];
    uint8_t st[GX_STACK_BYTES]; /* SB in bits 0..1, lane-varying in bit 6, taint in bit 7 */
    Reg spill[GX_STACK_BYTES / 8];
    u32 refs[8];
    uint8_t nrefs = 0;
    u32 c_insn = 0, c_help = 0, c_mem = 0; /* SIMT mode: this path's instructions, helper calls, memory ops */
    State() {
        memset(st, 0, sizeof st);
        memset(refs, 0, sizeof refs);
    }
};

struct Node {
    State st;
    int parent;
};

struct Pending {
    State st;
    u32 pc;
    int parent;
};

struct Verifier {
    const uint64_t *insns;
    u32 n;
    const gx_map_spec *maps;
    u32 n_maps;
    gx_prog_opts opts;
    VerifyOut *out;
    std::vector<uint16_t> live; /* registers live on entry, bit per register */
    std::vector<uint8_t> prune, second;
    std::vector<Node> nodes;
    std::vector<std::vector<int>> visited;
    /* deterministic mode: which atomic operation class updates which bytes of each map */
    struct OpRange {
        s64 lo, hi;
        int cls, size;
    };
    std::vector<OpRange> op_ranges[GX_MAX_MAPS];
    u32 next_id = 1;
    char msg[512];
    const SimtIn *simt = nullptr; /* SIMT mode when set */
    bool sm = false;
    std::vector<uint8_t> simt_branch, simt_vary; /* per instruction: a uniform open branch / a varying value */

    int vfail(u32 pc, const char *fmt, va_list ap) {
        vsnprintf(msg, sizeof msg, fmt, ap);
        char buf[640];
        snprintf(buf, sizeof buf, "insn %u: %s", pc, msg);
        out->log = buf;
        out->fail_pc = (int32_t)pc;
        return GX_E_VERIFY;
    }
    int fail(u32 pc, const char *fmt, ...) __attribute__((format(printf, 3, 4))) {
        va_list ap;
        va_start(ap, fmt);
        int rc = vfail(pc, fmt, ap);
        va_end(ap);
        return rc;
    }
    /* a SIMT-mode rejection with its GX_SIMT_V_* reason */
    int sfail(u32 pc, u32 why, const char *fmt, ...) __attribute__((format(printf, 4, 5))) {
        out->simt.violation = why;
        out->simt.pc = (int32_t)pc;
        va_list ap;
        va_start(ap, fmt);
        int rc = vfail(pc, fmt, ap);
        va_end(ap);
        return rc;
    }
    /* SIMT mode: some byte of ctx[a, a + size) is not declared warp-uniform */
    bool ctx_varies(s64 a, int size) {
        if (!sm) return false;
        for (s64 b = a; b < a + size; b++)
            if (!simt->uniform[(size_t)b]) return true;
        return false;
    }
    void note_vary(u32 pc, const Reg &r) {
        if (sm && varies(r)) simt_vary[pc] = 1;
    }

    /* ---------------------------------------------------- decode helpers */
    static int op_of(u64 w) { return (int)(w & 0xFF); }
    static int dst_of(u64 w) { return (int)((w >> 8) & 0xF); }
    static int src_of(u64 w) { return (int)((w >> 12) & 0xF); }
    static int off_of(u64 w) { return (int)(int16_t)(uint16_t)((w >> 16) & 0xFFFF); }
    static int32_t imm_of(u64 w) { return (int32_t)(uint32_t)(w >> 32); }
    static int size_of(int op) {
        switch (op & 0x18) {
        case 0x00: return 4;
        case 0x08: return 2;
        case 0x10: return 1;
        default: return 8;
        }
    }

    int helper_args(int32_t id) {
        switch (id) {
        case GX_HELPER_MAP_LOOKUP: return 2;
        case GX_HELPER_MAP_UPDATE: return 4;
        case GX_HELPER_MAP_DELETE: return 2;
        case GX_HELPER_RINGBUF_OUTPUT: return 4;
        case GX_HELPER_RINGBUF_RESERVE: return 3;
        case GX_HELPER_RINGBUF_SUBMIT: return 2;
        case GX_HELPER_RINGBUF_DISCARD: return 2;
        case GX_HELPER_ATOMIC_MAX_U64: return 2;
        case GX_HELPER_ATOMIC_MIN_U64: return 2;
        case GX_HELPER_WARP_SUM_U64:
        case GX_HELPER_WARP_MAX_U64:
        case GX_HELPER_WARP_MIN_U64:
        case GX_HELPER_WARP_OR_U64:
        case GX_HELPER_WARP_AND_U64:
        case GX_HELPER_WARP_COUNT: return sm ? 1 : -1;
        }
        return -1;
    }

    /* structural pass: successors, liveness, prune points */
    int structure() {
        second.assign(n, 0);
        prune.assign(n, 0);
        for (u32 pc = 0; pc < n; pc++) {
            if (op_of(insns[pc]) == 0x18) {
                if (pc + 1 >= n) return fail(pc, "64-bit immediate load is missing its second slot");
                u64 w2 = insns[pc + 1];
                if ((w2 & 0xFFFFFFFFULL) != 0) return fail(pc + 1, "second slot of a 64-bit immediate must be zero except imm");
                second[pc + 1] = 1;
                pc++;
            }
        }
        std::vector<std::vector<u32>> succ(n);
        std::vector<uint16_t> use(n, 0), def(n, 0);
        for (u32 pc = 0; pc < n; pc++) {
            if (second[pc]) continue;
            u64 w = insns[pc];
            int op = op_of(w), cls = op & 7, dst = dst_of(w), src = src_of(w);
            if (dst > 10 || src > 10) return fail(pc, "register number out of range");
            auto jt = [&](s64 rel, u32 &t) -> int {
                s64 tgt = (s64)pc + 1 + rel;
                if (tgt < 0 || tgt >= (s64)n) return fail(pc, "jump out of range");
                if (second[tgt]) return fail(pc, "jump into the middle of a 64-bit immediate load");
                t = (u32)tgt;
                return GX_OK;
            };
            u32 t;
            switch (cls) {
            case 4: case 7: {
                int code = op & 0xF0;
                bool x = op & 8;
                if (code == 0xB0 && !x) def[pc] |= 1 << dst;
                else if (code == 0xB0) {
                    use[pc] |= 1 << src;
                    def[pc] |= 1 << dst;
                } else {
                    use[pc] |= 1 << dst;
                    if (x && code != 0xD0 && code != 0x80) use[pc] |= 1 << src;
                    def[pc] |= 1 << dst;
                }
                if (pc + 1 < n) succ[pc].push_back(pc + 1);
                break;
            }
            case 5: case 6: {
                int code = op & 0xF0;
                if (code == 0x00) {
                    if (jt(cls == 6 ? imm_of(w) : off_of(w), t)) return GX_E_VERIFY;
                    succ[pc].push_back(t);
                    prune[t] = 1;
                } else if (code == 0x80 && cls == 5) {
                    int k = helper_args(imm_of(w));
                    for (int i = 1; i <= std::max(0, k); i++) use[pc] |= 1 << i;
                    def[pc] |= 0x3F; /* R0 written, R1..R5 clobbered */
                    if (pc + 1 < n) succ[pc].push_back(pc + 1);
                } else if (code == 0x90 && cls == 5) {
                    use[pc] |= 1;
                } else {
                    use[pc] |= 1 << dst;
                    if (op & 8) use[pc] |= 1 << src;
                    if (jt(off_of(w), t)) return GX_E_VERIFY;
                    succ[pc].push_back(t);
                    prune[t] = 1;
                    if (pc + 1 < n) {
                        succ[pc].push_back(pc + 1);
                        prune[pc + 1] = 1;
                    }
                }
                break;
            }
            case 0:
                def[pc] |= 1 << dst;
                if (pc + 2 < n) succ[pc].push_back(pc + 2);
                break;
            case 1:
                use[pc] |= 1 << src;
                def[pc] |= 1 << dst;
                if (pc + 1 < n) succ[pc].push_back(pc + 1);
                break;
            case 2:
                use[pc] |= 1 << dst;
                if (pc + 1 < n) succ[pc].push_back(pc + 1);
                break;
            case 3:
                use[pc] |= (1 << dst) | (1 << src);
                if ((op & 0xE0) == 0xC0) {
                    if ((imm_of(w) & 1)) def[pc] |= 1 << src;
                    if (imm_of(w) == 0xF1) {
                        use[pc] |= 1;
                        def[pc] |= 1;
                    }
                }
                if (pc + 1 < n) succ[pc].push_back(pc + 1);
                break;
            }
        }
        /* backward liveness to a fixed point */
        live.assign(n, 0);
        bool changed = true;
        while (changed) {
            changed = false;
            for (u32 k = n; k-- > 0;) {
                if (second[k]) continue;
                uint16_t outl = 0;
                for (u32 s : succ[k]) outl |= live[s];
                uint16_t in = (uint16_t)(use[k] | (outl & ~def[k]));
                if (in != live[k]) {
                    live[k] = in;
                    changed = true;
                }
            }
        }
        return GX_OK;
    }

    /* ---------------------------------------------------- state comparison */
    struct IdMap {
        std::vector<std::pair<u32, u32>> m;
        bool check(u32 a, u32 b) {
            for (auto &p : m) {
                if (p.first == a) return p.second == b;
                if (p.second == b) return false;
            }
            m.push_back({a, b});
            return true;
        }
    };

    static bool reg_within(const Reg &o, const Reg &c, IdMap &ids) {
        if (o.t == NI) return true;
        if (o.t != c.t) return false;
        if (c.taint && !o.taint) return false;
        if (c.lv && !o.lv) return false;
        if (o.t == CMAP) return o.map == c.map;
        if (o.t == CTX || o.t == STK || o.t == SC || o.t == MV || o.t == MVN || o.t == RB || o.t == RBN) {
            if (o.map != c.map || o.size != c.size) return false;
            if (!(o.umin <= c.umin && c.umax <= o.umax && o.smin <= c.smin && c.smax <= o.smax && o.tz <= c.tz))
                return false;
            if (o.t == MVN || o.t == RB || o.t == RBN) return ids.check(o.id, c.id);
            return true;
        }
        return false;
    }

    bool within(const State &o, const State &c, uint16_t livemask) {
        IdMap ids;
        for (int i = 0; i < 11; i++)
            if ((livemask >> i) & 1)
                if (!reg_within(o.r[i], c.r[i], ids)) return false;
        for (int b = 0; b < GX_STACK_BYTES; b++) {
            int ot = o.st[b] & 3, ct = c.st[b] & 3;
            if (ot == S_INV) continue;
            if ((c.st[b] & ST_TAINT) && !(o.st[b] & ST_TAINT)) return false;
            if ((c.st[b] & ST_LV) && !(o.st[b] & ST_LV)) return false;
            if (ot == S_MISC) {
                if (ct == S_INV) return false;
                if (ct == S_SPILL && c.spill[b / 8].t != SC) return false;
                continue;
            }
            if (ct != S_SPILL) return false;
            if (b % 8 == 0 && !reg_within(o.spill[b / 8], c.spill[b / 8], ids)) return false;
        }
        if (o.nrefs != c.nrefs) return false;
        for (int i = 0; i < o.nrefs; i++)
            if (!ids.check(o.refs[i], c.refs[i])) return false;
        return true;
    }

    bool equal(const State &o, const State &c, uint16_t livemask) {
        for (int i = 0; i < 11; i++)
            if (((livemask >> i) & 1) && !same(o.r[i], c.r[i])) return false;
        if (memcmp(o.st, c.st, sizeof o.st)) return false;
        for (int s = 0; s < GX_STACK_BYTES / 8; s++)
            if ((o.st[8 * s] & 3) == S_SPILL && !same(o.spill[s], c.spill[s])) return false;
        return o.nrefs == c.nrefs && !memcmp(o.refs, c.refs, sizeof o.refs);
    }

    /* operations that commute with themselves but not with each other must not share bytes */
    enum { OPC_ADD = 1, OPC_OR, OPC_AND, OPC_XOR, OPC_MAX, OPC_MIN };
    int note_update(u32 pc, const Reg &p, int off, int size, int cls) {
        if (!opts.deterministic) return GX_OK;
        s64 lo = p.smin + off, hi = p.smax + off + size;
        for (const OpRange &r : op_ranges[p.map]) {
            if (r.cls != cls && lo < r.hi && r.lo < hi)
                return fail(pc, "map memory updated by two different atomic operations (order-dependent)");
            /* a 32-bit add drops the carry a 64-bit add keeps: mixed, the order decides the result */
            if (cls == OPC_ADD && r.cls == OPC_ADD && r.size != size && lo < r.hi && r.lo < hi)
                return fail(pc, "map memory added to at two widths (order-dependent)");
        }
        op_ranges[p.map].push_back(OpRange{lo, hi, cls, size});
        /* the words this update may change, for merging copies (8-byte updates are 8-aligned) */
        static_assert((int)OPC_ADD == (int)UC_ADD && (int)OPC_MIN == (int)UC_MIN, "one numbering for update classes");
        MapUse &u = out->map_use[p.map];
        /* bitwise operations merge per 4-byte word whatever their width; ADD, MAX and MIN by width */
        const bool wide = size == 8 && (cls == OPC_ADD || cls == OPC_MAX || cls == OPC_MIN);
        const uint8_t code = (uint8_t)(cls | (wide ? UC_W8 : 0));
        const s64 a = std::max<s64>(lo, 0) & ~(s64)(size - 1), b = (hi + size - 1) & ~(s64)(size - 1);
        for (s64 w = a / 4; w < (b + 3) / 4 && w < (s64)u.merge_op.size(); w++) {
            if (u.merge_op[(size_t)w] == UC_NONE) u.merge_op[(size_t)w] = code;
            else if (u.merge_op[(size_t)w] != code) u.merge_mixed = true;
        }
        return GX_OK;
    }

    /* ---------------------------------------------------- map-value use (block-private combining) */
    void use_other(int m) {
        if (m >= 0 && m < (int)out->map_use.size()) out->map_use[m].other = true;
    }

    /* where an update lands: the map and constant value offset, merged over every path */
    void note_vmap(u32 pc, int m, int voff) {
        InsnInfo &ii = out->info[pc];
        int16_t vo = voff >= 0 ? (int16_t)voff : InsnInfo::ARG_VARIES;
        if (ii.vmap == -1) {
            ii.vmap = (int8_t)m;
            ii.voff = vo;
        } else if (ii.vmap != (int8_t)m) {
            ii.vmap = -2;
        } else if (ii.voff != vo) {
            ii.voff = InsnInfo::ARG_VARIES;
        }
    }

    /* a non-fetching commutative update of `size` bytes at p + off (p a map-value pointer) */
    void use_update(u32 pc, const Reg &p, int off, int size, int cls) {
        MapUse &u = out->map_use[p.map];
        if (!is_const(p)) {
            u.other = true;
            note_vmap(pc, p.map, -1);
            return;
        }
        int lo = (int)p.smin + off;
        note_vmap(pc, p.map, lo);
        uint8_t code = (uint8_t)(cls | (size == 8 ? UC_W8 : 0));
        for (int w = lo / 4; w < (lo + size) / 4; w++) {
            if (u.op[w] == UC_NONE) u.op[w] = code;
            else if (u.op[w] != code) u.mixed = true;
        }
    }

    /* ---------------------------------------------------- memory checks */
    int note(u32 pc, uint8_t kind, int off) {
        InsnInfo &ii = out->info[pc];
        if (kind == MK_STACK) ii.stk_any = 1;
        if (ii.kind == MK_NONE) {
            ii.kind = kind;
            ii.off = (int16_t)off;
            return GX_OK;
        }
        if (ii.kind == MK_CTX || kind == MK_CTX) {
            if (ii.kind != kind || ii.off != off) return fail(pc, "the same instruction reaches the ctx and other memory");
            return GX_OK;
        }
        if (ii.kind != kind || ii.off != off) ii.kind = MK_MEM; /* several stack slots / regions: generic access */
        return GX_OK;
    }

    /* a pointer range access [ptr.off + off, +size) inside [0, limit), naturally aligned */
    int check_range(u32 pc, const Reg &p, int off, int size, u64 limit, const char *what) {
        s64 lo = p.smin + off, hi = p.smax + off;
        if (p.smin < -(1 << 29) || p.smax > (1 << 29)) return fail(pc, "%s offset unbounded", what);
        if (lo < 0 || hi + size > (s64)limit) return fail(pc, "%s access out of bounds [%lld, %lld) of %llu", what,
                                                          (long long)lo, (long long)(hi + size), (unsigned long long)limit);
        int need = __builtin_ctz((unsigned)size);
        bool aligned = is_const(p) ? (((lo % size) + size) % size == 0) : (p.tz >= need && (off % size) == 0);
        if (!aligned) return fail(pc, "misaligned %d-byte %s access", size, what);
        return GX_OK;
    }

    int stack_abs(u32 pc, const Reg &p, int off, int size, int &abs) {
        if (!is_const(p)) return fail(pc, "variable stack offset");
        s64 a = p.smin + off;
        if (a < -GX_STACK_BYTES || a + size > 0) return fail(pc, "stack access out of bounds at %lld", (long long)a);
        if (a % size) return fail(pc, "misaligned %d-byte stack access at %lld", size, (long long)a);
        abs = (int)a;
        out->stack_depth = std::max<u32>(out->stack_depth, (u32)(-a));
        return GX_OK;
    }

    /* read `size` stack bytes at abs: fills *res (if non-null) */
    int stack_read(u32 pc, State &s, int abs, int size, Reg *res, bool sign) {
        int b0 = abs + GX_STACK_BYTES;
        bool taint = false, lv = false;
        for (int b = b0; b < b0 + size; b++) {
            if ((s.st[b] & 3) == S_INV) return fail(pc, "read of uninitialised stack at %d", b - GX_STACK_BYTES);
            if ((s.st[b] & 3) == S_SPILL && s.spill[b / 8].t != SC && !(size == 8 && b0 % 8 == 0))
                return fail(pc, "partial read of a spilled pointer");
            if (s.st[b] & ST_TAINT) taint = true;
            if ((s.st[b] & 3) == S_SPILL && s.spill[b / 8].taint) taint = true;
            if (s.st[b] & ST_LV) lv = true;
            if ((s.st[b] & 3) == S_SPILL && varies(s.spill[b / 8])) lv = true;
        }
        if (!res) return GX_OK;
        if (size == 8 && b0 % 8 == 0 && (s.st[b0] & 3) == S_SPILL) {
            *res = s.spill[b0 / 8];
            return GX_OK;
        }
        if (size == 8 || sign) *res = sc_unknown();
        else *res = sc_range(0, (1ULL << (8 * size)) - 1);
        if (sign) {
            s64 lim = (s64)1 << (8 * size - 1);
            res->smin = -lim;
            res->smax = lim - 1;
            sync(*res);
        }
        res->taint = taint;
        res->lv = lv;
        return GX_OK;
    }

    void stack_write(State &s, int abs, int size, const Reg *val, bool taint, bool lv) {
        int b0 = abs + GX_STACK_BYTES;
        if (size == 8 && b0 % 8 == 0 && val) {
            for (int b = b0; b < b0 + 8; b++) s.st[b] = S_SPILL;
            s.spill[b0 / 8] = *val;
            return;
        }
        for (int slot = b0 / 8; slot <= (b0 + size - 1) / 8; slot++) {
            if ((s.st[slot * 8] & 3) == S_SPILL) { /* breaking a spill: its bytes become plain data */
                uint8_t t = (s.spill[slot].taint ? ST_TAINT : 0) | (varies(s.spill[slot]) ? ST_LV : 0);
                for (int b = slot * 8; b < slot * 8 + 8; b++) s.st[b] = S_MISC | t;
            }
        }
        for (int b = b0; b < b0 + size; b++) s.st[b] = S_MISC | (taint ? ST_TAINT : 0) | (lv ? ST_LV : 0);
    }

    /* helper memory argument: readable `size` bytes at p; all_const reports constant spills */
    int mem_arg(u32 pc, State &s, const Reg &p, u64 size, const char *what, bool *tainted, bool *all_const,
                bool *varying = nullptr) {
        if (tainted) *tainted = false;
        if (all_const) *all_const = true;
        if (varying) *varying = p.lv != 0;
        int need = size % 8 == 0 ? 3 : size % 4 == 0 ? 2 : size % 2 == 0 ? 1 : 0;
        if (p.t == STK) {
            if (!is_const(p)) return fail(pc, "%s: variable stack offset", what);
            s64 a = p.smin;
            if (a < -GX_STACK_BYTES || a + (s64)size > 0) return fail(pc, "%s: stack range out of bounds", what);
            if (((-a) & ((1 << need) - 1)) != 0) return fail(pc, "%s: stack pointer misaligned for %llu bytes", what,
                                                             (unsigned long long)size);
            out->stack_depth = std::max<u32>(out->stack_depth, (u32)(-a));
            int b0 = (int)a + GX_STACK_BYTES;
            for (int b = b0; b < b0 + (int)size; b++) {
                int t = s.st[b] & 3;
                if (t == S_INV) return fail(pc, "%s: uninitialised stack byte at %d", what, b - GX_STACK_BYTES);
                if (t == S_SPILL && s.spill[b / 8].t != SC) return fail(pc, "%s: pointer spilled in the argument", what);
                bool tb = (s.st[b] & ST_TAINT) || (t == S_SPILL && s.spill[b / 8].taint);
                if (tb && tainted) *tainted = true;
                bool vb = (s.st[b] & ST_LV) || (t == S_SPILL && varies(s.spill[b / 8]));
                if (vb && varying) *varying = true;
                if (all_const && !(t == S_SPILL && is_const(s.spill[b / 8]) && b0 % 8 == 0 && size % 8 == 0))
                    *all_const = false;
            }
            return GX_OK;
        }
        if (all_const) *all_const = false;
        if (p.t == MV || p.t == RB) {
            u64 lim = p.t == MV ? maps[p.map].value_size : p.size;
            if (check_range(pc, p, 0, 1, lim, what)) return GX_E_VERIFY;
            if (p.smax + (s64)size > (s64)lim) return fail(pc, "%s: range beyond the region", what);
            if (!is_const(p) ? p.tz < need : (p.smin & ((1 << need) - 1)))
                return fail(pc, "%s: pointer misaligned", what);
            if (p.t == MV && opts.deterministic && tainted) *tainted = true;
            if (p.t == MV) use_other(p.map); /* a helper reads these bytes */
            return GX_OK;
        }
        return fail(pc, "%s: expected a stack or map-value pointer, got %s", what, rt_name(p.t));
    }

    void mark_null(State &s, u32 id, bool is_null) {
        auto fix = [&](Reg &r) {
            if ((r.t == MVN || r.t == RBN) && r.id == id) {
                if (is_null) {
                    r = sc_const(0);
                } else {
                    r.t = r.t == MVN ? MV : RB;
                    if (r.t == MV) r.id = 0;
                }
            }
        };
        for (auto &r : s.r) fix(r);
        for (int k = 0; k < GX_STACK_BYTES / 8; k++)
            if ((s.st[8 * k] & 3) == S_SPILL) fix(s.spill[k]);
        if (is_null)
            for (int i = 0; i < s.nrefs; i++)
                if (s.refs[i] == id) {
                    s.refs[i] = s.refs[--s.nrefs];
                    break;
                }
    }

    void release_ref(State &s, u32 id) {
        auto fix = [&](Reg &r) {
            if ((r.t == RB || r.t == RBN) && r.id == id) r = Reg();
        };
        for (auto &r : s.r) fix(r);
        for (int k = 0; k < GX_STACK_BYTES / 8; k++)
            if ((s.st[8 * k] & 3) == S_SPILL && (s.spill[k].t == RB || s.spill[k].t == RBN) && s.spill[k].id == id) {
                s.spill[k] = Reg();
                for (int b = 8 * k; b < 8 * k + 8; b++) s.st[b] = S_INV;
            }
        for (int i = 0; i < s.nrefs; i++)
            if (s.refs[i] == id) {
                s.refs[i] = s.refs[--s.nrefs];
                break;
            }
    }

    /* ---------------------------------------------------- branch refinement */
    /* refine scalars a (and b) assuming `a code b` is `taken`; false = infeasible */
    static bool refine(int code, bool taken, Reg &a, Reg &b) {
        if (!taken) {
            switch (code) {
            case 0x10: code = 0x50; break;
            case 0x50: code = 0x10; break;
            case 0x20: code = 0xB0; break; /* !(a > b) == a <= b */
            case 0x30: code = 0xA0; break;
            case 0xA0: code = 0x30; break;
            case 0xB0: code = 0x20; break;
            case 0x60: code = 0xD0; break;
            case 0x70: code = 0xC0; break;
            case 0xC0: code = 0x70; break;
            case 0xD0: code = 0x60; break;
            case 0x40:
                if (is_const(b)) { /* a & b == 0 */
                    if (is_const(a)) return (a.umin & b.umin) == 0;
                }
                return true;
            }
        } else if (code == 0x40) {
            if (is_const(a) && is_const(b)) return (a.umin & b.umin) != 0;
            return true;
        }
        switch (code) {
        case 0x10: { /* a == b */
            a.umin = b.umin = std::max(a.umin, b.umin);
            a.umax = b.umax = std::min(a.umax, b.umax);
            a.smin = b.smin = std::max(a.smin, b.smin);
            a.smax = b.smax = std::min(a.smax, b.smax);
            uint8_t tz = std::max(a.tz, b.tz);
            a.tz = b.tz = tz;
            break;
        }
        case 0x50: /* a != b */
            if (is_const(b)) {
                if (a.umin == b.umin) a.umin++;
                if (a.umax == b.umin) a.umax--;
                if (a.smin == b.smin) a.smin++;
                if (a.smax == b.smin) a.smax--;
                if (is_const(a) && a.umin == b.umin) return false;
            }
            if (is_const(a)) {
                if (b.umin == a.umin) b.umin++;
                if (b.umax == a.umin) b.umax--;
                if (b.smin == a.smin) b.smin++;
                if (b.smax == a.smin) b.smax--;
            }
            break;
        case 0x20: /* a > b */
            if (b.umin == ~0ULL || a.umax == 0) return false;
            a.umin = std::max(a.umin, b.umin + 1);
            b.umax = std::min(b.umax, a.umax - 1);
            break;
        case 0x30: /* a >= b */
            a.umin = std::max(a.umin, b.umin);
            b.umax = std::min(b.umax, a.umax);
            break;
        case 0xA0: /* a < b */
            if (a.umin == ~0ULL || b.umax == 0) return false;
            a.umax = std::min(a.umax, b.umax - 1);
            b.umin = std::max(b.umin, a.umin + 1);
            break;
        case 0xB0: /* a <= b */
            a.umax = std::min(a.umax, b.umax);
            b.umin = std::max(b.umin, a.umin);
            break;
        case 0x60:
            if (b.smin == INT64_MAX || a.smax == INT64_MIN) return false;
            a.smin = std::max(a.smin, b.smin + 1);
            b.smax = std::min(b.smax, a.smax - 1);
            break;
        case 0x70:
            a.smin = std::max(a.smin, b.smin);
            b.smax = std::min(b.smax, a.smax);
            break;
        case 0xC0:
            if (a.smin == INT64_MAX || b.smax == INT64_MIN) return false;
            a.smax = std::min(a.smax, b.smax - 1);
            b.smin = std::max(b.smin, a.smin + 1);
            break;
        case 0xD0:
            a.smax = std::min(a.smax, b.smax);
            b.smin = std::max(b.smin, a.smin);
            break;
        }
        return sync(a) && sync(b);
    }

    /* ---------------------------------------------------- one instruction */
    enum StepRes { STEP_NEXT, STEP_BRANCH, STEP_DONE, STEP_PRUNE };

    int step(State &s, u32 &pc, State *alt, u32 *alt_pc, int &res) {
        out->info[pc].visited = 1;
        u64 w = insns[pc];
        int op = op_of(w), cls = op & 7, dst = dst_of(w), src = src_of(w), off = off_of(w);
        int32_t imm = imm_of(w);
        bool det = opts.deterministic != 0;
        res = STEP_NEXT;
        auto rd = [&](int r) -> int {
            if (s.r[r].t == NI) return fail(pc, "read of uninitialised R%d", r);
            return GX_OK;
        };
        switch (cls) {
        case 4: case 7: { /* ALU / ALU64 */
            bool w32 = cls == 4, x = op & 8;
            int code = op & 0xF0;
            if (dst == 10) return fail(pc, "R10 is read-only");
            if (code == 0xD0) {
                if (x && !w32) return fail(pc, "invalid byte-swap form");
                if ((imm != 16 && imm != 32 && imm != 64) || src || off) return fail(pc, "invalid byte-swap");
                if (rd(dst) || s.r[dst].t != SC) return fail(pc, "byte swap of a non-scalar");
                Reg &d = s.r[dst];
                uint8_t t = d.taint, lv = d.lv;
                if (is_const(d)) {
                    u64 v = d.umin;
                    v = (w32 && !x) ? (imm == 64 ? v : v & ((1ULL << imm) - 1)) : bswap_n(v, imm);
                    d = sc_const(v);
                } else if (imm < 64) {
                    d = sc_range(0, (1ULL << imm) - 1);
                } else if (!(w32 && !x)) {
                    d = sc_unknown();
                }
                d.taint = t;
                d.lv = lv;
                note_vary(pc, d);
                pc++;
                return GX_OK;
            }
            if (code > 0xD0) return fail(pc, "unknown ALU operation 0x%x", op);
            if (code == 0x80 && (x || src || imm)) return fail(pc, "invalid NEG encoding");
            if (!x && src) return fail(pc, "reserved source field set");
            if (x && imm) return fail(pc, "reserved immediate field set");
            if (code == 0x30 || code == 0x90) {
                if (off != 0 && off != 1) return fail(pc, "invalid division offset");
            } else if (code == 0xB0) {
                if (off && !(x && (off == 8 || off == 16 || (off == 32 && !w32))))
                    return fail(pc, "invalid MOVSX");
            } else if (off) {
                return fail(pc, "reserved offset field set");
            }
            if (!x && (code == 0x60 || code == 0x70 || code == 0xC0) && (imm < 0 || imm >= (w32 ? 32 : 64)))
                return fail(pc, "shift by %d out of range", imm);
            Reg b;
            if (x) {
                if (rd(src)) return GX_E_VERIFY;
                b = s.r[src];
            } else {
                b = sc_const(w32 ? (u64)(uint32_t)imm : (u64)(s64)imm);
            }
            if (code == 0xB0 && off == 0) { /* MOV */
                if (b.t != SC) {
                    if (w32) return fail(pc, "32-bit move of a pointer");
                    s.r[dst] = b;
                } else {
                    s.r[dst] = w32 ? trunc32(b) : b;
                    if (w32) {
                        s.r[dst].smin = (s64)s.r[dst].umin;
                        s.r[dst].smax = (s64)s.r[dst].umax;
                    }
                }
                note_vary(pc, s.r[dst]);
                pc++;
                return GX_OK;
            }
            Reg a;
            if (code == 0xB0) {
                a = sc_const(0);
            } else {
                if (rd(dst)) return GX_E_VERIFY;
                a = s.r[dst];
            }
            if (code == 0x80) b = sc_const(0);
            if (a.t == SC && b.t == SC) {
                s.r[dst] = abs_alu(code, w32, off, a, b);
                note_vary(pc, s.r[dst]);
                pc++;
                return GX_OK;
            }
            /* pointer arithmetic: ptr +/- scalar, scalar + ptr */
            if (w32 || !(code == 0x00 || code == 0x10)) return fail(pc, "arithmetic on a pointer (%s)", rt_name(a.t == SC ? b.t : a.t));
            Reg p = a, k = b;
            if (a.t == SC) {
                if (code == 0x10) return fail(pc, "scalar minus pointer");
                p = b;
                k = a;
            }
            if (k.t != SC) return fail(pc, "pointer combined with a pointer");
            if (p.t == MVN || p.t == RBN) return fail(pc, "arithmetic on a maybe-NULL pointer");
            if (p.t == CMAP) return fail(pc, "arithmetic on a map handle");
            if (det && k.taint) return fail(pc, "order-dependent value used as a pointer offset");
            if ((p.t == CTX || p.t == STK) && !is_const(k)) return fail(pc, "variable offset on a %s pointer", rt_name(p.t));
            if (k.smin < -(1 << 28) || k.smax > (1 << 28)) {
                if (!is_const(k) || (s64)k.umin < -(1 << 28) || (s64)k.umin > (1 << 28))
                    return fail(pc, "pointer offset not bounded");
            }
            Reg sk = k;
            if (code == 0x10) {
                if (is_const(k)) sk = sc_const((u64)(-(s64)k.umin));
                else {
                    sk.smin = -k.smax;
                    sk.smax = -k.smin;
                    sk.umin = 0;
                    sk.umax = ~0ULL;
                    sync(sk);
                }
            }
            Reg np = p;
            s64 lo, hi;
            if (__builtin_add_overflow(p.smin, sk.smin, &lo) || __builtin_add_overflow(p.smax, sk.smax, &hi))
                return fail(pc, "pointer offset overflow");
            np.smin = lo;
            np.smax = hi;
            np.umin = (u64)lo;
            np.umax = (u64)hi;
            if (lo < 0 && hi >= 0) {
                np.umin = 0;
                np.umax = ~0ULL;
            }
            np.tz = std::min(p.tz, sk.tz);
            if (lo == hi) np.tz = (uint8_t)ctz64((u64)lo);
            np.lv = (p.t == MV || p.t == RB) ? (uint8_t)(p.lv || varies(k)) : 0; /* ctx / stack offsets are constants */
            s.r[dst] = np;
            pc++;
            return GX_OK;
        }
        case 5: case 6: { /* JMP / JMP32 */
            int code = op & 0xF0;
            bool w32 = cls == 6;
            if (code == 0x00) {
                if (cls == 5 && (imm || src || dst)) return fail(pc, "reserved fields in JA");
                if (cls == 6 && (off || src || dst)) return fail(pc, "reserved fields in JA");
                pc = (u32)((s64)pc + 1 + (cls == 6 ? imm : off));
                return GX_OK;
            }
            if (code == 0x80 && cls == 5) return call(s, pc, imm, src, res);
            if (code == 0x90 && cls == 5) {
                if (rd(0)) return GX_E_VERIFY;
                if (s.r[0].t != SC) return fail(pc, "R0 at exit is a %s, not a scalar", rt_name(s.r[0].t));
                if (det && s.r[0].taint) return fail(pc, "order-dependent value returned in R0");
                if (sm && varies(s.r[0])) return sfail(pc, GX_SIMT_V_RET, "lane-varying value returned in R0");
                if (s.nrefs) return fail(pc, "ring-buffer reservation neither submitted nor discarded");
                res = STEP_DONE;
                return GX_OK;
            }
            if (code == 0x80 || code == 0x90 || code > 0xD0) return fail(pc, "invalid jump 0x%x", op);
            bool x = op & 8;
            if (!x && src) return fail(pc, "reserved source field set");
            if (dst == 10 || (x && src == 10)) return fail(pc, "comparison involving the frame pointer R10");
            if (rd(dst)) return GX_E_VERIFY;
            if (x && rd(src)) return GX_E_VERIFY;
            Reg a = s.r[dst];
            Reg b = x ? s.r[src] : sc_const(w32 ? (u64)(uint32_t)imm : (u64)(s64)imm);
            u32 tgt = (u32)((s64)pc + 1 + off), fall = pc + 1;
            if (a.t != SC || b.t != SC) {
                /* only NULL checks of maybe-NULL pointers, or of pointers known non-NULL */
                bool a_ptr = a.t != SC;
                Reg &p = a_ptr ? a : b;
                Reg &z = a_ptr ? b : a;
                if (w32 || (code != 0x10 && code != 0x50) || z.t != SC || !is_const(z) || z.umin != 0)
                    return fail(pc, "pointer comparison other than a NULL check");
                if (sm && p.lv) return sfail(pc, GX_SIMT_V_BRANCH, "NULL check of a lane-varying pointer");
                if (p.t == MVN || p.t == RBN) {
                    if (sm) simt_branch[pc] = 1;
                    u32 id = p.id;
                    *alt = s;
                    /* taken branch: JEQ -> NULL, JNE -> non-NULL */
                    mark_null(*alt, id, code == 0x10);
                    mark_null(s, id, code != 0x10);
                    *alt_pc = tgt;
                    pc = fall;
                    res = STEP_BRANCH;
                    return GX_OK;
                }
                /* non-NULL pointer: the outcome is fixed */
                pc = code == 0x50 ? tgt : fall;
                return GX_OK;
            }
            if (det && (a.taint || b.taint)) return fail(pc, "branch on an order-dependent value");
            if (is_const(a) && is_const(b)) {
                pc = eval_cond(code, w32, a.umin, b.umin) ? tgt : fall;
                return GX_OK;
            }
            if (sm) {
                if (varies(a) || varies(b)) return sfail(pc, GX_SIMT_V_BRANCH, "branch on a lane-varying value");
                simt_branch[pc] = 1;
            }
            bool can_refine = !w32 || (a.umax <= 0x7FFFFFFFULL && b.umax <= 0x7FFFFFFFULL);
            State st_taken = s;
            bool ok_taken = true, ok_fall = true;
            if (can_refine) {
                Reg ta = a, tb = b, fa = a, fb = b;
                ok_taken = refine(code, true, ta, tb);
                ok_fall = refine(code, false, fa, fb);
                st_taken.r[dst] = ta;
                if (x) st_taken.r[src] = tb;
                s.r[dst] = fa;
                if (x) s.r[src] = fb;
            }
            if (ok_taken && ok_fall) {
                *alt = st_taken;
                *alt_pc = tgt;
                pc = fall;
                res = STEP_BRANCH;
            } else if (ok_taken) {
                s = st_taken;
                pc = tgt;
            } else if (ok_fall) {
                pc = fall;
            } else {
                res = STEP_PRUNE; /* no feasible successor */
            }
            return GX_OK;
        }
        case 0: { /* LD: 64-bit immediate only */
            if (op != 0x18) return fail(pc, "unsupported load class opcode 0x%x (legacy packet access)", op);
            if (dst == 10) return fail(pc, "R10 is read-only");
            if (off) return fail(pc, "reserved offset field set");
            if (src == 0) {
                u64 v = (u64)(uint32_t)imm | ((insns[pc + 1] >> 32) << 32);
                s.r[dst] = sc_const(v);
            } else if (src == 1) {
                if ((u32)imm >= n_maps) return fail(pc, "map index %d out of range", imm);
                Reg r;
                r.t = CMAP;
                r.map = (uint8_t)imm;
                s.r[dst] = r;
            } else {
                return fail(pc, "unsupported 64-bit immediate source %d", src);
            }
            pc += 2;
            return GX_OK;
        }
        case 1: { /* LDX */
            int mode = op & 0xE0, size = size_of(op);
            if (mode != 0x60 && mode != 0x80) return fail(pc, "unsupported load mode");
            if (mode == 0x80 && size == 8) return fail(pc, "sign-extending 8-byte load");
            if (dst == 10) return fail(pc, "R10 is read-only");
            if (imm) return fail(pc, "reserved immediate field set");
            if (rd(src)) return GX_E_VERIFY;
            const Reg p = s.r[src];
            bool sign = mode == 0x80;
            Reg v = (size == 8 || sign) ? sc_unknown() : sc_range(0, (1ULL << (8 * size)) - 1);
            if (sign) {
                s64 lim = (s64)1 << (8 * size - 1);
                v.smin = -lim;
                v.smax = lim - 1;
                v.umin = 0;
                v.umax = ~0ULL;
                sync(v);
            }
            switch (p.t) {
            case CTX: {
                if (!is_const(p)) return fail(pc, "variable ctx offset");
                s64 a = p.smin + off;
                if (a < 0 || a + size > (s64)opts.ctx_size) return fail(pc, "ctx read out of bounds at %lld", (long long)a);
                if (a % size) return fail(pc, "misaligned ctx read");
                if (note(pc, MK_CTX, (int)a)) return GX_E_VERIFY;
                v.lv = ctx_varies(a, size);
                break;
            }
            case STK: {
                int abs = 0;
                if (stack_abs(pc, p, off, size, abs)) return GX_E_VERIFY;
                if (stack_read(pc, s, abs, size, &v, sign)) return GX_E_VERIFY;
                if (note(pc, MK_STACK, abs)) return GX_E_VERIFY;
                break;
            }
            case MV:
                if (check_range(pc, p, off, size, maps[p.map].value_size, "map value")) return GX_E_VERIFY;
                v.taint = det ? 1 : 0;
                v.lv = p.lv; /* one address in every lane reads one value */
                use_other(p.map);
                if (note(pc, MK_MEM, 0)) return GX_E_VERIFY;
                break;
            case RB:
                if (check_range(pc, p, off, size, p.size, "ring-buffer record")) return GX_E_VERIFY;
                v.lv = p.lv;
                if (note(pc, MK_MEM, 0)) return GX_E_VERIFY;
                break;
            default: return fail(pc, "load through a %s", rt_name(p.t));
            }
            s.r[dst] = v;
            s.c_mem++;
            note_vary(pc, v);
            pc++;
            return GX_OK;
        }
        case 2: case 3: { /* ST / STX */
            int mode = op & 0xE0, size = size_of(op);
            if (rd(dst)) return GX_E_VERIFY;
            const Reg p = s.r[dst];
            s.c_mem++;
            if (mode == 0xC0) return atomic(s, pc, size, p, off, imm, src, cls);
            if (mode != 0x60) return fail(pc, "unsupported store mode");
            Reg v;
            if (cls == 3) {
                if (imm) return fail(pc, "reserved immediate field set");
                if (rd(src)) return GX_E_VERIFY;
                v = s.r[src];
            } else {
                if (src) return fail(pc, "reserved source field set");
                v = sc_const((u64)(s64)imm);
                if (size < 8) v = sc_const(((u64)(s64)imm) & ((size == 4) ? 0xFFFFFFFFULL : (1ULL << (8 * size)) - 1));
            }
            if (v.t != SC && !(p.t == STK && size == 8)) return fail(pc, "pointer stored outside a full stack slot");
            switch (p.t) {
            case STK: {
                int abs = 0;
                if (stack_abs(pc, p, off, size, abs)) return GX_E_VERIFY;
                if (v.t != SC && (abs + GX_STACK_BYTES) % 8) return fail(pc, "misaligned pointer spill");
                stack_write(s, abs, size, size == 8 ? &v : nullptr, v.taint, varies(v));
                if (note(pc, MK_STACK, abs)) return GX_E_VERIFY;
                break;
            }
            case MV:
                if (check_range(pc, p, off, size, maps[p.map].value_size, "map value")) return GX_E_VERIFY;
                if (det) return fail(pc, "plain store into map memory in deterministic mode");
                if (sm && (p.lv || varies(v)))
                    return sfail(pc, GX_SIMT_V_STORE, "lane-varying %s stored into map memory", p.lv ? "address" : "value");
                use_other(p.map);
                if (note(pc, MK_MEM, 0)) return GX_E_VERIFY;
                break;
            case RB:
                if (check_range(pc, p, off, size, p.size, "ring-buffer record")) return GX_E_VERIFY;
                if (det && v.taint) return fail(pc, "order-dependent value written to the ring buffer");
                if (sm && (p.lv || varies(v)))
                    return sfail(pc, GX_SIMT_V_STORE, "lane-varying %s stored into a ring-buffer record",
                                 p.lv ? "address" : "value");
                if (note(pc, MK_MEM, 0)) return GX_E_VERIFY;
                break;
            case CTX: return fail(pc, "the ctx is read-only");
            default: return fail(pc, "store through a %s", rt_name(p.t));
            }
            pc++;
            return GX_OK;
        }
        }
        return fail(pc, "unknown instruction class");
    }

    int atomic(State &s, u32 &pc, int size, const Reg &p, int off, int32_t imm, int src, int cls) {
        bool det = opts.deterministic != 0;
        if (cls != 3) return fail(pc, "atomic in the ST class");
        if (size != 4 && size != 8) return fail(pc, "atomic of size %d", size);
        int base = imm & ~1;
        bool fetch = imm & 1;
        bool xchg = imm == 0xE1, cmpx = imm == 0xF1;
        if (!(xchg || cmpx || ((base == 0x00 || base == 0x40 || base == 0x50 || base == 0xA0) && imm <= 0xA1)))
            return fail(pc, "unknown atomic operation 0x%x", imm);
        if (s.r[src].t == NI) return fail(pc, "read of uninitialised R%d", src);
        if (s.r[src].t != SC) return fail(pc, "atomic operand is a pointer");
        if (cmpx && (s.r[0].t != SC)) return fail(pc, "CMPXCHG needs a scalar R0");
        Reg old = sc_unknown();
        if (size == 4) old = sc_range(0, 0xFFFFFFFFULL);
        if (p.t == MV) {
            if (check_range(pc, p, off, size, maps[p.map].value_size, "map value")) return GX_E_VERIFY;
            if (det && (xchg || cmpx)) return fail(pc, "exchange on map memory in deterministic mode");
            if (det && s.r[src].taint) return fail(pc, "order-dependent value added into map memory");
            if (sm && (p.lv || varies(s.r[src]) || (cmpx && varies(s.r[0]))))
                return sfail(pc, GX_SIMT_V_ATOMIC, "non-uniform atomic on map memory (lane-varying %s)",
                             p.lv ? "address" : "operand");
            old.taint = det ? 1 : 0;
            if (!xchg && !cmpx) {
                int cls = base == 0x00 ? OPC_ADD : base == 0x40 ? OPC_OR : base == 0x50 ? OPC_AND : OPC_XOR;
                if (note_update(pc, p, off, size, cls)) return GX_E_VERIFY;
            }
            if (xchg || cmpx || fetch) {
                use_other(p.map);
                note_vmap(pc, -2, -1);
            } else {
                int uc = base == 0x00 ? UC_ADD : base == 0x40 ? UC_OR : base == 0x50 ? UC_AND : UC_XOR;
                use_update(pc, p, off, size, uc);
            }
            if (note(pc, MK_MEM, 0)) return GX_E_VERIFY;
        } else if (p.t == STK) {
            int abs = 0;
            if (stack_abs(pc, p, off, size, abs)) return GX_E_VERIFY;
            Reg cur;
            if (stack_read(pc, s, abs, size, &cur, false)) return GX_E_VERIFY;
            old.taint = cur.taint;
            old.lv = cur.lv;
            bool t = cur.taint || s.r[src].taint || (cmpx && s.r[0].taint);
            bool lv = varies(cur) || varies(s.r[src]) || (cmpx && varies(s.r[0]));
            stack_write(s, abs, size, nullptr, t, lv);
            note_vmap(pc, -2, -1);
            if (note(pc, MK_STACK, abs)) return GX_E_VERIFY;
        } else {
            return fail(pc, "atomic on a %s", rt_name(p.t));
        }
        if (cmpx) s.r[0] = old;
        else if (fetch || xchg) s.r[src] = old;
        pc++;
        return GX_OK;
    }

    int call(State &s, u32 &pc, int32_t id, int src, int &res) {
        bool det = opts.deterministic != 0;
        (void)res;
        if (src) return fail(pc, "only helper calls are supported (src_reg %d)", src);
        int nargs = helper_args(id);
        if (nargs < 0) return fail(pc, "unknown helper %d", id);
        for (int i = 1; i <= nargs; i++)
            if (s.r[i].t == NI) return fail(pc, "helper %d: argument R%d uninitialised", id, i);
        auto need_map = [&](int kind_ok) -> int {
            if (s.r[1].t != CMAP) return fail(pc, "helper %d: R1 must be a map", id);
            InsnInfo &ii = out->info[pc];
            if (ii.map == -1) ii.map = (int8_t)s.r[1].map;
            else if (ii.map != (int8_t)s.r[1].map) ii.map = -2;
            auto note_arg = [&](int16_t &slot, const Reg &r) {
                int16_t v = (r.t == STK && is_const(r)) ? (int16_t)r.smin : InsnInfo::ARG_VARIES;
                if (slot == InsnInfo::ARG_UNSET) slot = v;
                else if (slot != v) slot = InsnInfo::ARG_VARIES;
            };
            note_arg(ii.a2, s.r[2]);
            note_arg(ii.a3, s.r[3]);
            u32 t = maps[s.r[1].map].type;
            if (kind_ok == 1 && t == GX_MAP_RINGBUF) return fail(pc, "helper %d: ring buffer given", id);
            if (kind_ok == 2 && t != GX_MAP_RINGBUF) return fail(pc, "helper %d: ring buffer expected", id);
            return GX_OK;
        };
        Reg r0 = sc_unknown();
        bool r0_void = false;
        s.c_help++;
        switch (id) {
        case GX_HELPER_MAP_LOOKUP: {
            if (need_map(1)) return GX_E_VERIFY;
            const gx_map_spec &m = maps[s.r[1].map];
            bool t, vk;
            if (mem_arg(pc, s, s.r[2], m.key_size, "lookup key", &t, nullptr, &vk)) return GX_E_VERIFY;
            if (det && t) return fail(pc, "order-dependent map key");
            if (sm && vk) return sfail(pc, GX_SIMT_V_KEY, "lane-varying lookup key");
            r0 = Reg();
            r0.t = MVN;
            r0.map = s.r[1].map;
            r0.id = next_id++;
            r0.umin = r0.umax = 0;
            r0.smin = r0.smax = 0;
            r0.tz = 64;
            break;
        }
        case GX_HELPER_MAP_UPDATE: {
            if (need_map(1)) return GX_E_VERIFY;
            const gx_map_spec &m = maps[s.r[1].map];
            bool tk, tv, kc, vc, vk, vv;
            if (mem_arg(pc, s, s.r[2], m.key_size, "update key", &tk, &kc, &vk)) return GX_E_VERIFY;
            if (mem_arg(pc, s, s.r[3], m.value_size, "update value", &tv, &vc, &vv)) return GX_E_VERIFY;
            if (s.r[4].t != SC) return fail(pc, "update flags must be a scalar");
            if (sm && vk) return sfail(pc, GX_SIMT_V_KEY, "lane-varying update key");
            if (sm && vv) return sfail(pc, GX_SIMT_V_HELPER, "lane-varying value for a map update");
            if (sm && varies(s.r[4])) return sfail(pc, GX_SIMT_V_HELPER, "lane-varying update flags");
            if (!is_const(s.r[4]) || s.r[4].umin != GX_NOEXIST) use_other(s.r[1].map); /* may overwrite a value */
            if (det) {
                if (tk) return fail(pc, "order-dependent map key");
                if (!is_const(s.r[4]) || s.r[4].umin != GX_NOEXIST)
                    return fail(pc, "deterministic mode allows only NOEXIST inserts");
                if (!vc) return fail(pc, "deterministic mode: inserted value must be constant bytes");
                /* the constant bytes (whole constant spills) this insert writes, for merging copies */
                MapUse &u = out->map_use[s.r[1].map];
                std::vector<uint8_t> bytes(m.value_size);
                const int b0 = (int)s.r[3].smin + GX_STACK_BYTES;
                for (u32 k = 0; k < m.value_size; k++)
                    bytes[k] = (uint8_t)(s.spill[(b0 + (int)k) / 8].umin >> (8 * ((b0 + (int)k) % 8)));
                if (!u.insert_seen) {
                    u.insert = bytes;
                    u.insert_seen = true;
                } else if (u.insert != bytes) { /* two events inserting one key: the first one's bytes stay */
                    u.insert_conflict = true;
                    return fail(pc, "inserts of different constants into one map (order-dependent)");
                }
            }
            r0 = sc_unknown();
            r0.taint = det ? 1 : 0;
            break;
        }
        case GX_HELPER_MAP_DELETE: {
            if (need_map(1)) return GX_E_VERIFY;
            if (det) return fail(pc, "map delete in deterministic mode");
            if (maps[s.r[1].map].flags & GX_MAP_F_NO_DELETE) return fail(pc, "map delete on a map created without deletes");
            bool t, vk;
            if (mem_arg(pc, s, s.r[2], maps[s.r[1].map].key_size, "delete key", &t, nullptr, &vk)) return GX_E_VERIFY;
            if (sm && vk) return sfail(pc, GX_SIMT_V_KEY, "lane-varying delete key");
            r0 = sc_unknown();
            break;
        }
        case GX_HELPER_RINGBUF_OUTPUT: {
            if (need_map(2)) return GX_E_VERIFY;
            if (s.r[3].t != SC || !is_const(s.r[3]) || s.r[3].umin == 0 || s.r[3].umin > GX_MAX_VALUE)
                return fail(pc, "ringbuf_output size must be a constant in [1, %d]", GX_MAX_VALUE);
            bool t, vd;
            if (mem_arg(pc, s, s.r[2], s.r[3].umin, "ringbuf_output data", &t, nullptr, &vd)) return GX_E_VERIFY;
            if (det && t) return fail(pc, "order-dependent ring-buffer payload");
            if (sm && vd) return sfail(pc, GX_SIMT_V_HELPER, "lane-varying ring-buffer payload");
            if (s.r[4].t != SC || !is_const(s.r[4]) || (s.r[4].umin & ~3ULL)) return fail(pc, "bad ringbuf_output flags");
            r0 = sc_unknown();
            r0.taint = det ? 1 : 0;
            break;
        }
        case GX_HELPER_RINGBUF_RESERVE: {
            if (need_map(2)) return GX_E_VERIFY;
            if (s.r[2].t != SC || !is_const(s.r[2]) || s.r[2].umin == 0 || s.r[2].umin > GX_MAX_VALUE ||
                s.r[2].umin + GX_RB_HDR > maps[s.r[1].map].max_entries)
                return fail(pc, "ringbuf_reserve size must be a constant in [1, %d]", GX_MAX_VALUE);
            if (s.r[3].t != SC || !is_const(s.r[3]) || s.r[3].umin != 0) return fail(pc, "ringbuf_reserve flags must be 0");
            if (s.nrefs >= 8) return fail(pc, "too many outstanding ring-buffer reservations");
            r0 = Reg();
            r0.t = RBN;
            r0.map = s.r[1].map;
            r0.id = next_id++;
            r0.size = (u32)s.r[2].umin;
            r0.umin = r0.umax = 0;
            r0.smin = r0.smax = 0;
            r0.tz = 64;
            s.refs[s.nrefs++] = r0.id;
            break;
        }
        case GX_HELPER_RINGBUF_SUBMIT:
        case GX_HELPER_RINGBUF_DISCARD: {
            const Reg &p = s.r[1];
            if (p.t != RB || !is_const(p) || p.umin != 0) return fail(pc, "submit/discard needs an unmodified non-NULL reservation");
            if (s.r[2].t != SC) return fail(pc, "submit/discard flags must be a scalar");
            if (sm && (p.lv || varies(s.r[2]))) return sfail(pc, GX_SIMT_V_HELPER, "lane-varying submit/discard argument");
            release_ref(s, p.id);
            r0_void = true;
            break;
        }
        case GX_HELPER_ATOMIC_MAX_U64:
        case GX_HELPER_ATOMIC_MIN_U64: {
            const Reg &p = s.r[1];
            if (p.t != MV) return fail(pc, "atomic max/min needs a non-NULL map-value pointer");
            if (check_range(pc, p, 0, 8, maps[p.map].value_size, "map value")) return GX_E_VERIFY;
            if (s.r[2].t != SC) return fail(pc, "atomic max/min operand must be a scalar");
            if (det && s.r[2].taint) return fail(pc, "order-dependent value folded into map memory");
            if (sm && (p.lv || varies(s.r[2])))
                return sfail(pc, GX_SIMT_V_ATOMIC, "non-uniform atomic max/min (lane-varying %s)", p.lv ? "address" : "operand");
            if (note_update(pc, p, 0, 8, id == GX_HELPER_ATOMIC_MAX_U64 ? OPC_MAX : OPC_MIN)) return GX_E_VERIFY;
            use_update(pc, p, 0, 8, id == GX_HELPER_ATOMIC_MAX_U64 ? UC_MAX : UC_MIN);
            r0_void = true;
            if (note(pc, MK_MEM, 0)) return GX_E_VERIFY;
            break;
        }
        case GX_HELPER_WARP_SUM_U64:
        case GX_HELPER_WARP_MAX_U64:
        case GX_HELPER_WARP_MIN_U64:
        case GX_HELPER_WARP_OR_U64:
        case GX_HELPER_WARP_AND_U64:
        case GX_HELPER_WARP_COUNT: /* SIMT mode only (helper_args): a reduction over the lanes, uniform */
            if (s.r[1].t != SC) return fail(pc, "warp helper operand must be a scalar");
            r0 = id == GX_HELPER_WARP_COUNT ? sc_range(0, 32) : sc_unknown();
            break;
        }
        for (int i = 1; i <= 5; i++) s.r[i] = Reg();
        s.r[0] = r0_void ? Reg() : r0;
        pc++;
        return GX_OK;
    }

    /* ---------------------------------------------------- driver */
    int run() {
        out->info.assign(n, InsnInfo());
        out->map_use.assign(n_maps, MapUse());
        for (u32 m = 0; m < n_maps && m < GX_MAX_MAPS; m++) {
            out->map_use[m].op.assign((maps[m].value_size + 3) / 4, UC_NONE);
            out->map_use[m].merge_op.assign((maps[m].value_size + 3) / 4, UC_NONE);
        }
        if (n == 0 || n > GX_MAX_INSNS) return fail(0, "program length %u not in [1, %d]", n, GX_MAX_INSNS);
        if (opts.ctx_size < 8 || opts.ctx_size > GX_MAX_CTX || opts.ctx_size % 8)
            return fail(0, "ctx_size %u invalid", opts.ctx_size);
        if (n_maps > GX_MAX_MAPS) return fail(0, "too many maps");
        if (structure()) return GX_E_VERIFY;
        visited.assign(n, {});
        if (sm) {
            if (simt->uniform.size() != opts.ctx_size) return fail(0, "uniform flags must cover the %u ctx bytes", opts.ctx_size);
            simt_branch.assign(n, 0);
            simt_vary.assign(n, 0);
        }
        std::vector<Pending> stack;
        {
            Pending p;
            p.pc = 0;
            p.parent = -1;
            p.st.r[1].t = CTX;
            p.st.r[1].tz = 64;
            p.st.r[10].t = STK;
            p.st.r[10].tz = 64;
            stack.push_back(p);
        }
        std::vector<int> anc;
        State alt;
        while (!stack.empty()) {
            Pending cur = stack.back();
            stack.pop_back();
            for (;;) {
                if (++out->insns_processed > GX_VERIFY_BUDGET)
                    return fail(cur.pc, "program too complex: more than %llu instructions explored",
                                (unsigned long long)GX_VERIFY_BUDGET);
                if (cur.pc >= n) return fail(cur.pc, "execution falls off the end of the program");
                if (second[cur.pc]) return fail(cur.pc, "execution reaches the second slot of a 64-bit immediate");
                if (prune[cur.pc]) {
                    anc.clear();
                    for (int a = cur.parent; a >= 0; a = nodes[a].parent) anc.push_back(a);
                    bool pruned = false;
                    for (int idx : visited[cur.pc]) {
                        if (!within(nodes[idx].st, cur.st, live[cur.pc])) continue;
                        bool is_anc = std::find(anc.begin(), anc.end(), idx) != anc.end();
                        if (is_anc) {
                            if (equal(nodes[idx].st, cur.st, live[cur.pc]))
                                return fail(cur.pc, "infinite loop: a state repeats exactly");
                            continue;
                        }
                        const State &k = nodes[idx].st; /* its paths were counted from its own counts */
                        if (sm && (cur.st.c_insn > k.c_insn || cur.st.c_help > k.c_help || cur.st.c_mem > k.c_mem))
                            continue;
                        pruned = true;
                        break;
                    }
                    if (pruned) break;
                    if ((int)visited[cur.pc].size() < MAX_STATES_PER_PC && nodes.size() < MAX_STATES_TOTAL) {
                        nodes.push_back(Node{cur.st, cur.parent});
                        visited[cur.pc].push_back((int)nodes.size() - 1);
                        cur.parent = (int)nodes.size() - 1;
                        out->states_stored++;
                    }
                }
                int res;
                u32 alt_pc = 0, at = cur.pc;
                if (sm && simt->max_insns && ++cur.st.c_insn > simt->max_insns)
                    return sfail(at, GX_SIMT_V_INSNS, "a path exceeds the hook budget of %u instructions", simt->max_insns);
                if (sm && !simt->max_insns) ++cur.st.c_insn;
                if (step(cur.st, cur.pc, &alt, &alt_pc, res)) return GX_E_VERIFY;
                if (sm) {
                    if (simt->max_helpers && cur.st.c_help > simt->max_helpers)
                        return sfail(at, GX_SIMT_V_HELPERS, "a path exceeds the hook budget of %u helper calls",
                                     simt->max_helpers);
                    if (simt->max_mem && cur.st.c_mem > simt->max_mem)
                        return sfail(at, GX_SIMT_V_MEM, "a path exceeds the hook budget of %u memory operations",
                                     simt->max_mem);
                    if (res == STEP_DONE) {
                        SimtOut &o = out->simt;
                        o.max_insns = std::max<u64>(o.max_insns, cur.st.c_insn);
                        o.max_helpers = std::max(o.max_helpers, cur.st.c_help);
                        o.max_mem = std::max(o.max_mem, cur.st.c_mem);
                    }
                }
                if (res == STEP_DONE || res == STEP_PRUNE) break;
                if (res == STEP_BRANCH) {
                    Pending p;
                    p.st = alt;
                    p.pc = alt_pc;
                    p.parent = cur.parent;
                    stack.push_back(p);
                }
            }
        }
        if (sm) {
            for (u32 i = 0; i < n; i++) {
                out->simt.uniform_branches += simt_branch[i];
                out->simt.varying_insns += simt_vary[i];
            }
        }
        return GX_OK;
    }
};

} // namespace

int verify_program(const uint64_t *insns, uint32_t n, const gx_map_spec *maps, uint32_t n_maps, const gx_prog_opts &opts,
                   VerifyOut &out, const SimtIn *simt) {
    if (!insns || (n_maps && !maps)) return GX_EINVAL;
    for (uint32_t i = 0; i < n_maps; i++) {
        const gx_map_spec &m = maps[i];
        bool ok = false;
        if (m.type == GX_MAP_ARRAY) ok = m.key_size == 4 && m.value_size >= 1 && m.value_size <= GX_MAX_VALUE && m.max_entries >= 1;
        if (m.type == GX_MAP_HASH)
            ok = m.key_size >= 1 && m.key_size <= GX_MAX_KEY && m.value_size >= 1 && m.value_size <= GX_MAX_VALUE &&
                 m.max_entries >= 1 && m.max_entries <= (1u << 30);
        if (m.type == GX_MAP_RINGBUF) ok = m.max_entries >= 4096 && (m.max_entries & (m.max_entries - 1)) == 0;
        if ((m.flags & ~GX_MAP_F_NO_DELETE) || (m.flags && m.type != GX_MAP_HASH) || m.reserved) ok = false;
        if (!ok) {
            out.log = "invalid map spec at index " + std::to_string(i);
            return GX_EINVAL;
        }
    }
    Verifier v;
    v.insns = insns;
    v.n = n;
    v.maps = maps;
    v.n_maps = n_maps;
    v.opts = opts;
    v.out = &out;
    v.simt = simt;
    v.sm = simt != nullptr;
    return v.run();
}

} // namespace gx
