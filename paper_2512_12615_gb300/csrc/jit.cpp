/*
 * Load-time specialisation of verified programs (the paper's eBPF -> device-code JIT
 * with helper inlining, Sec. 4.4.2 and Sec. 5.3).
 *
 * Each verified program becomes one straight-line CUDA C++ function: eBPF registers are
 * local variables, every instruction is one C statement, jumps are gotos, ctx and stack
 * accesses use the offsets the verifier proved, helper calls name their map directly.
 * The function is wrapped into the same launch skeleton as the interpreter
 * (gx_device.cuh: exec_tiles), compiled by NVRTC for sm_103a and loaded with the CUDA
 * runtime's library API.  A kernel may hold several programs (a batch): it switches on
 * the chunk's program slot.  NVRTC is loaded with dlopen, so the engine library keeps
 * loading on hosts without the compiler or a GPU; compiled cubins are cached in memory
 * and, if GX_JIT_CACHE names a directory, on disk.  The disk cache is bounded: after each
 * write, the oldest cubins are removed until the directory holds at most GX_JIT_CACHE_MB
 * megabytes (default 1024).  If GX_JIT_DUMP_DIR names a directory, every generated source
 * is also written there as <key>.cu, for reading.
 */
#include <cuda_runtime.h>
#include <dirent.h>
#include <dlfcn.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "gx_jit.h"
#include "gx_runtime.h"

extern "C" const char gx_embed_gx_h[];
extern "C" const char gx_embed_gx_layout_h[];
extern "C" const char gx_embed_gx_device_cuh[];
extern "C" const char gx_embed_gx_steal_cuh[];

namespace gx {
namespace {

/* ---------------------------------------------------------------- NVRTC entry points */
typedef int nvrtcResult_;
typedef void *nvrtcProgram_;
struct Nvrtc {
    bool ok = false;
    std::string err;
    nvrtcResult_ (*create)(nvrtcProgram_ *, const char *, const char *, int, const char *const *,
                           const char *const *) = nullptr;
    nvrtcResult_ (*compile)(nvrtcProgram_, int, const char *const *) = nullptr;
    nvrtcResult_ (*log_size)(nvrtcProgram_, size_t *) = nullptr;
    nvrtcResult_ (*log)(nvrtcProgram_, char *) = nullptr;
    nvrtcResult_ (*cubin_size)(nvrtcProgram_, size_t *) = nullptr;
    nvrtcResult_ (*cubin)(nvrtcProgram_, char *) = nullptr;
    nvrtcResult_ (*destroy)(nvrtcProgram_ *) = nullptr;
};

Nvrtc &nvrtc() {
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                               "/usr/local/cuda/lib64/libnvrtc.so"};
        void *h = nullptr;
        for (const char *nm : names)
            if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) {
            n.err = "NVRTC library not found";
            return;
        }
        n.create = (decltype(n.create))dlsym(h, "nvrtcCreateProgram");
        n.compile = (decltype(n.compile))dlsym(h, "nvrtcCompileProgram");
        n.log_size = (decltype(n.log_size))dlsym(h, "nvrtcGetProgramLogSize");
        n.log = (decltype(n.log))dlsym(h, "nvrtcGetProgramLog");
        n.cubin_size = (decltype(n.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
        n.cubin = (decltype(n.cubin))dlsym(h, "nvrtcGetCUBIN");
        n.destroy = (decltype(n.destroy))dlsym(h, "nvrtcDestroyProgram");
        n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy;
        if (!n.ok) n.err = "NVRTC symbols missing";
    });
    return n;
}

/* ---------------------------------------------------------------- code generation */
std::string hex64(uint64_t v) {
    char b[32];
    snprintf(b, sizeof b, "0x%llxull", (unsigned long long)v);
    return b;
}

const char *alu_op(int code, int off) {
    switch (code) {
    case 0x00: return "O_ADD";
    case 0x10: return "O_SUB";
    case 0x20: return "O_MUL";
    case 0x30: return off ? "O_SDIV" : "O_DIV";
    case 0x40: return "O_OR";
    case 0x50: return "O_AND";
    case 0x60: return "O_LSH";
    case 0x70: return "O_RSH";
    case 0x90: return off ? "O_SMOD" : "O_MOD";
    case 0xA0: return "O_XOR";
    case 0xB0: return "O_MOV";
    case 0xC0: return "O_ARSH";
    }
    return nullptr;
}

const char *cond_op(int code) {
    switch (code) {
    case 0x10: return "C_EQ";
    case 0x20: return "C_GT";
    case 0x30: return "C_GE";
    case 0x40: return "C_SET";
    case 0x50: return "C_NE";
    case 0x60: return "C_SGT";
    case 0x70: return "C_SGE";
    case 0xA0: return "C_LT";
    case 0xB0: return "C_LE";
    case 0xC0: return "C_SLT";
    case 0xD0: return "C_SLE";
    }
    return nullptr;
}

int size_of(int op) { return (op & 0x18) == 0x00 ? 4 : (op & 0x18) == 0x08 ? 2 : (op & 0x18) == 0x10 ? 1 : 8; }

std::string R(int r) { return "r" + std::to_string(r); }

const uint32_t WC_FULL_MAX = 8192;  /* array maps up to this many bytes get a whole private copy */
const uint32_t WC_CACHE_MAX = 24576; /* shared bytes of one map's cache (tags + accumulators) */
const uint32_t WC_TOTAL_MAX = 32768; /* shared bytes of one program's combining area */
const uint32_t WC_BITS = 10;        /* widest cache: 1024 entries */

uint32_t up16(uint32_t v) { return (v + 15u) & ~15u; }

const char *uc_op(uint8_t c) {
    switch (c & 0xF) {
    case UC_ADD: return "AG_ADD";
    case UC_OR: return "AG_OR";
    case UC_AND: return "AG_AND";
    case UC_XOR: return "AG_XOR";
    case UC_MAX: return "AG_MAX";
    default: return "AG_MIN";
    }
}

/* bit j: word j of a value starts at all ones (AND / MIN identity) */
uint64_t and_mask(const ShardMap &sm) {
    uint64_t m = 0;
    for (size_t j = 0; j < sm.op.size() && j < 64; j++)
        if ((sm.op[j] & 0xF) == UC_AND || (sm.op[j] & 0xF) == UC_MIN) m |= 1ull << j;
    return m;
}

/* the flush of one value's accumulators at shared `acc` (expression) into device memory at `gbase` */
std::string flush_value(const ShardMap &sm, const std::string &acc, const std::string &gbase) {
    std::ostringstream o;
    for (uint32_t u = 0; u < sm.stride / 8; u++) {
        uint8_t lo = 2 * u < sm.op.size() ? sm.op[2 * u] : 0, hi = 2 * u + 1 < sm.op.size() ? sm.op[2 * u + 1] : 0;
        if (lo & UC_W8) {
            o << "      wc_flush_word<" << uc_op(lo) << ", 8>((void *)(" << gbase << " + " << u * 8 << "), ((const u64 *)("
              << acc << "))[" << u << "]);\n";
            continue;
        }
        for (int h = 0; h < 2; h++) {
            uint8_t c = h ? hi : lo;
            if (!c) continue;
            o << "      wc_flush_word<" << uc_op(c) << ", 4>((void *)(" << gbase << " + " << u * 8 + 4 * h
              << "), (u64)((const u32 *)(" << acc << "))[" << 2 * u + h << "]);\n";
        }
    }
    return o.str();
}

} // namespace

ShardPlan plan_shards(const JitProgram &p) {
    ShardPlan plan;
    /* only maps that some update instruction reaches with a known offset are worth a shard */
    std::vector<bool> targeted(p.maps.size(), false);
    std::vector<uint32_t> sites(p.maps.size(), 0);
    for (const InsnInfo &ii : p.info)
        if (ii.visited && ii.vmap >= 0 && ii.voff >= 0 && ii.voff < InsnInfo::ARG_VARIES && ii.vmap < (int)targeted.size()) {
            targeted[ii.vmap] = true;
            sites[ii.vmap]++;
        }
    /* private copies first (fixed offsets), then the caches (offsets follow the runtime width) */
    std::vector<ShardMap> caches;
    uint32_t off = 0, cache_max = 0;
    for (size_t m = 0; m < p.maps.size() && m < p.use.size(); m++) {
        const gx_map_spec &ms = p.maps[m];
        if (!targeted[m] || !p.use[m].combinable()) continue;
        if (ms.type != GX_MAP_ARRAY && ms.type != GX_MAP_HASH) continue;
        ShardMap sm;
        sm.map = (int)m;
        sm.stride = (ms.value_size + 7u) & ~7u;
        sm.op = p.use[m].op;
        sm.sites = sites[m];
        const uint64_t full_bytes = (uint64_t)ms.max_entries * sm.stride;
        if (ms.type == GX_MAP_ARRAY && full_bytes <= WC_FULL_MAX && sm.stride <= 256) {
            const uint32_t need = up16((uint32_t)full_bytes);
            if (off + need > WC_TOTAL_MAX) continue;
            sm.full = true;
            sm.n_values = ms.max_entries;
            sm.acc_off = off;
            off += need;
            plan.maps.push_back(sm);
        } else if (sm.stride <= 248) { /* an entry's words (tag + value) fit the 64-bit identity mask */
            uint32_t bits = WC_BITS;
            while (bits > 2 && (1u << bits) * (8u + sm.stride) > WC_CACHE_MAX) bits--;
            sm.max_bits = bits;
            caches.push_back(sm);
        }
    }
    plan.full_bytes = off;
    for (ShardMap &sm : caches) {
        /* narrow a cache that does not fit the program's area at its widest (down to 16 entries) */
        while (sm.max_bits > 4 && off + up16((1u << sm.max_bits) * (8u + sm.stride)) > WC_TOTAL_MAX) sm.max_bits--;
        const uint32_t need = up16((1u << sm.max_bits) * (8u + sm.stride));
        if (off + need > WC_TOTAL_MAX) continue;
        off += need;
        plan.max_bits = std::max(plan.max_bits, sm.max_bits);
        plan.maps.push_back(sm);
    }
    if (!plan.maps.empty() && plan.max_bits == 0) plan.max_bits = 1;
    for (uint32_t b = 0; b <= WC_BITS; b++) plan.bytes_for[b] = plan.bytes_at(b);
    return plan;
}

/* the area's bytes when caches hold 2^min(bits, their max) entries */
uint32_t ShardPlan::bytes_at(uint32_t bits) const {
    uint32_t off = full_bytes;
    for (const ShardMap &sm : maps)
        if (!sm.full) off += up16((1u << std::min(bits, sm.max_bits)) * (8u + sm.stride));
    return off;
}

namespace {

/* C++ expression: byte offset of cache `k` (index into sp.maps) for the runtime width env.wc_bits */
std::string cache_off(const ShardPlan &sp, size_t k) {
    std::string e = std::to_string(sp.full_bytes) + "u";
    for (size_t j = 0; j < k; j++) {
        const ShardMap &sm = sp.maps[j];
        if (sm.full) continue;
        e += " + (((1u << (env.wc_bits < " + std::to_string(sm.max_bits) + "u ? env.wc_bits : " +
             std::to_string(sm.max_bits) + "u)) * " + std::to_string(8 + sm.stride) + "u + 15u) & ~15u)";
    }
    return "(" + e + ")";
}

std::string cache_bits(const ShardMap &sm) {
    return "(env.wc_bits < " + std::to_string(sm.max_bits) + "u ? env.wc_bits : " + std::to_string(sm.max_bits) + "u)";
}

/* block start: identities everywhere (every thread of the block calls this) */
std::string gen_wc_init(const ShardPlan &sp, int slot) {
    std::ostringstream o;
    o << "__device__ __forceinline__ void gx_wc_init_" << slot << "(const ExecEnv &env) {\n";
    for (size_t k = 0; k < sp.maps.size(); k++) {
        const ShardMap &sm = sp.maps[k];
        const uint32_t wpv = sm.stride / 4;
        if (sm.full) {
            o << "  wc_fill(env.shard + " << sm.acc_off << ", " << sm.n_values * wpv << "u, " << wpv << "u, "
              << hex64(and_mask(sm)) << ");\n";
        } else { /* entries {u64 tag = 0, accumulators}: the tag's two words, then the value's */
            const uint32_t wpe = (8 + sm.stride) / 4;
            o << "  wc_fill(env.shard + " << cache_off(sp, k) << ", (1u << " << cache_bits(sm) << ") * " << wpe << "u, "
              << wpe << "u, " << hex64(and_mask(sm) << 2) << ");\n";
        }
    }
    o << "}\n";
    return o.str();
}

/* block end: add the block's totals into device memory (after a block barrier) */
std::string gen_wc_flush(const ShardPlan &sp, int slot) {
    std::ostringstream o;
    o << "__device__ __forceinline__ void gx_wc_flush_" << slot << "(const ExecEnv &env) {\n";
    for (size_t k = 0; k < sp.maps.size(); k++) {
        const ShardMap &sm = sp.maps[k];
        const std::string vals = "env.maps[" + std::to_string(sm.map) + "].values";
        if (sm.full) {
            o << "  for (u32 v_ = threadIdx.x; v_ < " << sm.n_values << "u; v_ += blockDim.x) {\n"
              << "    const uint8_t *a_ = env.shard + " << sm.acc_off << " + (size_t)v_ * " << sm.stride << ";\n"
              << "    const u64 g_ = (u64)(" << vals << " + (size_t)v_ * " << sm.stride << ");\n"
              << flush_value(sm, "a_", "g_") << "  }\n";
        } else {
            const uint32_t es = 8 + sm.stride;
            o << "  { const uint8_t *c_ = env.shard + " << cache_off(sp, k) << ";\n"
              << "    for (u32 e_ = threadIdx.x; e_ < (1u << " << cache_bits(sm) << "); e_ += blockDim.x) {\n"
              << "      const u64 g_ = *(const u64 *)(c_ + (size_t)e_ * " << es << ");\n"
              << "      if (!g_) continue;\n"
              << "      const uint8_t *a_ = c_ + (size_t)e_ * " << es << " + 8;\n"
              << flush_value(sm, "a_", "g_") << "    } }\n";
        }
    }
    o << "}\n\n";
    return o.str();
}

/* the longest run of arithmetic a forward jump may skip and still be emitted inline */
const int64_t FOLD_MAX = 8;

/* a program with more map-update and lookup sites than this calls their slow paths out of line */
const uint32_t OUTLINE_SITES = 8;

/* an update of map memory at `addr` by `val`: combined per block when the plan allows */
std::string gen_update(const ShardPlan &sp, const InsnInfo &ii, const char *op, int size, const std::string &addr,
                       const std::string &val, bool outline) {
    const std::string t0 = std::string("<") + op + ", " + std::to_string(size) + ">";
    std::string global = outline ? "dev_update" + t0 + "(" + addr + ", " + val + ", 1u);"
                                 : "agg_update" + t0 + "(" + addr + ", " + val + ", __activemask());";
    const ShardMap *sm = ii.vmap >= 0 && ii.voff >= 0 && ii.voff < InsnInfo::ARG_VARIES ? sp.find(ii.vmap) : nullptr;
    if (!sm) return global;
    const size_t k = (size_t)(sm - sp.maps.data());
    std::ostringstream o;
    std::string t = std::string("<") + op + ", " + std::to_string(size) + ">";
    o << "if (env.wc_bits) { const u64 a_ = " << addr << "; ";
    if (sm->full) {
        o << "sh_update" << t << "(sh_addr(env.shard + " << sm->acc_off << ") + (u32)(a_ - (u64)env.maps[" << sm->map
          << "].values), " << val << "); ";
    } else {
        const std::string look = "wc_entry(env.shard + " + cache_off(sp, k) + ", " + cache_bits(*sm) + ", " +
                                 std::to_string(8 + sm->stride) + "u, a_ - " + std::to_string(ii.voff) + "ull)";
        if (sm->sites > 1) {
            /* the event's last entry of this cache is reused for another word of the same value */
            const std::string kb = "wcb" + std::to_string(k), ke = "wce" + std::to_string(k);
            o << "uint8_t *e_ = " << ke << "; if (a_ - " << ii.voff << "ull != " << kb << ") { e_ = " << look << "; " << kb
              << " = a_ - " << ii.voff << "ull; " << ke << " = e_; } ";
        } else {
            o << "uint8_t *e_ = " << look << "; ";
        }
        o << "if (e_) sh_update" << t << "(sh_addr(e_) + " << ii.voff << "u, " << val << "); ";
        if (outline)
            o << "else dev_update" << t << "(a_, " << val << ", env.wc_agg); ";
        else
            o << "else if (env.wc_agg) agg_update" << t << "(a_, " << val << ", __activemask()); "
              << "else plain_atomic" << t << "((void *)a_, " << val << "); ";
    }
    o << "} else " << global;
    return o.str();
}

/*
 * The eBPF stack as 64 scalar slot variables s0..s63 (bytes 8k..8k+7 of the 512-byte
 * frame, little-endian), so the compiler keeps the live ones in registers.  Used when the
 * verifier proved every stack access has one constant offset.  Helpers that read stack
 * memory get the bytes copied into `stk_mem` (which R10 points into) just before the call.
 */
std::string stk_load(int abs, int size, bool sign) {
    const std::string v = "s" + std::to_string(abs / 8);
    const int b = abs % 8;
    if (size == 8) return v;
    const char *t = size == 4 ? (sign ? "int32_t" : "uint32_t") : size == 2 ? (sign ? "int16_t" : "uint16_t")
                                                                            : (sign ? "int8_t" : "uint8_t");
    std::string x = "(" + std::string(t) + ")(" + v + (b ? " >> " + std::to_string(8 * b) : "") + ")";
    return sign ? "(u64)(s64)" + x : "(u64)" + x;
}

std::string stk_store(int abs, int size, const std::string &val) {
    const std::string v = "s" + std::to_string(abs / 8);
    const int b = abs % 8;
    if (size == 8) return v + " = (u64)(" + val + ");";
    const std::string m = hex64(size == 4 ? 0xFFFFFFFFull : size == 2 ? 0xFFFFull : 0xFFull);
    const std::string sh = std::to_string(8 * b);
    return v + " = (" + v + " & ~(" + m + " << " + sh + ")) | (((u64)(" + val + ") & " + m + ") << " + sh + ");";
}

/* copy slots covering stack bytes [lo, 512) into stk_mem (lo = frame offset + 512) */
std::string stk_materialise(int lo) {
    std::string o;
    for (int k = std::max(0, lo) / 8; k < GX_STACK_BYTES / 8; k++)
        o += "stk_mem[" + std::to_string(k) + "] = s" + std::to_string(k) + "; ";
    return o;
}

/* one program -> `__device__ u64 gx_body_<slot>(env, ctxw, valid, ev_idx)` */
int gen_body(const JitProgram &p, const ShardPlan &sp, int slot, std::string &out, std::string &log) {
    const uint32_t n = (uint32_t)p.insns.size();
    std::vector<uint8_t> target(n + 1, 0);
    std::vector<uint8_t> leader(n + 1, 0); /* first instruction of a basic block */
    std::vector<uint32_t> tcount(n + 1, 0); /* jumps to each instruction */
    bool acyclic = true;
    leader[0] = 1;
    for (uint32_t pc = 0; pc < n; pc++) {
        if (!p.info[pc].visited) continue;
        uint64_t w = p.insns[pc];
        int op = (int)(w & 0xFF), cls = op & 7;
        int off = (int)(int16_t)(uint16_t)((w >> 16) & 0xFFFF);
        int32_t imm = (int32_t)(uint32_t)(w >> 32);
        if (op == 0x18) {
            pc++;
            continue;
        }
        if ((cls == 5 || cls == 6) && ((op & 0xF0) != 0x80)) {
            leader[pc + 1] = 1; /* after a jump or an exit */
            if ((op & 0xF0) == 0x90) continue;
            int64_t t = (int64_t)pc + 1 + ((cls == 6 && (op & 0xF0) == 0) ? imm : off);
            target[t] = 1;
            leader[t] = 1;
            tcount[t]++;
            if (t <= (int64_t)pc) acyclic = false;
        }
    }
    /*
     * Reconvergence by construction.  A program without loops (every jump forward) is
     * emitted as a sequence of its basic blocks, block b as "if (nb_ == b) { ...; nb_ =
     * successor; }" with nb_ the lane's next block, and an exit sets nb_ past every block
     * instead of returning.  So every valid lane passes every block boundary, in the same
     * order, and a __syncwarp over the valid lanes before a block that a jump lands on
     * joins lanes that took different branches.  Gotos are kept for programs with loops and for
     * warp-level handlers (whose lanes never diverge).
     */
    const bool structured = acyclic && !p.warp;
    /*
     * A conditional jump forward over a short run of register arithmetic (no memory,
     * helpers or jumps; reached only by falling through) stays inside its block as
     * "if (!cond) { run }": predicated code instead of two more blocks and joins.
     */
    std::vector<int64_t> fold(n + 1, -1); /* fold[pc]: the target of a jump at pc emitted inline */
    for (uint32_t pc = 0; structured && pc < n; pc++) {
        if (!p.info[pc].visited) continue;
        const uint64_t w = p.insns[pc];
        const int op = (int)(w & 0xFF), cls = op & 7, code = op & 0xF0;
        if (op == 0x18) {
            pc++;
            continue;
        }
        if ((cls != 5 && cls != 6) || code == 0x00 || code == 0x80 || code == 0x90) continue;
        const int64_t t = (int64_t)pc + 1 + (int)(int16_t)(uint16_t)((w >> 16) & 0xFFFF);
        if (t <= (int64_t)pc + 1 || t - pc - 1 > FOLD_MAX) continue;
        bool ok = true;
        for (int64_t k = pc + 1; k < t && ok; k++) {
            const int kc = (int)(p.insns[k] & 7);
            ok = p.info[k].visited && (kc == 4 || kc == 7) && tcount[k] == 0;
        }
        if (!ok) continue;
        fold[pc] = t;
        leader[pc + 1] = 0;
        if (tcount[t] == 1) leader[t] = 0; /* its other way in is falling through the run */
    }
    /*
     * Many map-update and lookup sites: their slow paths (device-memory updates, the
     * ordered hash probe) go out of line, so that a long program's code fits the
     * instruction cache; a few sites keep them inline and save the call.
     */
    uint32_t sites = 0;
    for (uint32_t pc = 0; pc < n; pc++) {
        if (!p.info[pc].visited) continue;
        const uint64_t w = p.insns[pc];
        const int op = (int)(w & 0xFF);
        const int32_t imm = (int32_t)(uint32_t)(w >> 32);
        if (op == 0x18) {
            pc++;
            continue;
        }
        if ((op & 0x07) == 3 && (op & 0xE0) == 0xC0 && p.info[pc].kind != MK_STACK) sites++;
        if (op == 0x85 && (imm == GX_HELPER_MAP_LOOKUP || imm == GX_HELPER_ATOMIC_MAX_U64 ||
                           imm == GX_HELPER_ATOMIC_MIN_U64))
            sites++;
    }
    const bool outline = sites > OUTLINE_SITES;
    /* scalar stack unless some load / store / atomic reaches the stack at a varying offset */
    bool scalar = true;
    for (uint32_t pc = 0; pc < n; pc++)
        if (p.info[pc].visited && p.info[pc].stk_any && p.info[pc].kind != MK_STACK) scalar = false;
    std::ostringstream o;
    o << "__device__ __forceinline__ u64 gx_body_" << slot
      << "(const ExecEnv &env, const u64 *ctxw, bool valid, u64 ev_idx) {\n";
    /*
     * Warp-level handler (SIMT-verified): the 32 lanes hold 32 consecutive events and follow
     * one path; helper calls and stores / atomics outside the lane's stack run on the first
     * valid lane and their results are broadcast; warp helpers reduce over the valid lanes.
     */
    if (p.warp) o << "  const u32 wmask = __ballot_sync(0xFFFFFFFFu, valid);\n";
    if (structured) o << "  const u32 vm_ = __ballot_sync(0xFFFFFFFFu, valid);\n";
    o << "  if (!valid) return 0;\n"
      << "  const u32 lane = threadIdx.x & 31;\n";
    if (p.warp) o << "  const u32 leader = (u32)__ffs(wmask) - 1u;\n  const bool lead = lane == leader;\n";
    if (scalar) {
        o << "  u64 stk_mem[" << GX_STACK_BYTES / 8 << "];\n  u64 ";
        for (int k = 0; k < GX_STACK_BYTES / 8; k++) o << (k ? ", s" : "s") << k << " = 0";
        o << ";\n  u64 r10 = (u64)(stk_mem + " << GX_STACK_BYTES / 8 << ");\n";
    } else {
        o << "  u64 stack[" << GX_STACK_BYTES / 8 << "];\n"
          << "  u64 r10 = (u64)(stack + " << GX_STACK_BYTES / 8 << ");\n";
    }
    o << "  u64 r0 = 0, r1 = 0, r2 = 0, r3 = 0, r4 = 0, r5 = 0, r6 = 0, r7 = 0, r8 = 0, r9 = 0;\n"
      << "  u64 back = 0;\n"
      << "  (void)lane; (void)ev_idx; (void)back; (void)r10;\n";
    if (structured) o << "  u32 nb_ = 0;\n";
    /*
     * Per cache: the value base and entry of the event's last cache lookup.  An entry holds
     * one value from its claim until the block's flush, so a lookup (or its miss) for the
     * same value stays valid for the rest of the event.  1 is no value's base.
     */
    for (size_t k = 0; k < sp.maps.size(); k++)
        if (!sp.maps[k].full && sp.maps[k].sites > 1)
            o << "  u64 wcb" << k << " = 1ull; uint8_t *wce" << k << " = nullptr; (void)wcb" << k << "; (void)wce" << k
              << ";\n";
    /* before a helper that reads stack memory through R2 / R3 */
    auto mat = [&](const InsnInfo &ii, bool r3_mem) -> std::string {
        if (!scalar) return "";
        int lo = GX_STACK_BYTES;
        for (int16_t a : {ii.a2, r3_mem ? ii.a3 : InsnInfo::ARG_UNSET}) {
            if (a == InsnInfo::ARG_UNSET) continue;
            if (a == InsnInfo::ARG_VARIES || a >= 0 || a < -GX_STACK_BYTES) lo = 0;
            else lo = std::min(lo, a + GX_STACK_BYTES);
        }
        return lo < GX_STACK_BYTES ? stk_materialise(lo) : "";
    };
    const uint64_t budget = p.budget;
    /* every path is shorter than the budget: no event can reach it, so no counting */
    const bool bounded = p.max_path && p.max_path <= budget;
    auto jump = [&](uint32_t pc, int64_t tgt) -> std::string {
        if (structured) return "nb_ = " + std::to_string(tgt) + "u;";
        std::string g = "goto L" + std::to_string(tgt) + ";";
        if (tgt <= (int64_t)pc && !bounded)
            return "{ if (++back > " + std::to_string(budget) + "ull) goto budget_trip; " + g + " }";
        return g;
    };
    bool block_ends = false; /* structured: the open block's last statement left it (jump or exit) */
    int64_t fold_end = -1;   /* structured: the end of an inline "if (!cond) { run }" */
    for (uint32_t pc = 0; pc < n; pc++) {
        const InsnInfo &ii = p.info[pc];
        uint64_t w = p.insns[pc];
        int op = (int)(w & 0xFF), cls = op & 7;
        int dst = (int)((w >> 8) & 0xF), src = (int)((w >> 12) & 0xF);
        int off = (int)(int16_t)(uint16_t)((w >> 16) & 0xFFFF);
        int32_t imm = (int32_t)(uint32_t)(w >> 32);
        if ((int64_t)pc == fold_end) {
            o << "  }\n";
            fold_end = -1;
        }
        if (structured && leader[pc] && ii.visited) {
            /* a join only where some jump lands: a block entered by falling through alone has
               the one way in, so its lanes need no regrouping */
            if (pc) o << (block_ends ? "  }\n" : "  nb_ = " + std::to_string(pc) + "u; }\n") << (tcount[pc] ? "  __syncwarp(vm_);\n" : "");
            o << "  if (nb_ == " << pc << "u) {\n";
            block_ends = false;
        } else if (!structured && target[pc]) {
            o << "L" << pc << ":;\n";
        }
        if (!ii.visited) {
            if (op == 0x18) pc++;
            continue;
        }
        o << "  ";
        switch (cls) {
        case 4: case 7: {
            bool w32 = cls == 4, x = op & 8;
            int code = op & 0xF0;
            std::string d = R(dst);
            if (code == 0xD0) {
                if (w32 && !x) {
                    if (imm == 16) o << d << " &= 0xFFFFull;";
                    else if (imm == 32) o << d << " &= 0xFFFFFFFFull;";
                    else o << ";";
                } else if (imm == 16) {
                    o << d << " = (u64)__byte_perm((u32)" << d << ", 0u, 0x4401u);";
                } else if (imm == 32) {
                    o << d << " = (u64)__byte_perm((u32)" << d << ", 0u, 0x0123u);";
                } else {
                    o << d << " = ((u64)__byte_perm((u32)" << d << ", 0u, 0x0123u) << 32) | (u64)__byte_perm((u32)("
                      << d << " >> 32), 0u, 0x0123u);";
                }
                break;
            }
            if (code == 0x80) {
                o << d << (w32 ? " = (u64)(u32)(0u - (u32)" + d + ");" : " = (u64)0 - " + d + ";");
                break;
            }
            if (code == 0xB0 && off) {
                const char *t = off == 8 ? "int8_t" : off == 16 ? "int16_t" : "int32_t";
                if (w32) o << d << " = (u64)(u32)(int32_t)(" << t << ")" << R(src) << ";";
                else o << d << " = (u64)(s64)(" << t << ")" << R(src) << ";";
                break;
            }
            const char *oname = alu_op(code, off);
            if (!oname) {
                log = "jit: unknown ALU op";
                return GX_EINVAL;
            }
            std::string s = x ? R(src) : (w32 ? hex64((uint32_t)imm) : hex64((uint64_t)(int64_t)imm));
            const bool call = x && (code == 0x30 || code == 0x90); /* division by a register: out of line */
            if (code == 0xB0 && !w32) o << d << " = " << s << ";";
            else
                o << d << " = " << (w32 ? (call ? "a32_call<" : "a32<") : (call ? "a64_call<" : "a64<")) << oname << ">("
                  << d << ", " << s << ");";
            break;
        }
        case 5: case 6: {
            int code = op & 0xF0;
            if (code == 0x00) {
                int64_t t = (int64_t)pc + 1 + (cls == 6 ? imm : off);
                o << jump(pc, t);
                block_ends = true;
                break;
            }
            if (code == 0x90) {
                o << (structured ? "nb_ = 0xFFFFFFFFu;" : "return r0;");
                block_ends = true;
                break;
            }
            if (code == 0x80 && p.warp && imm >= GX_HELPER_WARP_SUM_U64 && imm <= GX_HELPER_WARP_COUNT) {
                static const char *red[] = {"AG_ADD", "AG_MAX", "AG_MIN", "AG_OR", "AG_AND"};
                if (imm == GX_HELPER_WARP_COUNT) o << "r0 = (u64)__popc(__ballot_sync(wmask, r1 != 0ull));";
                else o << "r0 = group_reduce<" << red[imm - GX_HELPER_WARP_SUM_U64] << ", 8>(wmask, r1);";
                break;
            }
            if (code == 0x80) {
                std::string m = ii.map >= 0 ? "env.maps[" + std::to_string(ii.map) + "]" : "env.maps[r1]";
                const bool inline_lookup = imm == GX_HELPER_MAP_LOOKUP && ii.map >= 0 && ii.map < (int)p.maps.size() &&
                                           ii.a2 < 0 && ii.a2 >= -GX_STACK_BYTES &&
                                           (p.maps[ii.map].type == GX_MAP_ARRAY ||
                                            (p.maps[ii.map].type == GX_MAP_HASH &&
                                             (p.maps[ii.map].key_size == 1 || p.maps[ii.map].key_size == 2 ||
                                              p.maps[ii.map].key_size == 4 || p.maps[ii.map].key_size == 8)));
                if (!inline_lookup && imm != GX_HELPER_ATOMIC_MAX_U64 && imm != GX_HELPER_ATOMIC_MIN_U64 &&
                    imm != GX_HELPER_RINGBUF_SUBMIT && imm != GX_HELPER_RINGBUF_DISCARD &&
                    imm != GX_HELPER_RINGBUF_RESERVE)
                    o << mat(ii, imm == GX_HELPER_MAP_UPDATE);
                if (p.warp) o << "if (lead) { ";
                switch (imm) {
                case GX_HELPER_MAP_LOOKUP: {
                    /* one map and a key at a known stack slot: inline, per lane, layout as constants */
                    const gx_map_spec *ms = ii.map >= 0 && ii.map < (int)p.maps.size() ? &p.maps[ii.map] : nullptr;
                    const uint32_t vs = ms ? (ms->value_size + 7u) & ~7u : 0;
                    auto key = [&](int ks) {
                        const int abs = ii.a2 + GX_STACK_BYTES;
                        if (scalar) return stk_load(abs, ks, false);
                        return "load_sz<" + std::to_string(ks) + ", false>((const uint8_t *)stack + " +
                               std::to_string(abs) + ")";
                    };
                    if (inline_lookup && ms->type == GX_MAP_ARRAY) {
                        o << "{ const u32 k_ = (u32)" << key(4) << "; r0 = k_ < " << ms->max_entries
                          << "u ? (u64)(" << m << ".values + (u64)k_ * " << vs << "u) : 0ull; }";
                    } else if (inline_lookup) {
                        const std::string ks = std::to_string(ms->key_size);
                        o << "r0 = hash_find_word" << ((ms->flags & GX_MAP_F_NO_DELETE) ? "_nd<" : "<") << ks << ", "
                          << vs << ((ms->flags & GX_MAP_F_NO_DELETE) && outline ? ", true" : "") << ">(" << m << ", "
                          << key(ms->key_size) << ", env.stats);";
                    } else {
                        o << "r0 = map_lookup(" << m << ", (const uint8_t *)r2, __activemask(), env.stats);";
                    }
                    break;
                }
                case GX_HELPER_MAP_UPDATE:
                    o << "r0 = (u64)(s64)map_update(" << m
                      << ", (const uint8_t *)r2, (const uint8_t *)r3, r4, __activemask(), env.stats);";
                    break;
                case GX_HELPER_MAP_DELETE:
                    o << "r0 = (u64)(s64)(" << m << ".type == GX_MAP_HASH ? hash_delete(" << m
                      << ", (const uint8_t *)r2, env.stats) : GX_EINVAL);";
                    break;
                case GX_HELPER_RINGBUF_RESERVE:
                    o << "r0 = rb_reserve(" << m << ", r2, __activemask(), ev_idx);";
                    break;
                case GX_HELPER_RINGBUF_OUTPUT:
                    o << "{ u64 p_ = rb_reserve(" << m << ", r3, __activemask(), ev_idx); if (p_) copy_bytes((uint8_t *)p_, "
                      << "(const uint8_t *)r2, (u32)r3); r0 = p_ ? 0 : (u64)(s64)GX_EAGAIN; }";
                    break;
                case GX_HELPER_RINGBUF_SUBMIT:
                    o << ";";
                    break;
                case GX_HELPER_RINGBUF_DISCARD:
                    o << "((u32 *)(r1 - GX_RB_HDR))[1] = GX_RB_DISCARDED;";
                    break;
                case GX_HELPER_ATOMIC_MAX_U64:
                    o << gen_update(sp, ii, "AG_MAX", 8, "r1", "r2", outline);
                    break;
                case GX_HELPER_ATOMIC_MIN_U64:
                    o << gen_update(sp, ii, "AG_MIN", 8, "r1", "r2", outline);
                    break;
                default: log = "jit: unknown helper"; return GX_EINVAL;
                }
                /* the lanes wait for the leader's work and see its memory effects, then take its result */
                if (p.warp) o << " } __syncwarp(wmask); r0 = __shfl_sync(wmask, r0, leader);";
                break;
            }
            const char *c = cond_op(code);
            if (!c) {
                log = "jit: unknown jump";
                return GX_EINVAL;
            }
            bool w32 = cls == 6, x = op & 8;
            std::string s = x ? R(src) : (w32 ? hex64((uint32_t)imm) : hex64((uint64_t)(int64_t)imm));
            int64_t t = (int64_t)pc + 1 + off;
            if (structured && fold[pc] >= 0) {
                o << "if (!" << (w32 ? "c32<" : "c64<") << c << ">(" << R(dst) << ", " << s << ")) {";
                fold_end = t;
                break;
            }
            if (structured) {
                o << "nb_ = " << (w32 ? "c32<" : "c64<") << c << ">(" << R(dst) << ", " << s << ") ? " << t << "u : "
                  << pc + 1 << "u;";
                block_ends = true;
                break;
            }
            o << "if (" << (w32 ? "c32<" : "c64<") << c << ">(" << R(dst) << ", " << s << ")) " << jump(pc, t);
            break;
        }
        case 0: {
            if (src == 1) o << R(dst) << " = " << imm << "ull;";
            else o << R(dst) << " = " << hex64((uint64_t)(uint32_t)imm | ((p.insns[pc + 1] >> 32) << 32)) << ";";
            pc++;
            break;
        }
        case 1: {
            int size = size_of(op);
            bool sign = (op & 0xE0) == 0x80;
            std::string ld = "load_sz<" + std::to_string(size) + ", " + (sign ? "true" : "false") + ">(";
            if (ii.kind == MK_CTX)
                o << R(dst) << " = " << ld << "(const uint8_t *)(ctxw + " << (ii.off >> 3) * GX_CTX_ROW(p.ctx_size / 8)
                  << " + lane) + " << (ii.off & 7) << ");";
            else if (ii.kind == MK_STACK && scalar)
                o << R(dst) << " = " << stk_load(ii.off + GX_STACK_BYTES, size, sign) << ";";
            else if (ii.kind == MK_STACK)
                o << R(dst) << " = " << ld << "(const uint8_t *)stack + " << ii.off + GX_STACK_BYTES << ");";
            else
                o << R(dst) << " = " << ld << "(const uint8_t *)(" << R(src) << " + " << hex64((uint64_t)(int64_t)off)
                  << "));";
            break;
        }
        case 2: case 3: {
            int size = size_of(op);
            if (ii.kind == MK_STACK && scalar) {
                const int abs = ii.off + GX_STACK_BYTES;
                if ((op & 0xE0) != 0xC0) {
                    o << stk_store(abs, size, cls == 3 ? R(src) : hex64((uint64_t)(int64_t)imm));
                    break;
                }
                const std::string old_v = stk_load(abs, size, false), sr = R(src);
                const std::string mask = size == 4 ? " & 0xFFFFFFFFull" : "";
                o << "{ const u64 o_ = " << old_v << "; ";
                if (imm == 0xE1) {
                    o << stk_store(abs, size, sr) << " " << sr << " = o_; }";
                } else if (imm == 0xF1) {
                    o << "if (o_ == (r0" << mask << ")) " << stk_store(abs, size, sr) << " r0 = o_; }";
                } else {
                    int b = imm & ~1;
                    const char *opx = b == 0x00 ? "+" : b == 0x40 ? "|" : b == 0x50 ? "&" : "^";
                    o << stk_store(abs, size, "o_ " + std::string(opx) + " " + sr) << " ";
                    if (imm & 1) o << sr << " = o_; ";
                    o << "}";
                }
                break;
            }
            std::string addr = ii.kind == MK_STACK
                                   ? "(u64)((uint8_t *)stack + " + std::to_string(ii.off + GX_STACK_BYTES) + ")"
                                   : "(" + R(dst) + " + " + hex64((uint64_t)(int64_t)off) + ")";
            /* warp-level handler: outside the lane's stack the leader writes, the fetched value is broadcast */
            std::string bcast;
            if (p.warp && ii.kind != MK_STACK) {
                o << "{ const u64 wa_ = " << addr << "; const bool sh_ = !__isLocal((const void *)wa_); if (!sh_ || lead) { ";
                addr = "wa_"; /* gen_update declares its own a_ */
                if ((op & 0xE0) == 0xC0 && imm == 0xF1) bcast = "r0";
                else if ((op & 0xE0) == 0xC0 && (imm & 1)) bcast = R(src);
            }
            auto close = [&]() {
                if (!p.warp || ii.kind == MK_STACK) return;
                o << " } __syncwarp(wmask);"; /* later loads of any lane see the leader's write */
                if (!bcast.empty()) o << " if (sh_) " << bcast << " = __shfl_sync(wmask, " << bcast << ", leader);";
                o << " }";
            };
            if ((op & 0xE0) == 0xC0) {
                std::string sz = std::to_string(size);
                if (imm == 0xE1) o << R(src) << " = xchg<" << sz << ">(" << addr << ", " << R(src) << ");";
                else if (imm == 0xF1) o << "r0 = cmpxchg<" << sz << ">(" << addr << ", r0, " << R(src) << ");";
                else {
                    int b = imm & ~1;
                    const char *ag = b == 0x00 ? "AG_ADD" : b == 0x40 ? "AG_OR" : b == 0x50 ? "AG_AND" : "AG_XOR";
                    if (imm & 1) o << R(src) << " = fetch_update<" << ag << ", " << sz << ">(" << addr << ", " << R(src) << ");";
                    else if (ii.kind == MK_STACK) o << "agg_update<" << ag << ", " << sz << ">(" << addr << ", " << R(src) << ", __activemask());";
                    else o << gen_update(sp, ii, ag, size, addr, R(src), outline);
                }
                close();
                break;
            }
            std::string v = cls == 3 ? R(src) : hex64((uint64_t)(int64_t)imm);
            o << "store_sz<" << size << ">((uint8_t *)" << addr << ", " << v << ");";
            close();
            break;
        }
        }
        o << "\n";
    }
    if (structured) o << "  }\n  return r0;\n"; /* the verifier rules out falling off the end */
    o << "budget_trip:\n"
      << (p.warp ? "  if (lead) atomicAdd(&env.stats[GX_STAT_BUDGET], 1ull);\n" /* one handler per warp */
                 : "  atomicAdd(&env.stats[GX_STAT_BUDGET], 1ull);\n")
      << "  set_status(env.stats, GX_E_BUDGET);\n"
      << "  return 0;\n}\n\n";
    out += o.str();
    return GX_OK;
}

std::string fnv_hex(const std::string &s) {
    uint64_t h = 0xcbf29ce484222325ULL; /* FNV-1a (64-bit): offset basis, then xor and multiply by the prime */
    for (unsigned char c : s) {
        h ^= c;
        h *= 0x100000001b3ULL;
    }
    char b[24];
    snprintf(b, sizeof b, "%016llx", (unsigned long long)h);
    return b;
}

struct Cached {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kernel = nullptr;
    cudaKernel_t variant[5] = {};
};

/*
 * The compiled entries: a kernel is compiled once per minimum of resident 256-thread blocks
 * per SM (launch bounds), which caps its registers per thread.  Without a minimum the
 * compiler may still pick few registers and spill heavily, so every entry states one.
 * Index: GX_VARIANT_*; one program gets all four, several programs wide and capped.
 */
struct EntrySpec {
    uint32_t variant;
    const char *name;
    int min_blocks;
};
const EntrySpec ENTRIES[] = {{GX_VARIANT_WIDE, "gx_jit_kernel", 2},
                             {GX_VARIANT_CAPPED, "gx_jit_kernel_capped", 5},
                             {GX_VARIANT_3, "gx_jit_kernel_v3", 3},
                             {GX_VARIANT_4, "gx_jit_kernel_v4", 4}};

/* every kernel gets the four entries, except work-stealing ones (the wide and the capped) */
bool entry_built(uint32_t variant, size_t n_progs, bool sched) {
    (void)n_progs;
    return !sched || variant == GX_VARIANT_WIDE || variant == GX_VARIANT_CAPPED;
}
std::mutex cache_mu;
std::map<std::string, Cached> cache;

bool read_file(const std::string &path, std::vector<char> &out) {
    FILE *f = fopen(path.c_str(), "rb");
    if (!f) return false;
    fseek(f, 0, SEEK_END);
    long n = ftell(f);
    fseek(f, 0, SEEK_SET);
    out.resize(n > 0 ? (size_t)n : 0);
    bool ok = n > 0 && fread(out.data(), 1, (size_t)n, f) == (size_t)n;
    fclose(f);
    return ok;
}

void write_file(const std::string &path, const std::vector<char> &data) {
    /* a name of its own per writer (process and call), so concurrent writers of one key never
       share a temporary file; the rename publishes a complete file */
    static std::atomic<unsigned long> seq{0};
    std::string tmp = path + ".tmp" + std::to_string((unsigned long)getpid()) + "." + std::to_string(seq++);
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return;
    bool ok = fwrite(data.data(), 1, data.size(), f) == data.size();
    fclose(f);
    if (ok) rename(tmp.c_str(), path.c_str());
    else remove(tmp.c_str());
}

/* keep the disk cache within GX_JIT_CACHE_MB (default 1 GiB): remove the least recently
   written cubins first */
void trim_cache(const std::string &dir) {
    const char *mb = getenv("GX_JIT_CACHE_MB");
    const uint64_t cap = (mb && *mb ? strtoull(mb, nullptr, 10) : 1024ULL) << 20;
    DIR *d = opendir(dir.c_str());
    if (!d) return;
    struct Entry {
        std::string path;
        time_t mtime;
        uint64_t bytes;
    };
    std::vector<Entry> es;
    uint64_t total = 0;
    while (struct dirent *e = readdir(d)) {
        const std::string name = e->d_name;
        if (name.size() < 7 || name.compare(name.size() - 6, 6, ".cubin") != 0) continue;
        struct stat st;
        const std::string path = dir + "/" + name;
        if (stat(path.c_str(), &st) != 0) continue;
        es.push_back({path, st.st_mtime, (uint64_t)st.st_size});
        total += (uint64_t)st.st_size;
    }
    closedir(d);
    if (total <= cap) return;
    std::sort(es.begin(), es.end(), [](const Entry &a, const Entry &b) { return a.mtime < b.mtime; });
    for (const Entry &e : es) {
        if (total <= cap) break;
        if (remove(e.path.c_str()) == 0) total -= e.bytes;
    }
}

} // namespace

std::string jit_source(const std::vector<const JitProgram *> &progs, std::string &log, int &rc,
                       const JitProgram *sched = nullptr) {
    std::string src;
    src += "#include \"gx_device.cuh\"\n";
    if (sched) src += "#include \"gx_steal.cuh\"\n";
    src += "namespace gx {\n";
    rc = GX_OK;
    for (size_t i = 0; i < progs.size() && rc == GX_OK; i++) {
        const ShardPlan sp = plan_shards(*progs[i]);
        rc = gen_body(*progs[i], sp, (int)i, src, log);
        src += gen_wc_init(sp, (int)i);
        src += gen_wc_flush(sp, (int)i);
    }
    /* the scheduling program: per-lane code with no combining, out of line (run rarely, by warp 0) */
    const std::string hs = std::to_string(progs.size());
    if (sched && rc == GX_OK) {
        rc = gen_body(*sched, ShardPlan{}, (int)progs.size(), src, log);
        src += "__device__ __noinline__ u64 gx_sched_call(const ExecEnv &e, const u64 *c, bool v, u64 x) {\n"
               "  return gx_body_" + hs + "(e, c, v, x);\n}\n";
    }
    auto hook = [&](const char *what) {
        std::string h = std::string("  [](const gx::ExecEnv &env) {\n");
        if (progs.size() == 1) {
            h += std::string("    gx::gx_wc_") + what + "_0(env);\n";
        } else {
            h += "    switch (env.slot) {\n";
            for (size_t i = 0; i < progs.size(); i++)
                h += "    case " + std::to_string(i) + ": gx::gx_wc_" + what + "_" + std::to_string(i) + "(env); break;\n";
            h += "    }\n";
        }
        return h + "  }";
    };
    /*
     * Several programs: each one's chunk loop is its own out-of-line function, so every
     * program gets its own register allocation (one kernel-wide allocation over all bodies
     * spills) and the dispatch costs one call per chunk, not per event.
     */
    /* 32- and 64-byte records take the tile loop with the next tile's loads in flight */
    auto chunk_loop = [&progs](size_t i) {
        const uint32_t cs = progs[i]->ctx_size;
        const std::string loop = cs == 32 ? "chunk_tiles_cw<4>" : cs == 64 ? "chunk_tiles_cw<8>" : "chunk_tiles";
        return loop + "(env, ch, ctx_all, [](const ExecEnv &e, const u64 *c, bool v, u64 x) -> u64 { return gx_body_" +
               std::to_string(i) + "(e, c, v, x); });";
    };
    /* the stealing skeleton keeps its walk's state live across chunks: its chunk loops go out of line too */
    const bool ool = progs.size() > 1 || sched;
    if (ool)
        for (size_t i = 0; i < progs.size(); i++)
            src += "__device__ __noinline__ void gx_chunk_" + std::to_string(i) +
                   "(const gx_chunk ch, u32 wcp, u32 shard_off, u64 *ctx_all) {\n"
                   "  extern __shared__ __align__(16) uint8_t smem[];\n"
                   "  const ExecEnv env = stage_env_at(smem, shard_off, (u32)ch.pad, wcp);\n  " +
                   chunk_loop(i) + "\n}\n";
    std::string body = std::string("  gx::") + (sched ? "exec_steal" : "exec_tiles") +
                       "(P, [](const gx::ExecEnv &env, const gx_chunk &ch, gx::u64 *ctx_all) {\n";
    if (!ool) {
        body += "    using namespace gx;\n    " + chunk_loop(0) + "\n";
    } else {
        body += "    extern __shared__ __align__(16) uint8_t smem_base[];\n    switch (env.slot) {\n";
        for (size_t i = 0; i < progs.size(); i++)
            body += "    case " + std::to_string(i) + ": gx::gx_chunk_" + std::to_string(i) +
                    "(ch, env.wc_bits | (env.wc_agg << 8), (gx::u32)(env.shard - smem_base), ctx_all); break;\n";
        body += "    }\n";
    }
    body += "  },\n" + hook("init") + ",\n" + hook("flush");
    if (sched)
        body += ",\n  [](const gx::ExecEnv &e, const gx::u64 *c, bool v, gx::u64 x) -> gx::u64 { return "
                "gx::gx_sched_call(e, c, v, x); }";
    body += ");\n}\n";
    src += "} // namespace gx\n\n";
    /*
     * Four entries, from wide (two blocks per SM, up to 128 registers) to capped (five
     * blocks, 48 registers); the autotuner picks.  A kernel of several programs defaults to
     * the capped entry, so that one heavy program does not cut every program's occupancy;
     * a work-stealing kernel has the wide and the capped entry only.
     */
    for (const EntrySpec &e : ENTRIES) {
        if (!entry_built(e.variant, progs.size(), sched != nullptr)) continue;
        src += "extern \"C\" __global__ void __launch_bounds__(256, " + std::to_string(e.min_blocks) + ") " + e.name +
               "(gx::ExecParams P) {\n" + body;
    }
    return src;
}

/* generated source -> cubin (disk cache first, then NVRTC) */
int jit_cubin(const std::string &src, const std::string &key, std::vector<char> &cubin, std::string &log) {
    const char *dump = getenv("GX_JIT_DUMP_DIR");
    if (dump && *dump) {
        mkdir(dump, 0755);
        write_file(std::string(dump) + "/" + key + ".cu", std::vector<char>(src.begin(), src.end()));
    }
    const char *dir = getenv("GX_JIT_CACHE");
    std::string path = dir && *dir ? std::string(dir) + "/" + key + ".cubin" : "";
    if (!path.empty() && read_file(path, cubin)) return GX_OK;
    Nvrtc &nv = nvrtc();
    if (!nv.ok) {
        log = "jit: " + nv.err;
        return GX_E_NODEV;
    }
    const char *hdrs[] = {gx_embed_gx_h, gx_embed_gx_layout_h, gx_embed_gx_device_cuh, gx_embed_gx_steal_cuh};
    const char *names[] = {"gx.h", "gx_layout.h", "gx_device.cuh", "gx_steal.cuh"};
    nvrtcProgram_ prog = nullptr;
    if (nv.create(&prog, src.c_str(), "gx_prog.cu", 4, hdrs, names) != 0) {
        log = "jit: nvrtcCreateProgram failed";
        return GX_E_CUDA;
    }
    /* split compilation: the compiler optimises the kernel entries and out-of-line functions
       (one per program in a batch) on parallel threads */
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo", "-DNDEBUG", "-w",
                          "--split-compile=0"};
    int rc = nv.compile(prog, 6, opts);
    size_t ls = 0;
    nv.log_size(prog, &ls);
    std::string clog(ls, '\0');
    if (ls) nv.log(prog, &clog[0]);
    if (rc != 0) {
        log = "jit: compile failed: " + clog.substr(0, 4000);
        nv.destroy(&prog);
        return GX_E_CUDA;
    }
    size_t cs = 0;
    nv.cubin_size(prog, &cs);
    cubin.resize(cs);
    nv.cubin(prog, cubin.data());
    nv.destroy(&prog);
    if (!path.empty()) {
        mkdir(dir, 0755);
        write_file(path, cubin);
        trim_cache(dir);
    }
    return GX_OK;
}

std::string jit_key(const std::string &src) {
    return fnv_hex(src + gx_embed_gx_device_cuh + gx_embed_gx_layout_h + gx_embed_gx_h + gx_embed_gx_steal_cuh);
}

int jit_build(const std::vector<const JitProgram *> &progs, JitKernel &out, std::string &log,
              const JitProgram *sched) {
    int rc;
    const std::string src = jit_source(progs, log, rc, sched);
    if (rc) return rc;
    out.shard_bytes = 0;
    out.wc_max_bits = 0;
    for (uint32_t &b : out.shard_bytes_for) b = 0;
    for (const JitProgram *p : progs) {
        const ShardPlan sp = plan_shards(*p);
        out.wc_max_bits = std::max(out.wc_max_bits, sp.max_bits);
        for (uint32_t b = 0; b <= WC_BITS; b++) out.shard_bytes_for[b] = std::max(out.shard_bytes_for[b], sp.bytes_for[b]);
    }
    out.shard_bytes = out.shard_bytes_for[WC_BITS];
    const std::string key = jit_key(src);
    {
        std::lock_guard<std::mutex> g(cache_mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            out.kernel = it->second.kernel;
            for (int v = 0; v < 5; v++) out.variant[v] = it->second.variant[v];
            out.key = key;
            return GX_OK;
        }
    }
    std::vector<char> cubin;
    rc = jit_cubin(src, key, cubin, log);
    if (rc) return rc;
    Cached c;
    bool ok = cudaLibraryLoadData(&c.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) == cudaSuccess;
    for (const EntrySpec &e : ENTRIES) {
        if (!ok || !entry_built(e.variant, progs.size(), sched != nullptr)) continue;
        ok = cudaLibraryGetKernel(&c.variant[e.variant], c.lib, e.name) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        log = "jit: loading the compiled program failed";
        return GX_E_CUDA;
    }
    c.kernel = progs.size() == 1 && !sched ? c.variant[GX_VARIANT_4] : c.variant[GX_VARIANT_CAPPED];
    {
        std::lock_guard<std::mutex> g(cache_mu);
        cache[key] = c;
    }
    out.kernel = c.kernel;
    for (int v = 0; v < 5; v++) out.variant[v] = c.variant[v];
    out.key = key;
    return GX_OK;
}

uint64_t path_bound(const uint64_t *insns, uint32_t n, const gx_map_spec *maps, uint32_t n_maps,
                    const gx_prog_opts &opts) {
    /*
     * The SIMT pass with every ctx byte uniform accepts what the per-lane verifier accepts,
     * and it counts each path's instructions, pruning a state only by a kept state whose
     * count is at least as large: its maximum is the longest path's length.
     */
    SimtIn in;
    in.uniform.assign(opts.ctx_size, 1);
    VerifyOut v;
    if (verify_program(insns, n, maps, n_maps, opts, v, &in) != GX_OK) return 0;
    return v.simt.max_insns;
}

int check_sched_program(const uint64_t *insns, uint32_t n, const gx_map_spec *maps, uint32_t n_maps,
                        const gx_prog_opts &opts, const gx_simt_spec *limits, VerifyOut &v) {
    if (opts.ctx_size != GX_SCHED_CTX) {
        v.log = "scheduling program: ctx_size must be " + std::to_string(GX_SCHED_CTX);
        return GX_EINVAL;
    }
    if (limits && limits->reserved) {
        v.log = "scheduling program: limits->reserved must be 0";
        return GX_EINVAL;
    }
    SimtIn in;
    in.uniform.assign(GX_SCHED_CTX, 1); /* every field is the same for the block's threads */
    in.max_insns = limits ? limits->max_insns : GX_SCHED_MAX_INSNS;
    in.max_helpers = limits ? limits->max_helper_calls : GX_SCHED_MAX_HELPERS;
    in.max_mem = limits ? limits->max_mem_ops : GX_SCHED_MAX_MEM;
    return verify_program(insns, n, maps, n_maps, opts, v, &in);
}

cudaError_t jit_launch(const JitKernel &k, const ExecParams &p, unsigned grid, unsigned block, size_t smem,
                       cudaStream_t s, uint32_t variant) {
    void *args[] = {(void *)&p};
    return cudaLaunchKernel((const void *)jit_entry(k, variant), dim3(grid), dim3(block), args, smem, s);
}

cudaError_t jit_set_smem(JitKernel &k, size_t bytes) {
    if (bytes <= k.smem_attr) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute((const void *)k.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    for (int v = 1; v < 5 && e == cudaSuccess; v++)
        if (k.variant[v])
            e = cudaFuncSetAttribute((const void *)k.variant[v], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) k.smem_attr = bytes;
    return e;
}

cudaError_t jit_occupancy(const JitKernel &k, int block, size_t smem, int *blocks_per_sm, uint32_t variant) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, (const void *)jit_entry(k, variant), block, smem);
}

} // namespace gx

extern "C" int gx_jit_check(const uint64_t *insns, uint32_t n, const gx_map_spec *maps, uint32_t n_maps,
                            const gx_prog_opts *opts, char *log, size_t log_len) {
    if (!insns || !opts || (n_maps && !maps)) return GX_EINVAL;
    gx::VerifyOut v;
    int rc = gx::verify_program(insns, n, maps, n_maps, *opts, v);
    std::string msg = v.log;
    if (rc == GX_OK) {
        gx::JitProgram jp;
        jp.insns.assign(insns, insns + n);
        jp.info = v.info;
        jp.maps.assign(maps, maps + n_maps);
        jp.use = v.map_use;
        jp.ctx_size = opts->ctx_size;
        jp.budget = opts->insn_budget ? opts->insn_budget : (1ull << 16);
        jp.max_path = gx::path_bound(insns, n, maps, n_maps, *opts);
        const std::string src = gx::jit_source({&jp}, msg, rc);
        std::vector<char> cubin;
        if (rc == GX_OK) rc = gx::jit_cubin(src, gx::jit_key(src), cubin, msg);
    }
    if (log && log_len) {
        size_t k = std::min(log_len - 1, msg.size());
        memcpy(log, msg.data(), k);
        log[k] = 0;
    }
    return rc;
}

extern "C" int gx_jit_check_simt(const uint64_t *insns, uint32_t n, const gx_map_spec *maps, uint32_t n_maps,
                                 const gx_prog_opts *opts, const gx_simt_spec *simt, char *log, size_t log_len) {
    if (!insns || !opts || !simt || (n_maps && !maps) || simt->reserved) return GX_EINVAL;
    if (opts->ctx_size < 8 || opts->ctx_size > GX_MAX_CTX) return GX_EINVAL;
    const gx::SimtIn in = gx::simt_in(*simt, opts->ctx_size);
    gx::VerifyOut v;
    int rc = gx::verify_program(insns, n, maps, n_maps, *opts, v, &in);
    std::string msg = v.log;
    if (rc == GX_OK) {
        gx::JitProgram jp;
        jp.insns.assign(insns, insns + n);
        jp.info = v.info;
        jp.maps.assign(maps, maps + n_maps);
        jp.use = v.map_use;
        jp.ctx_size = opts->ctx_size;
        jp.budget = opts->insn_budget ? opts->insn_budget : (1ull << 16);
        jp.max_path = v.simt.max_insns;
        jp.warp = true;
        const std::string src = gx::jit_source({&jp}, msg, rc);
        std::vector<char> cubin;
        if (rc == GX_OK) rc = gx::jit_cubin(src, gx::jit_key(src), cubin, msg);
    }
    if (log && log_len) {
        size_t k = std::min(log_len - 1, msg.size());
        memcpy(log, msg.data(), k);
        log[k] = 0;
    }
    return rc;
}

extern "C" int gx_jit_check_sched(const uint64_t *insns, uint32_t n, const gx_map_spec *maps, uint32_t n_maps,
                                  const gx_prog_opts *opts, const uint64_t *hook, uint32_t n_hook,
                                  const gx_map_spec *hook_maps, uint32_t n_hook_maps, const gx_prog_opts *hook_opts,
                                  const gx_simt_spec *limits, char *log, size_t log_len) {
    if (!insns || !opts || (n_maps && !maps) || !hook || !hook_opts || (n_hook_maps && !hook_maps)) return GX_EINVAL;
    gx::VerifyOut v, hv;
    int rc = gx::verify_program(insns, n, maps, n_maps, *opts, v);
    std::string msg = v.log;
    if (rc == GX_OK) {
        rc = gx::check_sched_program(hook, n_hook, hook_maps, n_hook_maps, *hook_opts, limits, hv);
        msg = hv.log;
    }
    if (rc == GX_OK) {
        gx::JitProgram jp, hp;
        jp.insns.assign(insns, insns + n);
        jp.info = v.info;
        jp.maps.assign(maps, maps + n_maps);
        jp.use = v.map_use;
        jp.ctx_size = opts->ctx_size;
        jp.budget = opts->insn_budget ? opts->insn_budget : (1ull << 16);
        jp.max_path = gx::path_bound(insns, n, maps, n_maps, *opts);
        hp.insns.assign(hook, hook + n_hook);
        hp.info = hv.info;
        hp.maps.assign(hook_maps, hook_maps + n_hook_maps);
        hp.use = hv.map_use;
        hp.ctx_size = hook_opts->ctx_size;
        hp.budget = hook_opts->insn_budget ? hook_opts->insn_budget : (1ull << 16);
        hp.max_path = gx::path_bound(hook, n_hook, hook_maps, n_hook_maps, *hook_opts);
        const std::string src = gx::jit_source({&jp}, msg, rc, &hp);
        std::vector<char> cubin;
        if (rc == GX_OK) rc = gx::jit_cubin(src, gx::jit_key(src), cubin, msg);
    }
    if (log && log_len) {
        size_t k = std::min(log_len - 1, msg.size());
        memcpy(log, msg.data(), k);
        log[k] = 0;
    }
    return rc;
}
