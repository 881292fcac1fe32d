/* Host-side internals of the engine (not part of the C ABI). */
#ifndef GX_INTERNAL_H
#define GX_INTERNAL_H

#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gx.h"
#include "gx_layout.h"

namespace gx {

/* what the verifier learned about one instruction, consumed by the decoder */
enum MemKind : uint8_t { MK_NONE = 0, MK_CTX = 1, MK_STACK = 2, MK_MEM = 3 };

struct InsnInfo {
    uint8_t visited = 0;
    uint8_t kind = MK_NONE; /* region of a load / store / atomic */
    int16_t off = 0;        /* MK_CTX: absolute ctx offset; MK_STACK: offset from the frame top */
    int8_t map = -1;        /* helper call: map index in R1 on every path, -2 if it varies */
    int16_t a2 = ARG_UNSET; /* helper call: constant stack offset of R2 on every path (else ARG_VARIES) */
    int16_t a3 = ARG_UNSET; /* same for R3 */
    uint8_t stk_any = 0;    /* some path reaches the stack through this load / store / atomic */
    int8_t vmap = -1;       /* update of map memory (atomic, atomic max/min helper): the map on every path,
                               -2 if it varies or is not always a map value */
    int16_t voff = ARG_UNSET; /* ... and the constant byte offset within the value (else ARG_VARIES) */
    static const int16_t ARG_UNSET = 32767, ARG_VARIES = 32766;
};

/*
 * How a program touches the values of one map.  Updates that are non-fetching and
 * commutative (ADD / OR / AND / XOR atomics, the atomic max / min helpers) can be combined
 * per block in shared memory before they reach HBM, provided nothing else reads or
 * overwrites those values and every 4-byte word has a single operation.
 */
enum UpdClass : uint8_t { UC_NONE = 0, UC_ADD, UC_OR, UC_AND, UC_XOR, UC_MAX, UC_MIN, UC_W8 = 0x10 };
struct MapUse {
    bool other = false;      /* loaded, stored, exchanged, fetched, overwritten by update, passed to a helper,
                                or updated at a variable offset */
    bool mixed = false;      /* a word updated by two different operations or widths */
    std::vector<uint8_t> op; /* per 4-byte word of the value: UpdClass | UC_W8 for 8-byte operations */
    /*
     * Deterministic mode, for merging copies of the map built by several engines: per 4-byte
     * word the class of every update (any offset, fetching or not; UpdClass | UC_W8), and the
     * constant bytes the hash inserts write.  A word updated at two widths, or inserts of two
     * different constants, make the copies unmergeable.
     */
    std::vector<uint8_t> merge_op;
    bool merge_mixed = false;
    std::vector<uint8_t> insert;
    bool insert_seen = false, insert_conflict = false;
    bool combinable() const {
        if (other || mixed) return false;
        for (uint8_t c : op)
            if (c) return true;
        return false;
    }
};

/* SIMT-aware verification (gx_verify_simt): what to check and what was found */
struct SimtIn {
    std::vector<uint8_t> uniform; /* per ctx byte: nonzero = warp-uniform */
    uint32_t max_insns = 0, max_helpers = 0, max_mem = 0; /* per-path budgets, 0 = unlimited */
};
inline SimtIn simt_in(const gx_simt_spec &spec, uint32_t ctx_size) {
    SimtIn in;
    in.uniform.assign(ctx_size, 0);
    if (spec.uniform)
        for (uint32_t b = 0; b < ctx_size; b++) in.uniform[b] = spec.uniform[b] != 0;
    in.max_insns = spec.max_insns;
    in.max_helpers = spec.max_helper_calls;
    in.max_mem = spec.max_mem_ops;
    return in;
}
struct SimtOut {
    uint64_t max_insns = 0;
    uint32_t max_helpers = 0, max_mem = 0;
    uint32_t uniform_branches = 0, varying_insns = 0;
    int32_t pc = -1;
    uint32_t violation = GX_SIMT_V_NONE;
};

struct VerifyOut {
    std::vector<InsnInfo> info;
    std::string log;
    int32_t fail_pc = -1; /* the rejected instruction */
    SimtOut simt;
    uint64_t insns_processed = 0;
    uint64_t states_stored = 0;
    uint32_t stack_depth = 0; /* deepest stack byte touched */
    std::vector<MapUse> map_use; /* per map index */
};

/* returns GX_OK or GX_E_VERIFY / GX_EINVAL; out.log explains a rejection */
int verify_program(const uint64_t *insns, uint32_t n, const gx_map_spec *maps, uint32_t n_maps,
                   const gx_prog_opts &opts, VerifyOut &out, const SimtIn *simt = nullptr);

/* translate a verified program to micro-ops (see gx_layout.h) */
int decode_program(const uint64_t *insns, uint32_t n, const VerifyOut &v, std::vector<uint64_t> &uops,
                   std::string &log);

} // namespace gx

#endif
