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
    static const int16_t ARG_UNSET = 32767, ARG_VARIES = 32766;
};

struct VerifyOut {
    std::vector<InsnInfo> info;
    std::string log;
    uint64_t insns_processed = 0;
    uint64_t states_stored = 0;
    uint32_t stack_depth = 0; /* deepest stack byte touched */
};

/* returns GX_OK or GX_E_VERIFY / GX_EINVAL; out.log explains a rejection */
int verify_program(const uint64_t *insns, uint32_t n, const gx_map_spec *maps, uint32_t n_maps,
                   const gx_prog_opts &opts, VerifyOut &out);

/* translate a verified program to micro-ops (see gx_layout.h) */
int decode_program(const uint64_t *insns, uint32_t n, const VerifyOut &v, std::vector<uint64_t> &uops,
                   std::string &log);

} // namespace gx

#endif
