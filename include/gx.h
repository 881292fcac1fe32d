/*
 * gx -- a device-side eBPF execution engine for one GB300 GPU (sm_103a).
 *
 * The engine runs verified eBPF policy and observability programs over large batches
 * of device-resident event records, with array maps, lock-free hash maps and a ring
 * buffer kept in device memory.  It is the data-parallel core of the device-side eBPF
 * runtime of "gpu_ext: Extensible OS Policies for GPUs via eBPF" (arXiv 2512.12615):
 *   - device program type with a compact read-only context (Sec. 4.3, Sec. 4.3.1);
 *   - verification before execution: typed registers, bounded loops, memory safety,
 *     per-hook resource budgets (Sec. 4.4, Sec. 4.4.1, Sec. 5.3);
 *   - warp-level aggregated map updates (Sec. 4.4.2, and the hierarchical maps of Sec. 5.3);
 *   - maps as the shared key-value state, snapshotted at kernel completion (Sec. 4.4.3);
 *   - persistent workers claiming logical work units (Sec. 4.3.2, Sec. 5.3).
 * Instruction semantics follow the standard eBPF ISA (RFC 9669); map helpers use the
 * Linux UAPI helper numbers and return codes.
 *
 * Conventions for every entry point below:
 *   - return 0 on success or a negative status (GX_E*; errno values where one exists);
 *   - pointers named *_dev are device pointers owned by the caller and must stay valid
 *     until the work on `stream` completes; *_host pointers are host memory;
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream);
 *   - asynchronous calls only enqueue work; gx_last_status, gx_map_read and
 *     gx_ringbuf_drain synchronise `stream`;
 *   - device-side errors never trap: they are recorded in a sticky status word that
 *     gx_last_status returns;
 *   - objects are not thread-safe: one host thread drives a given context at a time
 *     (the server object below is the exception and documents its own rules).
 */
#ifndef GX_H
#define GX_H

#ifdef __CUDACC_RTC__ /* compiled by NVRTC as part of a load-time specialised program */
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef unsigned int uint32_t;
typedef unsigned long long uint64_t;
typedef signed char int8_t;
typedef short int16_t;
typedef int int32_t;
typedef long long int64_t;
typedef unsigned long long uintptr_t;
#else
#include <stddef.h>
#include <stdint.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define GX_OK 0
#define GX_ENOENT (-2)
#define GX_E2BIG (-7)
#define GX_EAGAIN (-11)
#define GX_ENOMEM (-12)
#define GX_EFAULT (-14)
#define GX_EEXIST (-17)
#define GX_EINVAL (-22)
#define GX_ENOSPC (-28)
#define GX_E_VERIFY (-1000)    /* program rejected by the verifier; see the log */
#define GX_E_CUDA (-1001)      /* a CUDA runtime call failed */
#define GX_E_BUDGET (-1002)    /* an event exceeded its dynamic instruction budget */
#define GX_E_TIMEOUT (-1003)   /* a bounded device wait gave up */
#define GX_E_DEVICE (-1004)    /* device-side invariant violated (sticky status) */
#define GX_E_ADMISSION (-1005) /* request larger than the server's memory budget */
#define GX_E_NODEV (-1006)     /* no CUDA device or wrong architecture */
#define GX_E_FAULT (-1007)     /* checked program: an access outside its regions was stopped */

/* ---------------------------------------------------------------- map types (Linux enum values) */
#define GX_MAP_HASH 1
#define GX_MAP_ARRAY 2
#define GX_MAP_RINGBUF 27

/* map update flags (Linux BPF_ANY / BPF_NOEXIST / BPF_EXIST) */
#define GX_ANY 0
#define GX_NOEXIST 1
#define GX_EXIST 2

/* helper ids usable in CALL instructions */
#define GX_HELPER_MAP_LOOKUP 1
#define GX_HELPER_MAP_UPDATE 2
#define GX_HELPER_MAP_DELETE 3
#define GX_HELPER_RINGBUF_OUTPUT 130
#define GX_HELPER_RINGBUF_RESERVE 131
#define GX_HELPER_RINGBUF_SUBMIT 132
#define GX_HELPER_RINGBUF_DISCARD 133
#define GX_HELPER_ATOMIC_MAX_U64 0x10000 /* void (u64 *p, u64 v): *p = max(*p, v) */
#define GX_HELPER_ATOMIC_MIN_U64 0x10001 /* void (u64 *p, u64 v): *p = min(*p, v) */
/*
 * Warp-level aggregation (Sec. 4.4.1: lane-varying values reach control flow or shared
 * state only through a warp-level reduction): u64 (u64 v) reduced over the warp's lanes,
 * the same result in every lane.  Accepted only by gx_verify_simt; the per-lane engine
 * (gx_verify / gx_verify_load) rejects them as unknown helpers.
 */
#define GX_HELPER_WARP_SUM_U64 0x10010 /* sum mod 2^64 */
#define GX_HELPER_WARP_MAX_U64 0x10011 /* unsigned maximum */
#define GX_HELPER_WARP_MIN_U64 0x10012 /* unsigned minimum */
#define GX_HELPER_WARP_OR_U64 0x10013
#define GX_HELPER_WARP_AND_U64 0x10014
#define GX_HELPER_WARP_COUNT 0x10015 /* number of lanes with v != 0 */

/* limits */
#define GX_MAX_INSNS 4096
#define GX_MAX_MAPS 16
#define GX_STACK_BYTES 512
#define GX_MAX_CTX 256
#define GX_MAX_KEY 64
#define GX_MAX_VALUE 4096

/*
 * Scheduling programs (gx_batch_set_sched; the `should_try_steal` hook over a block
 * context, Sec. 4.3.2).  The context is GX_SCHED_CTX bytes, little-endian, every field
 * warp-uniform: the block index, its SM, the chunks it has run, the chunks left in the
 * share it would take from, ns since the block started, and the batch's budget.
 */
#define GX_SCHED_CTX 32
#define GX_SCHED_OFF_BLOCK 0    /* u32 */
#define GX_SCHED_OFF_SM 4       /* u32 */
#define GX_SCHED_OFF_DONE 8     /* u32 */
#define GX_SCHED_OFF_LEFT 12    /* u32 */
#define GX_SCHED_OFF_ELAPSED 16 /* u64 */
#define GX_SCHED_OFF_BUDGET 24  /* u64 */
/* the hook budget a scheduling program is verified against unless the caller names one */
#define GX_SCHED_MAX_INSNS 64
#define GX_SCHED_MAX_HELPERS 2
#define GX_SCHED_MAX_MEM 16
/* per-block counters of a batch run with a scheduling program (gx_batch_sched_tally) */
#define GX_STEAL_OWNED 0   /* chunks of the block's own share it ran */
#define GX_STEAL_STOLEN 1  /* chunks of other shares it ran */
#define GX_STEAL_ASKED 2   /* times it ran the scheduling program */
#define GX_STEAL_GRANTED 3 /* times the program answered R0 != 0 */
#define GX_STEAL_WORDS 4

#ifndef __CUDACC_RTC__ /* device code sees the constants above only */
typedef struct gx_ctx gx_ctx;
typedef struct gx_map gx_map;
typedef struct gx_prog gx_prog;
typedef struct gx_batch gx_batch;
typedef struct gx_server gx_server;

/* ---------------------------------------------------------------- context */
/*
 * Open the engine on CUDA device `device`.  mem_budget: bytes of device memory the
 * engine's own allocations (maps, program images, scratch) may use; 0 = no limit.
 * Fails with GX_E_NODEV if the device is missing or not compute capability 10.3.
 */
int gx_init(int device, uint64_t mem_budget, gx_ctx **out);
/* Destroy the context; every map, program, batch and server made from it must be
 * destroyed first (GX_EINVAL otherwise).  Synchronises the device. */
int gx_shutdown(gx_ctx *ctx);
/* Bytes currently allocated by the engine on the device. */
uint64_t gx_mem_used(const gx_ctx *ctx);
/* Static text for a status code. */
const char *gx_strerror(int status);

/* ---------------------------------------------------------------- maps (Sec. 4.4.3) */
/*
 * Create a device-resident map.
 *   GX_MAP_ARRAY:   key_size must be 4 (u32 index); value_size 1..GX_MAX_VALUE;
 *                   max_entries >= 1; all values start at zero.
 *   GX_MAP_HASH:    key_size 1..GX_MAX_KEY, value_size 1..GX_MAX_VALUE; lock-free open
 *                   addressing over a power-of-two table of at least 2*max_entries slots;
 *                   at most max_entries live keys (further inserts return -E2BIG);
 *                   deleted slots are not reused until gx_map_clear.
 *   GX_MAP_RINGBUF: key_size = value_size = 0; max_entries = buffer bytes (power of two,
 *                   >= 4096).  Records are {u32 len; u32 flags; u64 event_idx} + payload
 *                   padded to 8 bytes; the buffer fills from offset 0 until drained.
 * flags: 0, or GX_MAP_F_NO_DELETE for a hash map whose keys are never removed: the
 *   verifier rejects map_delete_elem on it (gx_map_clear still empties it).  A published
 *   slot of such a map never changes, so specialised programs may read slots through
 *   the L1 cache; hot keys then stop converging on one L2 slice.
 * Memory is taken from the context budget (GX_ENOMEM when exceeded).
 */
#define GX_MAP_F_NO_DELETE 1u
int gx_map_create(gx_ctx *ctx, uint32_t type, uint32_t key_size, uint32_t value_size, uint32_t max_entries,
                  uint32_t flags, gx_map **out);
/* Drop the caller's reference; the map is freed once no program references it. */
int gx_map_destroy(gx_map *map);
/* Device bytes held by the map. */
uint64_t gx_map_bytes(const gx_map *map);

/*
 * Snapshot a map to host memory; synchronises `stream` (Sec. 4.4.3: snapshots at kernel
 * completion boundaries).
 *   array: max_entries * value_size bytes, entry i at offset i*value_size; *n_out = max_entries.
 *   hash:  packed {key, value} pairs (key_size + value_size bytes each), in unspecified
 *          order; *n_out = number of live pairs.  GX_E2BIG if cap_bytes is too small.
 *   ringbuf: not allowed (use gx_ringbuf_drain).
 */
int gx_map_read(gx_map *map, void *host_out, uint64_t cap_bytes, uint64_t *n_out, void *stream);
/*
 * Hash-map snapshot that allocates nothing.  The paper has no counterpart: this is for
 * callers that cannot call cudaMalloc, for example a control plane whose device-memory
 * budget is already used up, or a monitoring thread that must not add allocation (and
 * the device synchronisation cudaMalloc may bring) while the GPU serves requests.
 * gx_map_read compacts into a per-map scratch buffer that it allocates on first use;
 * this variant compacts into one fixed, file-scope device array of
 * GX_NOALLOC_SCRATCH_BYTES (256 bytes of counter + packed pairs) that every device
 * loading the library keeps until the process exits.  Same output format as
 * gx_map_read for hash maps; synchronises `stream`.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call before any
 *     stream capture.  The address is kept for the rest of the process: after a
 *     cudaDeviceReset of that device it is stale, so do not call this entry point again
 *     in a process that reset the device.
 *   - With lazy module loading (CUDA's default), the array itself is allocated when the
 *     library's device code is first loaded on a device, which may be this entry point's
 *     first call.  A caller that will have no memory to spare later should make one call
 *     early (any engine call that launches work on the device also loads it).
 *   - Every call shares the array and clears its counter: calls whose GPU work overlaps
 *     (other streams or host threads) race on it.
 *   - GX_EINVAL for array or ring-buffer maps.  GX_E2BIG, with *n_out = the live pair
 *     count and nothing copied, when the live pairs exceed the array
 *     ((GX_NOALLOC_SCRATCH_BYTES - 256) / (key_size + value_size) pairs) or cap_bytes.
 */
#define GX_NOALLOC_SCRATCH_BYTES (4u << 20)
int gx_map_read_noalloc(gx_map *map, void *host_out, uint64_t cap_bytes, uint64_t *n_out, void *stream);
/*
 * Restore a map from host memory (the inverse of gx_map_read); synchronises `stream`.
 *   array: exactly max_entries*value_size bytes, overwriting every value.
 *   hash:  packed {key, value} pairs, inserted or overwritten (BPF_ANY semantics);
 *          GX_E2BIG if the live count would exceed max_entries.
 */
int gx_map_write(gx_map *map, const void *host_in, uint64_t bytes, void *stream);
/* Reset to the empty state (zero values / no keys / empty ring, counters zeroed). Async. */
int gx_map_clear(gx_map *map, void *stream);
/*
 * Copy the committed ring-buffer records to host memory and empty the ring; synchronises
 * `stream`.  Discarded records are skipped; order is reservation order.  *bytes_out =
 * bytes written, *dropped = reservations refused for lack of space since the last drain.
 * GX_E2BIG (and nothing consumed) if cap is too small.
 */
int gx_ringbuf_drain(gx_map *rb, void *host_out, uint64_t cap, uint64_t *bytes_out, uint64_t *dropped,
                     void *stream);

/* ---------------------------------------------------------------- programs (Sec. 4.4, Sec. 5.3) */
typedef struct gx_map_spec {
    uint32_t type, key_size, value_size, max_entries;
    uint32_t flags;    /* GX_MAP_F_* as given to gx_map_create */
    uint32_t reserved; /* 0 */
} gx_map_spec;

typedef struct gx_prog_opts {
    uint32_t ctx_size;      /* bytes of one event record: multiple of 8 in [8, GX_MAX_CTX] */
    uint32_t deterministic; /* 1: also reject programs whose results could depend on event order */
    uint64_t insn_budget;   /* per-event limit on taken backward jumps; 0 = 1<<16 */
    uint32_t flags;         /* GX_PROG_* bits */
    uint32_t reserved;
} gx_prog_opts;

/*
 * opts.flags: GX_PROG_JIT runs the program as load-time specialised device code (one
 * CUDA function generated from the verified bytecode, compiled by NVRTC for sm_103a)
 * instead of through the interpreter kernel.  Results are identical; gx_verify_load
 * returns GX_E_NODEV if the runtime compiler is unavailable.
 */
#define GX_PROG_JIT 1u
/*
 * opts.flags: GX_PROG_CHECKED runs the program through a checked build of the
 * interpreter, which tests every memory access against the regions the event may touch
 * before making it: the record it reads (ctx, read-only), its 512-byte stack, the value
 * memory of the program's maps and the data of its ring buffers, with natural alignment;
 * and every helper's map index and buffer arguments.  An access that fails is not made:
 * the event stops with R0 = 0, the status becomes GX_E_FAULT and gx_run_stats.fault_pc
 * names the first failing micro-op.  It is the device-side stand-in for a memory checker,
 * for a program the verifier accepted: with a sound verifier nothing fails, and results
 * equal the unchecked tiers'.  The checked build runs every step in its divergent form,
 * so it is several times slower.  Not with GX_PROG_JIT (GX_EINVAL); plain launches only
 * (batches and servers refuse a checked program with GX_EINVAL).
 */
#define GX_PROG_CHECKED 2u

/*
 * Host only: verify a program and compile its specialised form to sm_103a code without
 * loading it (no device needed; NVRTC must be available).  0, GX_E_VERIFY, GX_E_NODEV
 * (no runtime compiler) or GX_E_CUDA (compile error); `log` explains.
 */
int gx_jit_check(const uint64_t *insns, uint32_t n_insns, const gx_map_spec *maps, uint32_t n_maps,
                 const gx_prog_opts *opts, char *log, size_t log_len);

/*
 * Verify `n_insns` raw eBPF slots (RFC 9669 encoding, little-endian) against map specs,
 * on the host only (no device needed).  Returns 0 if accepted, GX_E_VERIFY if rejected,
 * GX_EINVAL for bad arguments.  `log` (nullable) receives a NUL-terminated reason.
 * Map references are LD_IMM64 with src_reg = 1 and imm = index into `maps`.
 */
int gx_verify(const uint64_t *insns, uint32_t n_insns, const gx_map_spec *maps, uint32_t n_maps,
              const gx_prog_opts *opts, char *log, size_t log_len);
/*
 * What the verifier proved about an accepted program (host only, no device needed).
 * combinable_maps: bit m is set when the program changes map m's values only through
 * non-fetching commutative updates (BPF_ATOMIC ADD / OR / AND / XOR without FETCH, the
 * atomic max / min helpers) at constant offsets, one operation per 4-byte word, and never
 * loads, stores, exchanges or overwrites them or hands them to a helper.  Such updates
 * may be combined per thread block in shared memory before they reach device memory
 * (gx_launch.shards); the map's final contents are the same.  Returns as gx_verify.
 */
typedef struct gx_analysis {
    uint64_t insns_processed; /* instructions the verifier explored */
    uint32_t stack_depth;     /* deepest stack byte the program touches */
    uint32_t combinable_maps; /* bit m: see above */
} gx_analysis;
int gx_analyze(const uint64_t *insns, uint32_t n_insns, const gx_map_spec *maps, uint32_t n_maps,
               const gx_prog_opts *opts, gx_analysis *out, char *log, size_t log_len);
/*
 * SIMT-aware verification (host only, no device needed): the warp-uniformity pass and
 * per-hook resource budgets of Sec. 4.4.1 and Sec. 5.3, run together with the ordinary
 * checks of gx_verify.  The program is read as a warp-level handler: the lanes of a warp
 * run it in lockstep, each lane with its own ctx record, registers and stack, and shared
 * state changes once per warp.  A value is lane-varying when it derives from a ctx byte
 * that `uniform` does not mark (the role the paper gives BTF annotations), from a
 * lane-varying value, or from lane-varying stack bytes; constants, map handles, the ctx
 * and stack pointers, helper results and values loaded through a uniform pointer are
 * warp-uniform.  Rejected, with the instruction and a GX_SIMT_V_* reason:
 *   GX_SIMT_V_BRANCH  a conditional jump (so also a loop bound) on a lane-varying value;
 *   GX_SIMT_V_KEY     a lane-varying key for lookup, update or delete;
 *   GX_SIMT_V_ATOMIC  an atomic on map memory (BPF_ATOMIC or the max / min helpers) with a
 *                     lane-varying address or operand;
 *   GX_SIMT_V_STORE   a store into map or ring-buffer memory with a lane-varying address
 *                     or value;
 *   GX_SIMT_V_HELPER  another lane-varying helper argument (update value, ring-buffer
 *                     payload, flags);
 *   GX_SIMT_V_RET     a lane-varying R0 at exit (the decision broadcast to the lanes);
 *   GX_SIMT_V_INSNS / _HELPERS / _MEM  a path over the instruction, helper-call or
 *                     memory-operation budget;
 *   GX_SIMT_V_VERIFY  an ordinary verification failure (the log says which).
 * Lane-varying values reach these places only through GX_HELPER_WARP_* reductions.  The
 * helper set has no barrier or grid-wide synchronisation, and unknown helpers are refused.
 * Returns 0 if accepted, GX_E_VERIFY if rejected, GX_EINVAL for bad arguments; `out`
 * (nullable) is filled either way.
 */
typedef struct gx_simt_spec {
    const uint8_t *uniform;    /* opts->ctx_size flags, nonzero = warp-uniform ctx byte; NULL = none */
    uint32_t max_insns;        /* budget per path: instructions executed (a 64-bit immediate counts once);
                                  0 = unlimited */
    uint32_t max_helper_calls; /* budget per path: helper calls; 0 = unlimited */
    uint32_t max_mem_ops;      /* budget per path: loads, stores and atomics; 0 = unlimited */
    uint32_t reserved;         /* 0 */
} gx_simt_spec;
typedef struct gx_simt_report {
    uint64_t max_insns;        /* the most instructions on any path explored */
    uint32_t max_helper_calls; /* the most helper calls on any path */
    uint32_t max_mem_ops;      /* the most loads, stores and atomics on any path */
    uint32_t uniform_branches; /* conditional jumps with an open outcome, all on uniform values */
    uint32_t varying_insns;    /* instructions that compute a lane-varying value (lane-local work) */
    int32_t violation_pc;      /* the rejected instruction; -1 if accepted */
    uint32_t violation;        /* GX_SIMT_V_* */
} gx_simt_report;
#define GX_SIMT_V_NONE 0u
#define GX_SIMT_V_VERIFY 1u
#define GX_SIMT_V_BRANCH 2u
#define GX_SIMT_V_KEY 3u
#define GX_SIMT_V_ATOMIC 4u
#define GX_SIMT_V_STORE 5u
#define GX_SIMT_V_HELPER 6u
#define GX_SIMT_V_RET 7u
#define GX_SIMT_V_INSNS 8u
#define GX_SIMT_V_HELPERS 9u
#define GX_SIMT_V_MEM 10u
int gx_verify_simt(const uint64_t *insns, uint32_t n_insns, const gx_map_spec *maps, uint32_t n_maps,
                   const gx_prog_opts *opts, const gx_simt_spec *simt, gx_simt_report *out, char *log,
                   size_t log_len);
/*
 * Host only: SIMT-verify a program (as gx_verify_simt) and compile its warp-level form for
 * sm_103a without loading it (NVRTC must be available; no device needed).  In that form the
 * 32 lanes of a warp run the handler over 32 consecutive events; helper calls, and stores
 * and atomics outside the lane's stack, run on the warp's first valid lane with their
 * results broadcast; the warp helpers reduce over the valid lanes.  gx_verify_load_simt
 * loads it.  0, GX_E_VERIFY, GX_E_NODEV (no runtime compiler) or GX_E_CUDA (compile
 * error); `log` explains.
 */
int gx_jit_check_simt(const uint64_t *insns, uint32_t n_insns, const gx_map_spec *maps, uint32_t n_maps,
                      const gx_prog_opts *opts, const gx_simt_spec *simt, char *log, size_t log_len);
/*
 * Host only: compile, without loading it, the stealing kernel (both modes of
 * gx_batch_set_sched) of a batch whose one program (insns, maps, opts) runs under the
 * scheduling program (hook, hook_maps, hook_opts).  Both must verify; the hook must pass the
 * SIMT check within `limits` (nullable: the GX_SCHED_MAX_* budget) and have ctx_size
 * GX_SCHED_CTX.  0, GX_E_VERIFY, GX_EINVAL, GX_E_NODEV or GX_E_CUDA; `log` explains.
 */
int gx_jit_check_sched(const uint64_t *insns, uint32_t n_insns, const gx_map_spec *maps, uint32_t n_maps,
                       const gx_prog_opts *opts, const uint64_t *hook, uint32_t n_hook, const gx_map_spec *hook_maps,
                       uint32_t n_hook_maps, const gx_prog_opts *hook_opts, const gx_simt_spec *limits, char *log,
                       size_t log_len);
/*
 * SIMT-verify a program, compile its warp-level form (as gx_jit_check_simt) and load it.
 * opts->flags must be GX_PROG_JIT: the form exists only as specialised code.  A run of the
 * program treats each 32 consecutive events (from the batch's first) as one warp: the lanes
 * take one path, and shared state changes once per warp.  A batch or server that would run
 * it through the interpreter refuses it (GX_EINVAL).  This form has not yet run on a GPU.
 * Returns as gx_verify_load.
 */
int gx_verify_load_simt(gx_ctx *ctx, const uint64_t *insns, uint32_t n_insns, gx_map *const *maps, uint32_t n_maps,
                        const gx_prog_opts *opts, const gx_simt_spec *simt, gx_prog **out, char *log,
                        size_t log_len);

/*
 * Host only: how to merge copies of map `map_index` that several engines (one per GPU,
 * each with its own maps) built by running this program over disjoint parts of one batch
 * (Sec. 5.3: GPU-local map shards merged into a canonical snapshot).  The program is
 * verified in deterministic mode whatever opts->deterministic says: that mode is what makes
 * the merge exact.  word_ops (ceil(value_size / 4) entries) receives, per 4-byte word of a
 * value, the update that changes it: GX_MERGE_NONE (never changed) or GX_MERGE_ADD / _OR /
 * _AND / _XOR / _MAX / _MIN, with GX_MERGE_W8 set on both words of an 8-byte pair that a
 * 64-bit ADD, MAX or MIN updates (bitwise operations merge per 4-byte word at any width).  insert_value (value_size bytes, nullable) receives
 * the constant bytes a hash insert writes and *has_insert (nullable) whether the program
 * inserts into this map at all.  A word merges over the copies that hold the entry, with i
 * its starting value (the array's contents before the runs; insert_value for a new hash
 * key): ADD i + sum(v - i) and XOR i ^ xor(v ^ i), both modulo the width; OR, AND, MAX and
 * MIN (unsigned) are the operation over the copies.  Hash maps merge as the union of their
 * keys; ring buffers as the records of all copies ordered by event index (no ops needed).
 * Returns 0, GX_E_VERIFY (rejected in deterministic mode) or GX_EINVAL (bad arguments, or
 * copies that cannot be merged: inserts of different constants; `log` says which).  A
 * program that adds to the same bytes at two widths is rejected (GX_E_VERIFY).
 */
#define GX_MERGE_NONE 0u
#define GX_MERGE_ADD 1u
#define GX_MERGE_OR 2u
#define GX_MERGE_AND 3u
#define GX_MERGE_XOR 4u
#define GX_MERGE_MAX 5u
#define GX_MERGE_MIN 6u
#define GX_MERGE_W8 0x10u
int gx_merge_ops(const uint64_t *insns, uint32_t n_insns, const gx_map_spec *maps, uint32_t n_maps,
                 const gx_prog_opts *opts, uint32_t map_index, uint8_t *word_ops, uint8_t *insert_value,
                 uint32_t *has_insert, char *log, size_t log_len);

/* Verify, decode and upload a program; it holds a reference on each map. */
int gx_verify_load(gx_ctx *ctx, const uint64_t *insns, uint32_t n_insns, gx_map *const *maps, uint32_t n_maps,
                   const gx_prog_opts *opts, gx_prog **out, char *log, size_t log_len);
int gx_prog_destroy(gx_prog *prog);
/* Number of device micro-ops the program decoded to. */
uint32_t gx_prog_uops(const gx_prog *prog);

/* ---------------------------------------------------------------- runs */
typedef struct gx_launch {
    uint32_t block;  /* threads per block: 64..1024, multiple of 32; 0 = tuned/default */
    uint32_t ept;    /* events per thread: 1..64; 0 = tuned/default */
    uint32_t grid;   /* blocks: 0 = one wave (as many as the device holds at once; each block runs the
                        chunks of block * ept events b, b + grid, ...), GX_GRID_PER_CHUNK = one block per
                        chunk, else that many blocks (at most one per chunk); the tuner picks between
                        one wave and one block per chunk */
    uint32_t shards; /* map-sharding width of load-time specialised programs (GX_PROG_JIT): updates of
                        combinable maps (gx_analyze) are first combined in shared memory per block,
                        small array maps whole, other maps in a cache of 2^shards entries (2..10, capped
                        per map by its value size); GX_SHARDS_OFF sends every update to device memory
                        (warp-aggregated); 0 = tuned/default.  OR GX_SHARDS_AGG into a width (or into 0
                        for the default width) to warp-aggregate the updates that miss the cache, which
                        pays when hot values miss and costs a warp match on every miss.  Ignored by the
                        interpreter. */
    uint32_t variant; /* specialised programs: which compiled entry runs.  Each entry is compiled for a
                         number of resident 256-thread blocks per SM, which caps its registers per
                         thread: GX_VARIANT_WIDE 2 blocks (<= 128 registers), GX_VARIANT_CAPPED 5 (<= 48),
                         GX_VARIANT_3 3 (<= 80), GX_VARIANT_4 4 (<= 64).  Programs and batches have all
                         four (a batch steered by a scheduling program WIDE and CAPPED only).  0 =
                         tuned/default (GX_VARIANT_4 for a single program, CAPPED for a batch).  Ignored
                         by the interpreter. */
    uint32_t reserved;
} gx_launch;
#define GX_VARIANT_WIDE 1u
#define GX_VARIANT_CAPPED 2u
#define GX_VARIANT_3 3u
#define GX_VARIANT_4 4u
#define GX_GRID_PER_CHUNK 0xFFFFFFFFu
#define GX_SHARDS_OFF 255u
#define GX_SHARDS_AGG 0x100u

/*
 * Run the program once per event over n records at events_dev (n * ctx_size bytes,
 * 16-byte aligned), one event per thread, asynchronously on `stream`.  Maps keep their
 * state across runs.  Ring-buffer records get event_idx = index within this call.
 */
int gx_run_batch(gx_prog *prog, const void *events_dev, uint64_t n, void *stream);
/*
 * As gx_run_batch, plus: event_idx_base is added to ring-buffer event indices;
 * ret_out_dev (nullable) receives R0 of every event as int64; lp (nullable) fixes the
 * launch shape instead of the tuned one.
 */
int gx_run_batch_ex(gx_prog *prog, const void *events_dev, uint64_t n, uint64_t event_idx_base,
                    int64_t *ret_out_dev, const gx_launch *lp, void *stream);
/*
 * End-to-end form for host-resident events: copies events_host (pinned or pageable) to
 * the device in chunks on two internal streams overlapping copy and execution, runs the
 * program, and copies R0 back to ret_out_host (nullable).  Synchronous.
 */
int gx_run_batch_host(gx_prog *prog, const void *events_host, uint64_t n, int64_t *ret_out_host);

typedef struct gx_run_stats {
    int32_t status;         /* first device error (GX_E_BUDGET, GX_E_TIMEOUT, GX_E_DEVICE, GX_E_FAULT) or 0 */
    uint32_t fault_pc;      /* GX_PROG_CHECKED: 1 + the micro-op (instruction) index of the first stopped
                               access, 0 if none */
    uint64_t budget_trips;  /* events stopped by the instruction budget */
    uint64_t waits_expired; /* bounded device waits that gave up */
    uint64_t launches;      /* kernel launches issued for this program */
} gx_run_stats;
/* Synchronise `stream`, then report (and if reset != 0, clear) the program's status. */
int gx_last_status(gx_prog *prog, gx_run_stats *out, int reset, void *stream);

/*
 * Pick the launch for (prog, n) by timing candidates on a scratch copy of the program's
 * maps (the real maps, ring buffers included, are not touched): block size, events per
 * thread and, for specialised programs, the map-sharding width and miss policy
 * (gx_launch.shards) and the kernel variant.  Each candidate's time is the median of three
 * launches after an untimed one, over the first 64M events; the best three are then timed
 * again over all n events (the median of five) and the fastest is chosen.  The choice is
 * cached per program and size bucket and used by later runs, and its sharding choice is
 * the program's default in batches and served ticks; *best (nullable) gets it.
 * Synchronous; GX_EINVAL for n == 0 or a null events_dev.
 * With the environment variable GX_TUNE_CACHE naming a directory, each choice is also
 * written there, one file per program, map specs and options, size bucket, device and
 * engine build. A later call that finds a valid file uses it without timing anything.
 * Batch planning's per-program sharding choice is cached the same way.
 */
int gx_autotune(gx_prog *prog, const void *events_dev, uint64_t n, void *stream, gx_launch *best);

/* ---------------------------------------------------------------- batched form (Sec. 4.3.2, Sec. 5.3) */
/*
 * A batch is a fixed set of (program, events, n) items run by ONE persistent kernel:
 * blocks claim chunks of events from an atomic cursor, switch programs by restaging the
 * decoded program into shared memory, and the whole launch (cursor reset + kernel) is
 * captured once into a CUDA graph.  When every item's program is specialised, the kernel
 * holds all of them; each chunk carries its program's tuned map sharding (at most the
 * default width, so that one program does not cost all of them occupancy).
 */
int gx_batch_create(gx_ctx *ctx, gx_batch **out);
/* Add an item; ret_out_dev nullable.  Items may share programs and maps. */
int gx_batch_add(gx_batch *b, gx_prog *prog, const void *events_dev, uint64_t n, int64_t *ret_out_dev);
/* Build the chunk table and capture the graph; lp (nullable) fixes block/ept (else autotuned). */
int gx_batch_plan(gx_batch *b, const gx_launch *lp, void *stream);
/* Launch the captured graph on `stream` (async). */
int gx_batch_launch(gx_batch *b, void *stream);
int gx_batch_destroy(gx_batch *b);
/*
 * Steer the batch's blocks with a scheduling program, the `should_try_steal` hook of
 * Sec. 4.3.2 (policies such as FixedWork, Greedy and LatencyBudget, Sec. 6).  Call before
 * gx_batch_plan.  The chunk table is then cut into one contiguous share per block: a
 * block drains its own share, then, before each chunk it would take from another share,
 * runs `hook` once (one lane, warp 0) on a GX_SCHED_CTX-byte context (offsets
 * GX_SCHED_OFF_*, `budget_ns` in the budget field).  R0 != 0 takes the chunk; R0 == 0 ends
 * the block's work.  Every chunk still runs exactly once, whatever the program answers.
 * Ring-buffer records the program writes carry the block index as their event index.
 *
 * `hook` must be loaded with GX_PROG_JIT and ctx_size GX_SCHED_CTX, and it must be a
 * warp-uniform handler (gx_verify_simt with every ctx byte uniform) within `limits`
 * (nullable: GX_SCHED_MAX_INSNS / _HELPERS / _MEM; `limits->uniform` is ignored).  Every
 * item's program must be specialised too.  Its maps keep their state across launches
 * like any program's, and it must stay loaded while the batch exists (as the items'
 * programs must).  GX_EINVAL for a planned batch or a program that does not qualify,
 * GX_E_VERIFY if the SIMT check refuses it (`log` explains).
 */
int gx_batch_set_sched(gx_batch *b, gx_prog *hook, uint64_t budget_ns, const gx_simt_spec *limits, uint32_t flags,
                       char *log, size_t log_len);
/*
 * gx_batch_set_sched flags.  GX_SCHED_F_LAUNCH_CONTROL: instead of persistent blocks with
 * shares, launch one block per chunk; a block that has run its chunk asks `hook` and, on
 * R0 != 0, cancels a block that has not started yet (cluster launch control) and runs
 * that block's chunk.  The context's "left" field is the number of chunks not yet
 * started.  A cancelled block never runs, so every chunk still runs exactly once; a cancel
 * whose response does not come within the wait bound ends that block's stealing and sets
 * the scheduling program's status to GX_E_TIMEOUT (the chunk it may have cancelled is then
 * lost).  The block waits once more, bounded, for the response before it exits; should
 * that wait end too, the response may still land in the shared memory of a later block on
 * that SM.  So once gx_last_status of a scheduling program under launch control has
 * reported GX_E_TIMEOUT, launch control is refused on the context for good:
 * gx_batch_set_sched with this flag and gx_batch_launch of such a batch return
 * GX_E_TIMEOUT.  Tallies are per launched block; cancelled blocks' rows stay zero.
 */
#define GX_SCHED_F_LAUNCH_CONTROL 1u
/*
 * Synchronise `stream`, then copy the last launch's per-block counters (GX_STEAL_WORDS
 * u32 per block, indexed GX_STEAL_*) of a batch with a scheduling program to `out`
 * (`cap_blocks` blocks at most); *n_blocks gets the launch's block count.  GX_EINVAL
 * without a scheduling program or before gx_batch_plan; GX_ENOSPC if cap_blocks is short.
 */
int gx_batch_sched_tally(gx_batch *b, uint32_t *out, uint32_t cap_blocks, uint32_t *n_blocks, void *stream);

/* ---------------------------------------------------------------- served form */
typedef struct gx_server_opts {
    uint64_t mem_budget;   /* admission budget: resident map bytes + in-flight event bytes (0 = none) */
    uint32_t max_inflight; /* launches in flight, each on its own stream, 1..8 */
    uint32_t max_items;    /* requests per tick, 1..4096 */
    uint32_t block;        /* persistent kernel block size, 64..256 (0 = 256) */
    uint32_t ept;          /* events per thread per chunk (0 = 4) */
    uint32_t plain;        /* 1: no batching, one gx_run_batch launch per request (the baseline) */
    uint32_t n_progs;      /* programs registered up front (may be 0) */
    gx_prog *const *progs; /* if every one of them was loaded with GX_PROG_JIT, ticks run one
                              multi-program specialised kernel and only these programs are accepted */
} gx_server_opts;

typedef struct gx_completion {
    uint64_t tag;         /* caller's tag from gx_server_submit */
    int32_t status;       /* 0 or a GX_E* code */
    uint32_t reserved;
    double t_arrival;     /* seconds, steady clock: the request's (scheduled) arrival */
    double t_start;       /* when the launch that ran it was issued */
    double t_done;        /* when that launch was seen complete */
} gx_completion;

/*
 * Continuous-batching server over one device.  A host thread admits submitted requests
 * while (resident map bytes + event bytes of admitted, unfinished requests) stays within
 * mem_budget, packs admitted requests into the next tick's chunk table, and launches the
 * tick's captured graph (cursor reset + persistent kernel) on one of max_inflight
 * streams, so ticks overlap on the device.  Requests that arrive while ticks run join the
 * next tick as soon as a stream and memory are free.  Map state stays resident across
 * requests.  With opts.plain = 1 the same loop issues one plain launch per request
 * instead, which is the baseline the batched form is compared with.
 * submit/poll may be called from one host thread concurrently with the server thread.
 */
int gx_server_create(gx_ctx *ctx, const gx_server_opts *opts, gx_server **out);
/*
 * Enqueue a request (non-blocking).  t_arrival: its arrival time on the gx_now() clock
 * used for latency (0 = now).  GX_E_ADMISSION if it alone exceeds the budget.
 */
int gx_server_submit(gx_server *s, gx_prog *prog, const void *events_dev, uint64_t n, int64_t *ret_out_dev,
                     uint64_t tag, double t_arrival);

typedef struct gx_request {
    gx_prog *prog;
    const void *events_dev;
    uint64_t n;
    int64_t *ret_out_dev; /* nullable */
    uint64_t tag;
    double t_offset; /* seconds after the replay start */
} gx_request;
/*
 * Open-loop load generator: submit reqs[i] at t0 + reqs[i].t_offset (busy-waiting on the
 * calling thread), with that time as its arrival.  t0 = 0 means now.  Returns once every
 * request has been submitted; collect results with gx_server_poll.
 */
int gx_server_replay(gx_server *s, const gx_request *reqs, uint32_t n, double t0);
/* Collect up to cap completions; waits up to wait_ms for at least one (0 = no wait). */
int gx_server_poll(gx_server *s, gx_completion *out, uint32_t cap, uint32_t *n_out, int wait_ms);
/* Stop after finishing admitted work; frees the server. */
int gx_server_destroy(gx_server *s);
/* Steady-clock seconds, the time base of gx_completion. */
double gx_now(void);
#endif /* !__CUDACC_RTC__ */

#ifdef __cplusplus
}
#endif
#endif /* GX_H */
