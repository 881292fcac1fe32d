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

#include "../../include/gx.h"
#include "gx_kernels.h"
#include "gx_layout.h"

namespace gx {

typedef unsigned long long u64;
typedef long long s64;
typedef unsigned int u32;

#define FULLM 0xFFFFFFFFu
#define PC_DONE 0xFFFFFFFFu
#define WAIT_SPINS (1 << 20)

/* ------------------------------------------------------------------ small device utilities */
__device__ __forceinline__ u32 lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ u32 ld_acquire(const u32 *p) {
    u32 v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(u32 *p, u32 v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void set_status(u64 *stats, int code) {
    atomicCAS(&stats[GX_STAT_STATUS], 0ULL, (u64)(u32)code);
}

__device__ __forceinline__ u64 sx32(int32_t v) { return (u64)(s64)v; }

template <int SZ, bool SIGN>
__device__ __forceinline__ u64 load_sz(const void *p) {
    if (SZ == 1) return SIGN ? (u64)(s64) * (const int8_t *)p : (u64) * (const uint8_t *)p;
    if (SZ == 2) return SIGN ? (u64)(s64) * (const int16_t *)p : (u64) * (const uint16_t *)p;
    if (SZ == 4) return SIGN ? (u64)(s64) * (const int32_t *)p : (u64) * (const uint32_t *)p;
    return *(const u64 *)p;
}

template <int SZ>
__device__ __forceinline__ void store_sz(void *p, u64 v) {
    if (SZ == 1) *(uint8_t *)p = (uint8_t)v;
    else if (SZ == 2) *(uint16_t *)p = (uint16_t)v;
    else if (SZ == 4) *(uint32_t *)p = (uint32_t)v;
    else *(u64 *)p = v;
}

/* ------------------------------------------------------------------ ALU (RFC 9669 Sec. 4.1) */
enum { O_ADD, O_SUB, O_MUL, O_DIV, O_SDIV, O_MOD, O_SMOD, O_OR, O_AND, O_XOR, O_LSH, O_RSH, O_ARSH, O_MOV };

template <int O>
__device__ __forceinline__ u64 a64(u64 d, u64 s) {
    switch (O) {
    case O_ADD: return d + s;
    case O_SUB: return d - s;
    case O_MUL: return d * s;
    case O_DIV: return s ? d / s : 0;
    case O_SDIV: {
        s64 a = (s64)d, b = (s64)s;
        if (b == 0) return 0;
        if (b == -1) return (u64)0 - d; /* wraps INT64_MIN to itself */
        return (u64)(a / b);
    }
    case O_MOD: return s ? d % s : d;
    case O_SMOD: {
        s64 a = (s64)d, b = (s64)s;
        if (b == 0) return d;
        if (b == -1) return 0;
        return (u64)(a % b);
    }
    case O_OR: return d | s;
    case O_AND: return d & s;
    case O_XOR: return d ^ s;
    case O_LSH: return d << (s & 63);
    case O_RSH: return d >> (s & 63);
    case O_ARSH: return (u64)((s64)d >> (s & 63));
    default: return s; /* MOV */
    }
}

template <int O>
__device__ __forceinline__ u64 a32(u64 dd, u64 ss) {
    u32 d = (u32)dd, s = (u32)ss, r;
    switch (O) {
    case O_ADD: r = d + s; break;
    case O_SUB: r = d - s; break;
    case O_MUL: r = d * s; break;
    case O_DIV: r = s ? d / s : 0; break;
    case O_SDIV: {
        int a = (int)d, b = (int)s;
        r = b == 0 ? 0u : b == -1 ? 0u - d : (u32)(a / b);
        break;
    }
    case O_MOD: r = s ? d % s : d; break;
    case O_SMOD: {
        int a = (int)d, b = (int)s;
        r = b == 0 ? d : b == -1 ? 0u : (u32)(a % b);
        break;
    }
    case O_OR: r = d | s; break;
    case O_AND: r = d & s; break;
    case O_XOR: r = d ^ s; break;
    case O_LSH: r = d << (s & 31); break;
    case O_RSH: r = d >> (s & 31); break;
    case O_ARSH: r = (u32)((int)d >> (s & 31)); break;
    default: r = s; break;
    }
    return (u64)r;
}

enum { C_EQ, C_GT, C_GE, C_SET, C_NE, C_SGT, C_SGE, C_LT, C_LE, C_SLT, C_SLE };

template <int C>
__device__ __forceinline__ bool c64(u64 a, u64 b) {
    switch (C) {
    case C_EQ: return a == b;
    case C_GT: return a > b;
    case C_GE: return a >= b;
    case C_SET: return (a & b) != 0;
    case C_NE: return a != b;
    case C_SGT: return (s64)a > (s64)b;
    case C_SGE: return (s64)a >= (s64)b;
    case C_LT: return a < b;
    case C_LE: return a <= b;
    case C_SLT: return (s64)a < (s64)b;
    default: return (s64)a <= (s64)b;
    }
}

template <int C>
__device__ __forceinline__ bool c32(u64 aa, u64 bb) {
    u32 a = (u32)aa, b = (u32)bb;
    switch (C) {
    case C_EQ: return a == b;
    case C_GT: return a > b;
    case C_GE: return a >= b;
    case C_SET: return (a & b) != 0;
    case C_NE: return a != b;
    case C_SGT: return (int)a > (int)b;
    case C_SGE: return (int)a >= (int)b;
    case C_LT: return a < b;
    case C_LE: return a <= b;
    case C_SLT: return (int)a < (int)b;
    default: return (int)a <= (int)b;
    }
}

/* ------------------------------------------------------------------ warp-aggregated atomics */
enum { AG_ADD, AG_OR, AG_AND, AG_XOR, AG_MAX, AG_MIN };

/* reduce v over the lanes of `grp` (each lane passes its own group's mask) */
template <int OP, int SZ>
__device__ __forceinline__ u64 group_reduce(u32 grp, u64 v) {
    if (SZ == 4) {
        u32 x = (u32)v;
        if (OP == AG_ADD) return __reduce_add_sync(grp, x);
        if (OP == AG_OR) return __reduce_or_sync(grp, x);
        if (OP == AG_AND) return __reduce_and_sync(grp, x);
        return __reduce_xor_sync(grp, x);
    }
    if (OP == AG_ADD) { /* three limbs of at most 22 bits: 32 lanes cannot carry out of a u32 */
        u32 l0 = (u32)(v & 0x3FFFFFu), l1 = (u32)((v >> 22) & 0x1FFFFFu), l2 = (u32)(v >> 43);
        u64 s0 = __reduce_add_sync(grp, l0), s1 = __reduce_add_sync(grp, l1), s2 = __reduce_add_sync(grp, l2);
        return s0 + (s1 << 22) + (s2 << 43);
    }
    u32 lo = (u32)v, hi = (u32)(v >> 32);
    if (OP == AG_OR) return (u64)__reduce_or_sync(grp, lo) | ((u64)__reduce_or_sync(grp, hi) << 32);
    if (OP == AG_AND) return (u64)__reduce_and_sync(grp, lo) | ((u64)__reduce_and_sync(grp, hi) << 32);
    if (OP == AG_XOR) return (u64)__reduce_xor_sync(grp, lo) | ((u64)__reduce_xor_sync(grp, hi) << 32);
    if (OP == AG_MAX) {
        u32 h = __reduce_max_sync(grp, hi);
        u32 l = __reduce_max_sync(grp, hi == h ? lo : 0u);
        return ((u64)h << 32) | l;
    }
    u32 h = __reduce_min_sync(grp, hi);
    u32 l = __reduce_min_sync(grp, hi == h ? lo : 0xFFFFFFFFu);
    return ((u64)h << 32) | l;
}

template <int OP, int SZ>
__device__ __forceinline__ void plain_atomic(void *p, u64 v) {
    if (SZ == 4) {
        u32 *q = (u32 *)p;
        if (OP == AG_ADD) atomicAdd(q, (u32)v);
        else if (OP == AG_OR) atomicOr(q, (u32)v);
        else if (OP == AG_AND) atomicAnd(q, (u32)v);
        else atomicXor(q, (u32)v);
    } else {
        u64 *q = (u64 *)p;
        if (OP == AG_ADD) atomicAdd(q, v);
        else if (OP == AG_OR) atomicOr(q, v);
        else if (OP == AG_AND) atomicAnd(q, v);
        else if (OP == AG_XOR) atomicXor(q, v);
        else if (OP == AG_MAX) atomicMax(q, v);
        else atomicMin(q, v);
    }
}

template <int OP, int SZ>
__device__ __forceinline__ u64 local_rmw(void *p, u64 v) {
    u64 old = load_sz<SZ, false>(p), r;
    if (OP == AG_ADD) r = old + v;
    else if (OP == AG_OR) r = old | v;
    else if (OP == AG_AND) r = old & v;
    else if (OP == AG_XOR) r = old ^ v;
    else if (OP == AG_MAX) r = v > old ? v : old;
    else r = v < old ? v : old;
    store_sz<SZ>(p, r);
    return old;
}

/* non-fetching update of `p` by the executing lanes `exec` */
template <int OP, int SZ>
__device__ __forceinline__ void agg_update(u64 addr, u64 v, u32 exec) {
    if (__isLocal((const void *)addr)) { /* the eBPF stack: private, plain read-modify-write */
        local_rmw<OP, SZ>((void *)addr, v);
        return;
    }
    u32 grp = __match_any_sync(exec, addr);
    u64 agg = group_reduce<OP, SZ>(grp, v);
    if (lane_id() == (u32)(__ffs(grp) - 1)) plain_atomic<OP, SZ>((void *)addr, agg);
}

template <int OP, int SZ>
__device__ __forceinline__ u64 fetch_update(u64 addr, u64 v) {
    if (__isLocal((const void *)addr)) return local_rmw<OP, SZ>((void *)addr, v);
    if (SZ == 4) {
        u32 *q = (u32 *)addr;
        if (OP == AG_ADD) return atomicAdd(q, (u32)v);
        if (OP == AG_OR) return atomicOr(q, (u32)v);
        if (OP == AG_AND) return atomicAnd(q, (u32)v);
        return atomicXor(q, (u32)v);
    }
    u64 *q = (u64 *)addr;
    if (OP == AG_ADD) return atomicAdd(q, v);
    if (OP == AG_OR) return atomicOr(q, v);
    if (OP == AG_AND) return atomicAnd(q, v);
    return atomicXor(q, v);
}

template <int SZ>
__device__ __forceinline__ u64 xchg(u64 addr, u64 v) {
    if (__isLocal((const void *)addr)) {
        u64 old = load_sz<SZ, false>((void *)addr);
        store_sz<SZ>((void *)addr, v);
        return old;
    }
    if (SZ == 4) return atomicExch((u32 *)addr, (u32)v);
    return atomicExch((u64 *)addr, v);
}

template <int SZ>
__device__ __forceinline__ u64 cmpxchg(u64 addr, u64 expect, u64 v) {
    if (__isLocal((const void *)addr)) {
        u64 old = load_sz<SZ, false>((void *)addr);
        if (old == (SZ == 4 ? (expect & 0xFFFFFFFFull) : expect)) store_sz<SZ>((void *)addr, v);
        return old;
    }
    if (SZ == 4) return atomicCAS((u32 *)addr, (u32)expect, (u32)v);
    return atomicCAS((u64 *)addr, expect, v);
}

/* ------------------------------------------------------------------ hash map (lock-free) */
__device__ __forceinline__ u64 mix64(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* key bytes -> words; keys up to 8 bytes come back in k0 (zero-padded) */
__device__ __forceinline__ u64 key_word(const uint8_t *k, u32 ks, u32 w) {
    u32 lo = w * 8, n = ks - lo < 8 ? ks - lo : 8;
    if (n == 8 && (((u64)k & 7) == 0)) return *(const u64 *)(k + lo);
    if (n == 4 && (((u64)(k + lo) & 3) == 0)) return *(const u32 *)(k + lo);
    u64 v = 0;
    for (u32 i = 0; i < n; i++) v |= (u64)k[lo + i] << (8 * i);
    return v;
}

__device__ __forceinline__ u64 hash_key(const uint8_t *k, u32 ks) {
    u64 h = 0x9E3779B97F4A7C15ull ^ ks;
    for (u32 w = 0; w * 8 < ks; w++) h = mix64(h ^ key_word(k, ks, w));
    return h;
}

__device__ __forceinline__ bool slot_key_eq(const uint8_t *slot, const uint8_t *k, u32 ks) {
    const u64 *sk = (const u64 *)(slot + 8);
    for (u32 w = 0; w * 8 < ks; w++)
        if (sk[w] != key_word(k, ks, w)) return false;
    return true;
}

__device__ u32 wait_published(u32 *st, u64 *stats) {
    for (int it = 0; it < WAIT_SPINS; it++) {
        u32 s = ld_acquire(st);
        if (s != GX_SLOT_BUSY) return s;
        __nanosleep(32);
    }
    atomicAdd(&stats[GX_STAT_WAITS], 1ull);
    set_status(stats, GX_E_TIMEOUT);
    return GX_SLOT_BUSY;
}

/* pointer to the value of key k, or 0 */
__device__ u64 hash_find(const gx_dmap &m, const uint8_t *k, u64 *stats) {
    u64 i = hash_key(k, m.key_size) & m.mask;
    for (u64 probes = 0; probes <= m.mask; probes++, i = (i + 1) & m.mask) {
        uint8_t *slot = m.slots + i * m.sstride;
        u32 s = ld_acquire((u32 *)slot);
        if (s == GX_SLOT_EMPTY) return 0;
        if (s == GX_SLOT_BUSY) {
            s = wait_published((u32 *)slot, stats);
            if (s == GX_SLOT_BUSY) return 0;
        }
        if (s == GX_SLOT_FULL && slot_key_eq(slot, k, m.key_size)) return (u64)(m.values + i * m.vstride);
    }
    return 0;
}

__device__ __forceinline__ void copy_bytes(uint8_t *dst, const uint8_t *src, u32 n) {
    if ((((u64)dst | (u64)src | n) & 7) == 0) {
        for (u32 i = 0; i < n; i += 8) *(u64 *)(dst + i) = *(const u64 *)(src + i);
    } else if ((((u64)dst | (u64)src | n) & 3) == 0) {
        for (u32 i = 0; i < n; i += 4) *(u32 *)(dst + i) = *(const u32 *)(src + i);
    } else {
        for (u32 i = 0; i < n; i++) dst[i] = src[i];
    }
}

/* insert or overwrite; returns 0 / -EEXIST / -ENOENT / -E2BIG (Linux update semantics) */
__device__ int hash_update(const gx_dmap &m, const uint8_t *k, const uint8_t *v, u64 flags, u64 *stats) {
    u64 i = hash_key(k, m.key_size) & m.mask;
    for (u64 probes = 0; probes <= m.mask;) {
        uint8_t *slot = m.slots + i * m.sstride;
        u32 *st = (u32 *)slot;
        u32 s = ld_acquire(st);
        if (s == GX_SLOT_EMPTY) {
            if (flags == GX_EXIST) return GX_ENOENT;
            if (atomicCAS(st, GX_SLOT_EMPTY, GX_SLOT_BUSY) != GX_SLOT_EMPTY) continue; /* lost the race: look again */
            if (atomicAdd(&m.ctr[0], 1ull) >= m.max_entries) {
                atomicAdd(&m.ctr[0], ~0ull);
                atomicAdd(&m.ctr[1], 1ull);
                st_release(st, GX_SLOT_TOMB);
                return GX_E2BIG;
            }
            u64 *sk = (u64 *)(slot + 8);
            for (u32 w = 0; w * 8 < m.key_size; w++) sk[w] = key_word(k, m.key_size, w);
            copy_bytes(m.values + i * m.vstride, v, m.value_size);
            __threadfence();
            st_release(st, GX_SLOT_FULL);
            return 0;
        }
        if (s == GX_SLOT_BUSY) {
            if (wait_published(st, stats) == GX_SLOT_BUSY) return GX_E2BIG;
            continue;
        }
        if (s == GX_SLOT_FULL && slot_key_eq(slot, k, m.key_size)) {
            if (flags == GX_NOEXIST) return GX_EEXIST;
            copy_bytes(m.values + i * m.vstride, v, m.value_size);
            return 0;
        }
        probes++;
        i = (i + 1) & m.mask;
    }
    atomicAdd(&m.ctr[1], 1ull);
    return GX_E2BIG;
}

__device__ int hash_delete(const gx_dmap &m, const uint8_t *k, u64 *stats) {
    u64 i = hash_key(k, m.key_size) & m.mask;
    for (u64 probes = 0; probes <= m.mask; probes++, i = (i + 1) & m.mask) {
        uint8_t *slot = m.slots + i * m.sstride;
        u32 *st = (u32 *)slot;
        u32 s = ld_acquire(st);
        if (s == GX_SLOT_EMPTY) return GX_ENOENT;
        if (s == GX_SLOT_BUSY) s = wait_published(st, stats);
        if (s == GX_SLOT_FULL && slot_key_eq(slot, k, m.key_size)) {
            if (atomicCAS(st, GX_SLOT_FULL, GX_SLOT_TOMB) == GX_SLOT_FULL) {
                atomicAdd(&m.ctr[0], ~0ull);
                return 0;
            }
            return GX_ENOENT; /* somebody else deleted it first */
        }
    }
    return GX_ENOENT;
}

/* lookup with lanes that look up the same (<= 8 byte) key sharing one probe */
__device__ __noinline__ u64 map_lookup(const gx_dmap &m, const uint8_t *k, u32 exec, u64 *stats) {
    if (m.type == GX_MAP_ARRAY) {
        u32 key = *(const u32 *)k;
        return key < m.max_entries ? (u64)(m.values + (u64)key * m.vstride) : 0;
    }
    if (m.key_size <= 8) {
        u64 kw = key_word(k, m.key_size, 0);
        u32 grp = __match_any_sync(exec, kw);
        int leader = __ffs(grp) - 1;
        u64 r = 0;
        if ((int)lane_id() == leader) r = hash_find(m, k, stats);
        return __shfl_sync(grp, r, leader);
    }
    return hash_find(m, k, stats);
}

__device__ __noinline__ int map_update(const gx_dmap &m, const uint8_t *k, const uint8_t *v, u64 flags, u32 exec,
                                          u64 *stats) {
    if (flags > GX_EXIST) return GX_EINVAL;
    if (m.type == GX_MAP_ARRAY) {
        u32 key = *(const u32 *)k;
        if (key >= m.max_entries) return GX_E2BIG;
        if (flags == GX_NOEXIST) return GX_EEXIST;
        copy_bytes(m.values + (u64)key * m.vstride, v, m.value_size);
        return 0;
    }
    if (m.key_size <= 8 && flags == GX_NOEXIST) {
        /* one insert per distinct key in the warp; the others see the key present */
        u64 kw = key_word(k, m.key_size, 0);
        u32 grp = __match_any_sync(exec, kw);
        int leader = __ffs(grp) - 1;
        int r = 0;
        if ((int)lane_id() == leader) r = hash_update(m, k, v, flags, stats);
        r = __shfl_sync(grp, r, leader);
        if ((int)lane_id() != leader && r == 0) r = GX_EEXIST;
        return r;
    }
    return hash_update(m, k, v, flags, stats);
}

/* ------------------------------------------------------------------ ring buffer */
/* reserve `size` payload bytes for every lane of exec; returns payload pointer or 0 */
__device__ __noinline__ u64 rb_reserve(const gx_dmap &m, u64 size, u32 exec, u64 ev_idx) {
    u32 rec = GX_RB_HDR + (u32)((size + 7) & ~7ull);
    u32 lane = lane_id();
    u32 below = exec & ((1u << lane) - 1u);
    u32 prefix;
    int same_size;
    if (__match_all_sync(exec, rec, &same_size) != 0) {
        prefix = (u32)__popc(below) * rec;
    } else {
        prefix = 0;
        u32 bits = exec;
        while (bits) {
            int l = __ffs(bits) - 1;
            bits &= bits - 1;
            u32 r = __shfl_sync(exec, rec, l);
            if ((u32)l < lane) prefix += r;
        }
    }
    u32 total = __reduce_add_sync(exec, rec);
    int leader = __ffs(exec) - 1;
    u64 base = 0;
    if ((int)lane == leader) base = atomicAdd(&m.ctr[0], (u64)total);
    base = __shfl_sync(exec, base, leader);
    u64 off = base + prefix, cap = m.mask;
    if (off + rec > cap) {
        atomicAdd(&m.ctr[1], 1ull);
        if (off < cap && off + GX_RB_HDR <= cap) { /* first failed record marks the end of the data */
            u32 *h = (u32 *)(m.values + off);
            h[0] = (u32)(cap - off - GX_RB_HDR);
            h[1] = GX_RB_PAD;
        }
        return 0;
    }
    uint8_t *p = m.values + off;
    u32 *h = (u32 *)p;
    h[0] = (u32)size;
    h[1] = 0;
    *(u64 *)(p + 8) = ev_idx;
    for (u32 i = GX_RB_HDR; i < rec; i += 8) *(u64 *)(p + i) = 0;
    return (u64)(p + GX_RB_HDR);
}

/* ------------------------------------------------------------------ the interpreter */
struct ExecEnv {
    const u64 *uops;
    const gx_dmap *maps;
    u64 *stats;
    u64 budget;
};

/* handler-case generators: one case per eBPF register */
#define RC10(FAM, M, A, B)                                                                  \
    case (FAM)*16 + 0: { M(r0, A, B) } break;                                               \
    case (FAM)*16 + 1: { M(r1, A, B) } break;                                               \
    case (FAM)*16 + 2: { M(r2, A, B) } break;                                               \
    case (FAM)*16 + 3: { M(r3, A, B) } break;                                               \
    case (FAM)*16 + 4: { M(r4, A, B) } break;                                               \
    case (FAM)*16 + 5: { M(r5, A, B) } break;                                               \
    case (FAM)*16 + 6: { M(r6, A, B) } break;                                               \
    case (FAM)*16 + 7: { M(r7, A, B) } break;                                               \
    case (FAM)*16 + 8: { M(r8, A, B) } break;                                               \
    case (FAM)*16 + 9: { M(r9, A, B) } break;
#define RC11(FAM, M, A, B) RC10(FAM, M, A, B) case (FAM)*16 + 10: { M(r10, A, B) } break;

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

/* ctx word w of this lane lives at ctxw[w * 32 + lane]; AUX is the byte offset */
#define CTX_PTR ((const uint8_t *)(ctxw + ((AUX >> 3) << 5) + lane) + (AUX & 7))
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
/* stage `bytes` (multiple of 16) from global to shared memory with cp.async */
__device__ __forceinline__ void stage_image(uint8_t *dst, const uint8_t *src, u32 bytes) {
    for (u32 o = threadIdx.x * 16u; o < bytes; o += blockDim.x * 16u) {
        u32 sa = (u32)__cvta_generic_to_shared(dst + o);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(src + o) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
}

/* the warp's next 32 records -> transposed shared tile ctxw[word * 32 + record] */
__device__ __forceinline__ void load_ctx_tile(u64 *ctxw, const uint8_t *events, u64 first, u64 n, u32 cw) {
    const u32 lane = lane_id();
    const u64 nrec = n > first ? (n - first < 32 ? n - first : 32) : 0;
    const u32 chunks = cw * 16; /* 16-byte chunks in a full tile */
    const ulonglong2 *src = (const ulonglong2 *)(events + first * (u64)cw * 8);
    for (u32 c = lane; c < chunks; c += 32) {
        u32 word = 2 * c, rec = word / cw;
        if (rec < nrec) {
            ulonglong2 v = __ldcs(src + c);
            u32 f = word % cw;
            ctxw[f * 32 + rec] = v.x;
            ctxw[(f + 1) * 32 + rec] = v.y;
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(256, 3) gx_exec_kernel(ExecParams P) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ u32 s_chunk;
    __shared__ const uint8_t *s_image;
    const u32 warp = threadIdx.x >> 5, lane = lane_id();
    const u32 warps = blockDim.x >> 5;
    u64 *ctx_all = (u64 *)(smem + P.image_area);
    if (P.mode == 0) {
        stage_image(smem, P.image, P.image_bytes);
        const gx_dprog_hdr *hdr = (const gx_dprog_hdr *)smem;
        ExecEnv env;
        env.maps = (const gx_dmap *)(smem + sizeof(gx_dprog_hdr));
        env.uops = (const u64 *)(smem + sizeof(gx_dprog_hdr) + hdr->n_maps * sizeof(gx_dmap));
        env.stats = hdr->stats;
        env.budget = hdr->budget;
        const u32 cw = P.ctx_size / 8;
        u64 *ctxw = ctx_all + warp * cw * 32;
        const u64 tile0 = (u64)blockIdx.x * blockDim.x * P.ept;
        for (u32 e = 0; e < P.ept; e++) {
            const u64 first = tile0 + (u64)e * blockDim.x + warp * 32;
            if (first >= P.n) break; /* warp-uniform */
            load_ctx_tile(ctxw, P.events, first, P.n, cw);
            const u64 idx = first + lane;
            const bool valid = idx < P.n;
            u64 r0 = interp(env, ctxw, valid, P.idx_base + idx);
            if (valid && P.ret_out) P.ret_out[idx] = (long long)r0;
            __syncwarp();
        }
        return;
    }
    /* persistent mode: claim chunks until the table is exhausted */
    const u32 nchunks = P.nchunks_dev ? *P.nchunks_dev : P.nchunks;
    if (threadIdx.x == 0) s_image = nullptr;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_chunk = atomicAdd(P.cursor, 1u);
        __syncthreads();
        const u32 c = s_chunk;
        if (c >= nchunks) break;
        const gx_chunk ch = P.chunks[c];
        if (ch.image != s_image) {
            stage_image(smem, ch.image, ch.image_bytes);
            if (threadIdx.x == 0) s_image = ch.image;
        }
        const gx_dprog_hdr *hdr = (const gx_dprog_hdr *)smem;
        ExecEnv env;
        env.maps = (const gx_dmap *)(smem + sizeof(gx_dprog_hdr));
        env.uops = (const u64 *)(smem + sizeof(gx_dprog_hdr) + hdr->n_maps * sizeof(gx_dmap));
        env.stats = hdr->stats;
        env.budget = hdr->budget;
        const u32 cw = ch.ctx_size / 8;
        u64 *ctxw = ctx_all + warp * cw * 32;
        for (u64 first = ch.begin + (u64)warp * 32; first < ch.end; first += (u64)warps * 32) {
            load_ctx_tile(ctxw, ch.events, first, ch.end, cw);
            const u64 idx = first + lane;
            const bool valid = idx < ch.end;
            u64 r0 = interp(env, ctxw, valid, ch.idx_base + idx);
            if (valid && ch.ret_out) ch.ret_out[idx] = (long long)r0;
            __syncwarp();
        }
    }
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
