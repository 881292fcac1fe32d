/*
 * Device-side runtime shared by the interpreter kernel (interp.cu) and by programs
 * compiled at load time (jit.cpp hands this header to NVRTC): ALU semantics
 * (RFC 9669 Sec. 4.1 / 4.3), warp-aggregated map-value atomics (the per-warp leader
 * update of Sec. 4.4.2), the lock-free hash map, the ring buffer and the event-tile
 * staging.  Every wait on another lane is bounded.
 */
#ifndef GX_DEVICE_CUH
#define GX_DEVICE_CUH

#include "gx.h"
#include "gx_layout.h"

namespace gx {

typedef unsigned long long u64;
typedef long long s64;
typedef unsigned int u32;

#define FULLM 0xFFFFFFFFu
#define PC_DONE 0xFFFFFFFFu
#define WAIT_SPINS (1 << 20)

typedef gx_exec_params ExecParams;

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

/*
 * Division and modulo by a register, out of line: a long instruction sequence that every
 * site would otherwise carry.  By a constant they stay inline (a64 / a32), where the
 * compiler turns them into multiplications.
 */
template <int O>
__device__ __noinline__ u64 a64_call(u64 d, u64 s) {
    return a64<O>(d, s);
}
template <int O>
__device__ __noinline__ u64 a32_call(u64 d, u64 s) {
    return a32<O>(d, s);
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

/*
 * An update that goes to device memory, out of line: specialised programs with many update
 * sites call it from each site whose block-private combining is off or missed, so a site
 * carries a call instead of its own copy of the aggregation code (code size is what the
 * instruction cache of a long program pays for).  agg: warp-aggregate the lanes that call
 * together, else one atomic per lane.
 */
template <int OP, int SZ>
__device__ __noinline__ void dev_update(u64 addr, u64 v, u32 agg) {
    if (agg) agg_update<OP, SZ>(addr, v, __activemask());
    else plain_atomic<OP, SZ>((void *)addr, v);
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

/*
 * Per-lane lookup of a key of KS <= 8 bytes (KS in 1, 2, 4, 8), given as its zero-padded
 * little-endian word, in a hash map whose slots are 16 bytes and values VS bytes apart:
 * the form specialised programs inline.  No warp collectives.
 */
template <int KS, int VS>
__device__ __forceinline__ u64 hash_find_word(const gx_dmap &m, u64 kw, u64 *stats) {
    const u64 mask = m.mask;
    u64 i = mix64(0x9E3779B97F4A7C15ull ^ (u64)KS ^ kw) & mask;
    for (u64 probes = 0; probes <= mask; probes++, i = (i + 1) & mask) {
        const uint8_t *slot = m.slots + i * 16u;
        u32 s = ld_acquire((const u32 *)slot);
        if (s == GX_SLOT_EMPTY) return 0;
        if (s == GX_SLOT_BUSY) {
            s = wait_published((u32 *)slot, stats);
            if (s == GX_SLOT_BUSY) return 0;
        }
        if (s == GX_SLOT_FULL && *(const u64 *)(slot + 8) == kw) return (u64)(m.values + i * (u64)VS);
    }
    return 0;
}

/*
 * The same lookup for a map whose keys are never deleted (GX_MAP_F_NO_DELETE).  A slot's
 * key word is written once, before the slot is published as FULL, and a FULL slot never
 * changes again; so a plain (L1-cached) read of {state, key} that shows FULL and the
 * searched non-zero key is the final truth, and hot keys are served from L1 instead of
 * one L2 slice.  Anything else (a stale or empty line, another key, key 0) takes the
 * ordered probe above.
 */
template <int KS, int VS>
__device__ __noinline__ u64 hash_find_word_probe(const gx_dmap &m, u64 kw, u64 *stats) {
    return hash_find_word<KS, VS>(m, kw, stats);
}

/* OUTLINE: the ordered probe out of line (programs with many lookup sites) */
template <int KS, int VS, bool OUTLINE = false>
__device__ __forceinline__ u64 hash_find_word_nd(const gx_dmap &m, u64 kw, u64 *stats) {
    const u64 i = mix64(0x9E3779B97F4A7C15ull ^ (u64)KS ^ kw) & m.mask;
    const ulonglong2 v = *(const ulonglong2 *)(m.slots + i * 16u);
    if ((u32)v.x == GX_SLOT_FULL && v.y == kw && kw != 0) return (u64)(m.values + i * (u64)VS);
    return OUTLINE ? hash_find_word_probe<KS, VS>(m, kw, stats) : hash_find_word<KS, VS>(m, kw, stats);
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

/* ------------------------------------------------------------------ event tiles */
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

/* the warp's next 32 records -> transposed shared tile ctxw[word * GX_CTX_ROW(cw) + record] */
__device__ __forceinline__ void load_ctx_tile(u64 *ctxw, const uint8_t *events, u64 first, u64 n, u32 cw) {
    const u32 row = GX_CTX_ROW(cw);
    const u32 lane = lane_id();
    const u64 nrec = n > first ? (n - first < 32 ? n - first : 32) : 0;
    const u32 chunks = cw * 16; /* 16-byte chunks in a full tile */
    const ulonglong2 *src = (const ulonglong2 *)(events + first * (u64)cw * 8);
    for (u32 c = lane; c < chunks; c += 32) {
        u32 word = 2 * c, rec = word / cw;
        if (rec < nrec) {
            ulonglong2 v = __ldcs(src + c);
            u32 f = word % cw;
            ctxw[f * row + rec] = v.x;
            ctxw[(f + 1) * row + rec] = v.y;
        }
    }
    __syncwarp();
}

/*
 * A warp's tile in flight, for records of CW = 4 or 8 words: its 32 * CW * 8 bytes as
 * 16-byte chunks, CW / 2 per lane, held in registers.  tile_fetch issues every load of a
 * tile at once (the loads of the next tile go out before the current tile runs, so
 * streaming overlaps execution); tile_store transposes the chunks into the shared tile.
 */
template <u32 CW>
struct Tile {
    ulonglong2 v[CW / 2];
};

template <u32 CW>
__device__ __forceinline__ void tile_fetch(Tile<CW> &t, const uint8_t *events, u64 first, u64 n) {
    const u32 lane = lane_id();
    const u64 nrec = n > first ? (n - first < 32 ? n - first : 32) : 0;
    const ulonglong2 *src = (const ulonglong2 *)(events + first * (u64)CW * 8);
#pragma unroll
    for (u32 k = 0; k < CW / 2; k++) {
        const u32 c = lane + 32u * k; /* chunk c holds words 2c, 2c + 1 of the tile */
        t.v[k] = (2u * c) / CW < nrec ? __ldcs(src + c) : make_ulonglong2(0ull, 0ull);
    }
}

template <u32 CW>
__device__ __forceinline__ void tile_store(u64 *ctxw, const Tile<CW> &t) {
    const u32 row = GX_CTX_ROW(CW), lane = lane_id();
#pragma unroll
    for (u32 k = 0; k < CW / 2; k++) {
        const u32 word = 2u * (lane + 32u * k), rec = word / CW, f = word % CW;
        ctxw[f * row + rec] = t.v[k].x;
        ctxw[(f + 1) * row + rec] = t.v[k].y;
    }
}

/* ------------------------------------------------------------------ kernel skeleton */
/* what a per-event body sees: the staged program image and its maps */
struct ExecEnv {
    const u64 *uops;
    const gx_dmap *maps;
    u64 *stats;
    u64 budget;
    u32 slot;      /* which program of a multi-program specialised kernel (chunk.pad); 0 in plain mode */
    u32 wc_bits;   /* block-private combining: log2 cache entries per map, 0 = off */
    u32 wc_agg;    /* updates that miss the cache are warp-aggregated */
    u32 ctx_row;   /* words between rows of the event tile (GX_CTX_ROW) */
    uint8_t *shard; /* the block's combining area (shared memory) */
    u32 n_maps;    /* the program's maps (descriptors at `maps`) */
    u32 ctx_size;  /* bytes of one event record */
};

/* ------------------------------------------------------------------ block-private combining */
/*
 * Hierarchical map updates (the per-SM shards merged into the global map of Sec. 5.3):
 * when the verifier proved that a program only updates a map's values with non-fetching
 * commutative operations, those updates first land in shared memory and each block adds
 * its totals to device memory once, when it finishes (or, in the persistent kernel, when
 * its chunk ends).  Small array maps get a whole private copy; other maps get a cache of
 * 2^wc_bits entries tagged by value address, and an update whose entry is held by another
 * value goes straight to device memory.  Every operation here is per lane: no warp
 * collectives.  A 64-bit add is split into 32-bit halves (the low half's carry is added
 * into the high half), since 32-bit shared atomics are native.
 */
__device__ __forceinline__ u32 sh_addr(const void *p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ u32 sh_atom_add(u32 a, u32 v) {
    u32 r;
    asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(r) : "r"(a), "r"(v) : "memory");
    return r;
}
__device__ __forceinline__ void sh_red(u32 a, u32 v, int op) {
    if (op == AG_ADD) asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
    else if (op == AG_OR) asm volatile("red.shared.or.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
    else if (op == AG_AND) asm volatile("red.shared.and.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
    else asm volatile("red.shared.xor.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

/* identity of an operation on 32 / 64 bits */
template <int OP>
__device__ __forceinline__ u64 wc_ident() {
    return (OP == AG_AND || OP == AG_MIN) ? ~0ull : 0ull;
}

/* apply v to the shared word at a (8-byte aligned for SZ == 8) */
template <int OP, int SZ>
__device__ __forceinline__ void sh_update(u32 a, u64 v) {
    if (SZ == 4) {
        if (OP == AG_ADD || ((u32)v != (u32)wc_ident<OP>())) sh_red(a, (u32)v, OP);
        return;
    }
    if (OP == AG_ADD) {
        u32 lo = (u32)v, hi = (u32)(v >> 32);
        u32 old = sh_atom_add(a, lo);
        hi += (old + lo < old) ? 1u : 0u;
        if (hi) sh_red(a + 4, hi, AG_ADD);
    } else if (OP == AG_MAX) {
        asm volatile("red.shared.max.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
    } else if (OP == AG_MIN) {
        asm volatile("red.shared.min.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
    } else {
        u32 lo = (u32)v, hi = (u32)(v >> 32), id = (u32)wc_ident<OP>();
        if (lo != id) sh_red(a, lo, OP);
        if (hi != id) sh_red(a + 4, hi, OP);
    }
}

/* fill n 32-bit words of a combining area with identities: word i gets ident(i % wpv) */
__device__ __forceinline__ void wc_fill(uint8_t *area, u32 n_words, u32 wpv, u64 and_mask) {
    u32 *w = (u32 *)area;
    for (u32 i = threadIdx.x; i < n_words; i += blockDim.x) w[i] = ((and_mask >> (i % wpv)) & 1) ? ~0u : 0u;
}

/*
 * Cache lookup for the value at `base` in a cache of 2^bits entries of `esize` bytes
 * ({u64 tag, accumulators}): the entry's accumulators, claiming a free entry if needed,
 * or nullptr when the entry holds another value.
 */
__device__ __forceinline__ uint8_t *wc_entry(uint8_t *cache, u32 bits, u32 esize, u64 base) {
    const u32 h = (u32)((base * 0x9E3779B97F4A7C15ull) >> (64 - bits));
    uint8_t *entry = cache + (size_t)h * esize;
    const u32 ta = sh_addr(entry);
    u64 t;
    asm volatile("ld.volatile.shared.u64 %0, [%1];" : "=l"(t) : "r"(ta));
    if (t == 0) {
        asm volatile("atom.shared.cas.b64 %0, [%1], %2, %3;" : "=l"(t) : "r"(ta), "l"(0ull), "l"(base) : "memory");
        if (t == 0) t = base;
    }
    return t == base ? entry + 8 : nullptr;
}

/* device-memory form of a combined total (the block's flush) */
template <int OP, int SZ>
__device__ __forceinline__ void wc_flush_word(void *g, u64 v) {
    if (v == (SZ == 4 ? (wc_ident<OP>() & 0xFFFFFFFFull) : wc_ident<OP>())) return;
    plain_atomic<OP, SZ>(g, v);
}

/*
 * One chunk's events: warp w takes tiles begin + 32w, begin + 32w + blockDim, ...; each
 * warp transposes its 32 records into shared memory, then `run_event` executes one event
 * per lane and returns R0.
 */
template <typename RunEvent>
__device__ __forceinline__ void chunk_tiles(const ExecEnv &env, const gx_chunk &ch, u64 *ctx_all, RunEvent run_event) {
    const u32 warp = threadIdx.x >> 5, lane = lane_id();
    const u32 cw = ch.ctx_size / 8;
    u64 *ctxw = ctx_all + warp * cw * GX_CTX_ROW(cw);
    for (u64 first = ch.begin + (u64)warp * 32; first < ch.end; first += blockDim.x) {
        load_ctx_tile(ctxw, ch.events, first, ch.end, cw);
        const u64 idx = first + lane;
        const bool valid = idx < ch.end;
        u64 r0 = run_event(env, ctxw, valid, ch.idx_base + idx);
        if (valid && ch.ret_out) ch.ret_out[idx] = (long long)r0;
        __syncwarp();
    }
}

/* chunk_tiles for records of CW (4 or 8) words, with the next tile's loads in flight while
   the current tile runs */
template <u32 CW, typename RunEvent>
__device__ __forceinline__ void chunk_tiles_cw(const ExecEnv &env, const gx_chunk &ch, u64 *ctx_all, RunEvent run_event) {
    const u32 warp = threadIdx.x >> 5, lane = lane_id();
    u64 *ctxw = ctx_all + warp * CW * GX_CTX_ROW(CW);
    u64 first = ch.begin + (u64)warp * 32;
    if (first >= ch.end) return;
    Tile<CW> t;
    tile_fetch<CW>(t, ch.events, first, ch.end);
    for (; first < ch.end; first += blockDim.x) {
        tile_store<CW>(ctxw, t);
        __syncwarp();
        const u64 next = first + blockDim.x;
        if (next < ch.end) tile_fetch<CW>(t, ch.events, next, ch.end);
        const u64 idx = first + lane;
        const bool valid = idx < ch.end;
        u64 r0 = run_event(env, ctxw, valid, ch.idx_base + idx);
        if (valid && ch.ret_out) ch.ret_out[idx] = (long long)r0;
        __syncwarp();
    }
}

/* chunk_tiles for any record size, choosing the pipelined form for 32- and 64-byte records */
template <typename RunEvent>
__device__ __forceinline__ void chunk_tiles_any(const ExecEnv &env, const gx_chunk &ch, u64 *ctx_all, RunEvent run_event) {
    if (ch.ctx_size == 32) chunk_tiles_cw<4>(env, ch, ctx_all, run_event);
    else if (ch.ctx_size == 64) chunk_tiles_cw<8>(env, ch, ctx_all, run_event);
    else chunk_tiles(env, ch, ctx_all, run_event);
}

/* ExecEnv of the program image staged at smem */
__device__ __forceinline__ ExecEnv stage_env_at(uint8_t *smem, u32 shard_off, u32 slot, u32 wcp) {
    const gx_dprog_hdr *hdr = (const gx_dprog_hdr *)smem;
    ExecEnv env;
    env.maps = (const gx_dmap *)(smem + sizeof(gx_dprog_hdr));
    env.uops = (const u64 *)(smem + sizeof(gx_dprog_hdr) + hdr->n_maps * sizeof(gx_dmap));
    env.stats = hdr->stats;
    env.budget = hdr->budget;
    env.slot = slot;
    env.wc_bits = wcp & 0xFFu;
    env.wc_agg = (wcp >> 8) & 1u;
    env.ctx_row = GX_CTX_ROW(hdr->ctx_size / 8);
    env.n_maps = hdr->n_maps;
    env.ctx_size = hdr->ctx_size;
    env.shard = smem + shard_off;
    return env;
}

__device__ __forceinline__ ExecEnv stage_env(uint8_t *smem, const ExecParams &P, u32 slot, u32 wcp) {
    return stage_env_at(smem, P.shard_off, slot, wcp);
}

/*
 * The launch skeleton shared by the interpreter and by load-time specialised programs.
 * Plain mode (P.mode == 0): block b stages the program image into shared memory and runs
 * events [b*ept*blockDim, (b+1)*ept*blockDim) as one chunk.  Persistent mode (1): blocks
 * claim chunks {program image, event range} from an atomic cursor until the table is
 * exhausted, restaging the image only when the program changes.  `run_chunk(env, chunk,
 * ctx_area)` runs one chunk (chunk_tiles with the program's per-event code).  The
 * combining area (wc_init / wc_flush) stays open across consecutive chunks of the same
 * program and choice; its totals go to device memory when the program or choice changes
 * and when the block runs out of work, while that program's image is still staged.
 */
template <typename RunChunk, typename Init, typename Flush>
__device__ __forceinline__ void exec_tiles(const ExecParams &P, RunChunk run_chunk, Init wc_init, Flush wc_flush) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ u32 s_chunk;
    u64 *ctx_all = (u64 *)(smem + P.image_area);
    /*
     * One loop for both modes, so the per-event code is inlined once.  Plain: chunks of
     * blockDim * ept events, block b taking the chunks that start at b, b + gridDim, ...
     * of one program.  Persistent: chunks claimed from the table.  Every decision below is
     * block-uniform (plain: this block's position; persistent: the claimed chunk in shared
     * memory), so the barriers inside are reached by every thread.
     */
    const bool plain = P.mode == 0;
    const u64 per = (u64)blockDim.x * P.ept;
    const u32 nchunks = plain ? 0u : (P.nchunks_dev ? *P.nchunks_dev : P.nchunks);
    u64 next = (u64)blockIdx.x * per; /* plain: the first event of this block's next chunk */
    const uint8_t *staged = nullptr;  /* the image in shared memory */
    ExecEnv open;
    u32 open_wcp = 0;
    bool is_open = false;
    for (;;) {
        gx_chunk ch;
        u32 wcp = 0;
        bool done;
        if (plain) {
            done = next >= P.n;
            if (!done) {
                ch.image = P.image;
                ch.events = P.events;
                ch.ret_out = P.ret_out;
                ch.begin = next;
                ch.end = next + per < P.n ? next + per : P.n;
                ch.idx_base = P.idx_base;
                ch.image_bytes = P.image_bytes;
                ch.ctx_size = P.ctx_size;
                ch.pad = 0;
                wcp = P.wc_bits;
                next += (u64)gridDim.x * per;
            } else if (is_open) {
                __syncthreads(); /* every warp is done with its last tile before the flush */
            }
        } else {
            __syncthreads();
            if (threadIdx.x == 0) s_chunk = atomicAdd(P.cursor, 1u);
            __syncthreads();
            const u32 c = s_chunk;
            done = c >= nchunks;
            if (!done) {
                ch = P.chunks[c];
                wcp = (ch.pad >> 63) ? (u32)(ch.pad >> 32) & 0x1FFu : P.wc_bits; /* the chunk's own choice */
            }
        }
        if (is_open && (done || (u32)ch.pad != open.slot || wcp != open_wcp)) {
            wc_flush(open);
            __syncthreads();
            is_open = false;
        }
        if (done) break;
        if (ch.image != staged) {
            stage_image(smem, ch.image, ch.image_bytes);
            staged = ch.image;
        }
        const ExecEnv env = stage_env(smem, P, (u32)ch.pad, wcp);
        if (env.wc_bits && !is_open) {
            wc_init(env);
            __syncthreads();
            open = env;
            open_wcp = wcp;
            is_open = true;
        }
        run_chunk(env, ch, ctx_all);
    }
}

/* the interpreter: per-event code inline, no block-private combining */
template <typename RunEvent>
__device__ __forceinline__ void exec_tiles(const ExecParams &P, RunEvent run_event) {
    exec_tiles(
        P,
        [&](const ExecEnv &env, const gx_chunk &ch, u64 *ctx_all) { chunk_tiles_any(env, ch, ctx_all, run_event); },
        [](const ExecEnv &) {}, [](const ExecEnv &) {});
}

} // namespace gx

#endif /* GX_DEVICE_CUH */
