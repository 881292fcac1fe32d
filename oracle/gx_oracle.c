/*
 * ORACLE -- test infrastructure only.
 *
 * A plain, slow, sequential CPU eBPF interpreter with its own array map, hash map and
 * ring buffer.  It is the parity authority for the GPU engine and shares no code with
 * it: only tests, the package smoke check and the benchmark's CPU-baseline leg may load
 * it; the engine never does.
 *
 * What it computes (the plain definition of a batch run):
 *   for every event i in index order, run the program once on a fresh register file
 *   with R1 = pointer to that event's ctx_size-byte record and R10 = the top of a fresh
 *   512-byte stack; map and ring-buffer state carries over from event to event.
 * Two further forms, defined where they are written out below: the warp run (or_run_warps,
 * the warp-level execution of Sec. 4.4.1 / 4.4.2) and the strict-alignment run
 * (or_run_flags with OR_STRICT_ALIGN).
 * The paper runs verified eBPF handlers on device events (Sec. 4.3, Sec. 4.4, Sec. 5.3)
 * and names the instruction set only as a restricted eBPF subset, so the instruction
 * semantics follow the standard eBPF ISA (RFC 9669):
 *   Sec. 4.1 arithmetic (ALU/ALU64), incl. division by zero -> 0, modulo by zero keeps
 *            the dividend (ALU zero-extends), shift counts masked, signed division and
 *            modulo truncate toward zero (SDIV/SMOD via off = 1), MOVSX (off 8/16/32);
 *   Sec. 4.2 byte swaps (END: to-le / to-be on ALU, unconditional swap on ALU64);
 *   Sec. 4.3 jumps (JMP/JMP32, JA with imm offset in the JMP32 class, CALL, EXIT);
 *   Sec. 5   loads/stores (LDX MEM / MEMSX, ST, STX), 64-bit immediates, atomics
 *            (ADD/OR/AND/XOR with optional FETCH, XCHG, CMPXCHG on W/DW).
 * Helper numbering follows the Linux UAPI (1 lookup, 2 update, 3 delete, 130..133 ring
 * buffer) plus two engine-private helpers 0x10000 / 0x10001 (unsigned atomic max/min of
 * a u64 in map-value memory).  Choices where neither the paper nor the RFC fixes the
 * result:
 *   - signed division overflow INT_MIN / -1 gives INT_MIN, INT_MIN % -1 gives 0;
 *   - ringbuf_reserve returns zero-filled memory; each record carries a 16-byte header
 *     {u32 len; u32 flags (bit0 = discarded); u64 event_idx}, payload padded to 8;
 *   - ringbuf_output returns -EAGAIN (-11) when the ring is full; reserve returns NULL
 *     and both count a drop;
 *   - a ring closes at the first record that does not fit: that reservation and every
 *     later one fail (and count a drop), whatever their size, until the ring is drained.
 *     The records kept are a prefix of the reservations, so the data is one contiguous
 *     run from the start of the ring;
 *   - array update with key >= max_entries -> -E2BIG, NOEXIST -> -EEXIST, delete ->
 *     -EINVAL; hash update NOEXIST on a present key -> -EEXIST, EXIST on an absent key ->
 *     -ENOENT, insert beyond max_entries -> -E2BIG; hash delete of an absent key -> -ENOENT;
 *   - after a helper call R1..R5 are set to 0 and a void helper leaves R0 = 0.
 * Every memory access is checked against the regions the event may touch (its ctx
 * read-only, its stack, the values returned by lookups and the ring-buffer records it
 * reserved), so the oracle is safe on programs nobody verified.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ENOENT (-2)
#define OR_E2BIG (-7)
#define OR_EAGAIN (-11)
#define OR_ENOMEM (-12)
#define OR_EFAULT (-14)
#define OR_EEXIST (-17)
#define OR_EINVAL (-22)
#define OR_EBUDGET (-1002)

#define MAP_HASH 1
#define MAP_ARRAY 2
#define MAP_RINGBUF 27

#define STACK_BYTES 512
#define MAX_REGIONS 256

/* ------------------------------------------------------------------ maps */
typedef struct hnode {
    struct hnode *next;     /* bucket chain */
    struct hnode *all_next; /* every node ever allocated (freed at destroy) */
    int live;
    uint8_t *key;
    uint8_t *value;
} hnode;

typedef struct or_map {
    uint32_t type, key_size, value_size, max_entries;
    uint8_t *values; /* array: max_entries * value_size */
    hnode **buckets; /* hash */
    uint32_t nbuckets, count;
    hnode *all;
    uint8_t *ring; /* ring buffer: max_entries bytes */
    uint64_t ring_used, dropped;
    int ring_closed; /* a reservation did not fit: every later one fails until a drain */
} or_map;

static uint64_t fnv1a(const uint8_t *p, uint32_t n) {
    uint64_t h = 1469598103934665603ULL;
    for (uint32_t i = 0; i < n; i++) {
        h ^= p[i];
        h *= 1099511628211ULL;
    }
    return h;
}

or_map *or_map_create(uint32_t type, uint32_t key_size, uint32_t value_size, uint32_t max_entries) {
    or_map *m = (or_map *)calloc(1, sizeof(or_map));
    if (!m) return NULL;
    m->type = type;
    m->key_size = key_size;
    m->value_size = value_size;
    m->max_entries = max_entries;
    if (type == MAP_ARRAY) {
        if (key_size != 4 || value_size == 0 || max_entries == 0) goto bad;
        m->values = (uint8_t *)calloc((size_t)max_entries, value_size);
        if (!m->values) goto bad;
    } else if (type == MAP_HASH) {
        if (key_size == 0 || value_size == 0 || max_entries == 0) goto bad;
        m->nbuckets = 1024;
        while (m->nbuckets < max_entries && m->nbuckets < (1u << 22)) m->nbuckets <<= 1;
        m->buckets = (hnode **)calloc(m->nbuckets, sizeof(hnode *));
        if (!m->buckets) goto bad;
    } else if (type == MAP_RINGBUF) {
        if (max_entries < 64) goto bad;
        m->ring = (uint8_t *)calloc(max_entries, 1);
        if (!m->ring) goto bad;
    } else {
        goto bad;
    }
    return m;
bad:
    free(m->values);
    free(m->buckets);
    free(m->ring);
    free(m);
    return NULL;
}

void or_map_destroy(or_map *m) {
    if (!m) return;
    hnode *n = m->all;
    while (n) {
        hnode *x = n->all_next;
        free(n->key);
        free(n->value);
        free(n);
        n = x;
    }
    free(m->values);
    free(m->buckets);
    free(m->ring);
    free(m);
}

static hnode *hash_find(or_map *m, const uint8_t *key) {
    hnode *n = m->buckets[fnv1a(key, m->key_size) & (m->nbuckets - 1)];
    for (; n; n = n->next)
        if (memcmp(n->key, key, m->key_size) == 0) return n;
    return NULL;
}

static int hash_insert(or_map *m, const uint8_t *key, const uint8_t *value) {
    if (m->count >= m->max_entries) return OR_E2BIG;
    hnode *n = (hnode *)calloc(1, sizeof(hnode));
    if (!n) return OR_ENOMEM;
    n->key = (uint8_t *)malloc(m->key_size);
    n->value = (uint8_t *)malloc(m->value_size);
    if (!n->key || !n->value) {
        free(n->key);
        free(n->value);
        free(n);
        return OR_ENOMEM;
    }
    memcpy(n->key, key, m->key_size);
    memcpy(n->value, value, m->value_size);
    n->live = 1;
    uint64_t b = fnv1a(key, m->key_size) & (m->nbuckets - 1);
    n->next = m->buckets[b];
    m->buckets[b] = n;
    n->all_next = m->all;
    m->all = n;
    m->count++;
    return OR_OK;
}

static int hash_delete(or_map *m, const uint8_t *key) {
    uint64_t b = fnv1a(key, m->key_size) & (m->nbuckets - 1);
    hnode **pp = &m->buckets[b];
    for (; *pp; pp = &(*pp)->next) {
        if (memcmp((*pp)->key, key, m->key_size) == 0) {
            hnode *n = *pp;
            *pp = n->next; /* unlinked; memory stays until destroy, like a deferred free */
            n->live = 0;
            m->count--;
            return OR_OK;
        }
    }
    return OR_ENOENT;
}

/* map-level operations used by both the helpers and the host API */
static uint8_t *map_lookup(or_map *m, const uint8_t *key) {
    if (m->type == MAP_ARRAY) {
        uint32_t k;
        memcpy(&k, key, 4);
        return k < m->max_entries ? m->values + (size_t)k * m->value_size : NULL;
    }
    if (m->type == MAP_HASH) {
        hnode *n = hash_find(m, key);
        return n ? n->value : NULL;
    }
    return NULL;
}

static int map_update(or_map *m, const uint8_t *key, const uint8_t *value, uint64_t flags) {
    if (flags > 2) return OR_EINVAL;
    if (m->type == MAP_ARRAY) {
        uint32_t k;
        memcpy(&k, key, 4);
        if (k >= m->max_entries) return OR_E2BIG;
        if (flags == 1) return OR_EEXIST;
        memcpy(m->values + (size_t)k * m->value_size, value, m->value_size);
        return OR_OK;
    }
    if (m->type == MAP_HASH) {
        hnode *n = hash_find(m, key);
        if (n) {
            if (flags == 1) return OR_EEXIST;
            memcpy(n->value, value, m->value_size);
            return OR_OK;
        }
        if (flags == 2) return OR_ENOENT;
        return hash_insert(m, key, value);
    }
    return OR_EINVAL;
}

static int map_delete(or_map *m, const uint8_t *key) {
    if (m->type == MAP_HASH) return hash_delete(m, key);
    return OR_EINVAL;
}

int or_map_update(or_map *m, const void *key, const void *value, uint64_t flags) {
    return map_update(m, (const uint8_t *)key, (const uint8_t *)value, flags);
}

int or_map_delete(or_map *m, const void *key) { return map_delete(m, (const uint8_t *)key); }

int or_map_lookup(or_map *m, const void *key, void *value_out) {
    uint8_t *v = map_lookup(m, (const uint8_t *)key);
    if (!v) return OR_ENOENT;
    memcpy(value_out, v, m->value_size);
    return OR_OK;
}

/* array: all values; returns bytes copied or an error */
int64_t or_array_read(or_map *m, void *out, uint64_t cap) {
    if (m->type != MAP_ARRAY) return OR_EINVAL;
    uint64_t bytes = (uint64_t)m->max_entries * m->value_size;
    if (cap < bytes) return OR_E2BIG;
    memcpy(out, m->values, bytes);
    return (int64_t)bytes;
}

int64_t or_hash_count(or_map *m) { return m->type == MAP_HASH ? (int64_t)m->count : OR_EINVAL; }

/* hash: live pairs as packed {key, value} in bucket order; returns the pair count */
int64_t or_hash_dump(or_map *m, void *out, uint64_t cap_pairs) {
    if (m->type != MAP_HASH) return OR_EINVAL;
    if (cap_pairs < m->count) return OR_E2BIG;
    uint8_t *o = (uint8_t *)out;
    int64_t k = 0;
    for (uint32_t b = 0; b < m->nbuckets; b++)
        for (hnode *n = m->buckets[b]; n; n = n->next) {
            memcpy(o, n->key, m->key_size);
            memcpy(o + m->key_size, n->value, m->value_size);
            o += m->key_size + m->value_size;
            k++;
        }
    return k;
}

/* ring buffer: committed records (header + padded payload) packed, in emission order */
int64_t or_ringbuf_read(or_map *m, void *out, uint64_t cap, uint64_t *dropped) {
    if (m->type != MAP_RINGBUF) return OR_EINVAL;
    uint8_t *o = (uint8_t *)out;
    uint64_t w = 0;
    for (uint64_t pos = 0; pos + 16 <= m->ring_used;) {
        uint32_t len, flags;
        memcpy(&len, m->ring + pos, 4);
        memcpy(&flags, m->ring + pos + 4, 4);
        uint64_t rec = 16 + (((uint64_t)len + 7) & ~7ULL);
        if (!(flags & 1)) {
            if (w + rec > cap) return OR_E2BIG;
            memcpy(o + w, m->ring + pos, rec);
            w += rec;
        }
        pos += rec;
    }
    if (dropped) *dropped = m->dropped;
    return (int64_t)w;
}

void or_ringbuf_reset(or_map *m) {
    if (m->type != MAP_RINGBUF) return;
    memset(m->ring, 0, m->max_entries);
    m->ring_used = 0;
    m->dropped = 0;
    m->ring_closed = 0;
}

/* ------------------------------------------------------------------ deferred updates */
/*
 * Deferral (or_run_flags with a defer mask): the engine's block-private combining taken to
 * its extreme.  Non-fetching ADD / OR / AND / XOR atomics and the max / min helpers into
 * the values of a deferred map are logged instead of applied, and the log is applied in
 * order after the last event.  Any other access to a deferred map's values stops the run
 * with OR_EDEFER: a load, a plain store, a fetch or exchange, a helper reading them, an
 * update that may overwrite, a delete.  For a map the verifier calls combinable none of
 * these happens, and then the deferred run's results equal the plain run's.
 */
#define OR_EDEFER (-1004)
#define DEFER_MAX 1 /* op codes besides the BPF_ATOMIC ones (0x00, 0x40, 0x50, 0xA0) */
#define DEFER_MIN 2

typedef struct {
    uint8_t *p;
    int size, op;
    uint64_t v;
} dop;

typedef struct {
    uint32_t mask;
    or_map **maps;
    uint32_t n_maps;
    dop *log;
    size_t n, cap;
} defer_t;

static int overlaps_values(const or_map *m, uint64_t a, uint64_t size) {
    if (m->type == MAP_ARRAY) {
        uint64_t b = (uint64_t)(uintptr_t)m->values;
        return a < b + (uint64_t)m->max_entries * m->value_size && a + size > b;
    }
    if (m->type == MAP_HASH)
        for (const hnode *n = m->all; n; n = n->all_next) {
            uint64_t b = (uint64_t)(uintptr_t)n->value;
            if (a < b + m->value_size && a + size > b) return 1;
        }
    return 0;
}

/* [a, a + size) overlaps the values of a deferred map */
static int deferred(const defer_t *d, uint64_t a, uint64_t size) {
    if (!d) return 0;
    for (uint32_t i = 0; i < d->n_maps; i++)
        if (((d->mask >> i) & 1) && overlaps_values(d->maps[i], a, size)) return 1;
    return 0;
}

static int deferred_map(const defer_t *d, const or_map *m) {
    if (!d) return 0;
    for (uint32_t i = 0; i < d->n_maps; i++)
        if (d->maps[i] == m) return (d->mask >> i) & 1;
    return 0;
}

static int defer_log(defer_t *d, uint8_t *p, int size, int op, uint64_t v) {
    if (d->n == d->cap) {
        size_t cap = d->cap ? 2 * d->cap : 1024;
        dop *log = (dop *)realloc(d->log, cap * sizeof(dop));
        if (!log) return OR_ENOMEM;
        d->log = log;
        d->cap = cap;
    }
    d->log[d->n].p = p;
    d->log[d->n].size = size;
    d->log[d->n].op = op;
    d->log[d->n].v = v;
    d->n++;
    return OR_OK;
}

/* ------------------------------------------------------------------ interpreter */
typedef struct {
    uint8_t *base;
    uint64_t size;
    int writable;
} region;

typedef struct {
    region r[MAX_REGIONS];
    int n;
    int strict_align; /* or_run_flags OR_STRICT_ALIGN: instruction accesses must be naturally aligned */
    defer_t *defer;   /* or_run_flags with a defer mask: the deferral state */
} regions;

static void grant(regions *g, uint8_t *base, uint64_t size, int writable) {
    if (g->n < MAX_REGIONS) {
        g->r[g->n].base = base;
        g->r[g->n].size = size;
        g->r[g->n].writable = writable;
        g->n++;
    } else { /* keep the newest grants: drop the oldest non-fixed one (index >= 2) */
        memmove(&g->r[2], &g->r[3], sizeof(region) * (MAX_REGIONS - 3));
        g->r[MAX_REGIONS - 1].base = base;
        g->r[MAX_REGIONS - 1].size = size;
        g->r[MAX_REGIONS - 1].writable = writable;
    }
}

/* pointer to `size` bytes at address `a` if it lies inside one granted region */
static uint8_t *check(const regions *g, uint64_t a, uint64_t size, int write) {
    for (int i = 0; i < g->n; i++) {
        uint64_t b = (uint64_t)(uintptr_t)g->r[i].base;
        if (a >= b && size <= g->r[i].size && a - b <= g->r[i].size - size) {
            if (write && !g->r[i].writable) return NULL;
            return (uint8_t *)(uintptr_t)a;
        }
    }
    return NULL;
}

static uint64_t load_le(const uint8_t *p, int size) {
    uint64_t v = 0;
    for (int i = size - 1; i >= 0; i--) v = (v << 8) | p[i];
    return v;
}

static void store_le(uint8_t *p, int size, uint64_t v) {
    for (int i = 0; i < size; i++) {
        p[i] = (uint8_t)(v & 0xFF);
        v >>= 8;
    }
}

static uint64_t sext(uint64_t v, int bits) {
    if (bits >= 64) return v;
    uint64_t m = 1ULL << (bits - 1);
    v &= (1ULL << bits) - 1ULL;
    return (v ^ m) - m;
}

static uint64_t bswap(uint64_t v, int bits) {
    uint64_t r = 0;
    for (int i = 0; i < bits / 8; i++) r = (r << 8) | ((v >> (8 * i)) & 0xFF);
    return r;
}

static int size_of(uint8_t op) { /* bits 3..4 of a load/store opcode */
    switch (op & 0x18) {
    case 0x00: return 4;
    case 0x08: return 2;
    case 0x10: return 1;
    default: return 8;
    }
}

/* 64-bit ALU result of `op` on (d, s); is32 selects ALU (32-bit) semantics */
static int alu(uint8_t code, int is32, int16_t off, uint64_t d, uint64_t s, uint64_t *out) {
    if (is32) {
        d &= 0xFFFFFFFFULL;
        s &= 0xFFFFFFFFULL;
    }
    uint64_t r;
    int sh = is32 ? 31 : 63;
    switch (code) {
    case 0x00: r = d + s; break;
    case 0x10: r = d - s; break;
    case 0x20: r = d * s; break;
    case 0x30:
        if (off == 0) {
            r = s ? d / s : 0;
        } else if (off == 1) {
            if (is32) {
                int32_t a = (int32_t)(uint32_t)d, b = (int32_t)(uint32_t)s;
                if (b == 0) r = 0;
                else if (a == INT32_MIN && b == -1) r = (uint32_t)INT32_MIN;
                else r = (uint32_t)(a / b);
            } else {
                int64_t a = (int64_t)d, b = (int64_t)s;
                if (b == 0) r = 0;
                else if (a == INT64_MIN && b == -1) r = (uint64_t)INT64_MIN;
                else r = (uint64_t)(a / b);
            }
        } else {
            return OR_EINVAL;
        }
        break;
    case 0x40: r = d | s; break;
    case 0x50: r = d & s; break;
    case 0x60: r = d << (s & sh); break;
    case 0x70: r = d >> (s & sh); break;
    case 0x80: r = (uint64_t)0 - d; break;
    case 0x90:
        if (off == 0) {
            r = s ? d % s : d;
        } else if (off == 1) {
            if (is32) {
                int32_t a = (int32_t)(uint32_t)d, b = (int32_t)(uint32_t)s;
                if (b == 0) r = (uint32_t)a;
                else if (b == -1) r = 0;
                else r = (uint32_t)(a % b);
            } else {
                int64_t a = (int64_t)d, b = (int64_t)s;
                if (b == 0) r = (uint64_t)a;
                else if (b == -1) r = 0;
                else r = (uint64_t)(a % b);
            }
        } else {
            return OR_EINVAL;
        }
        break;
    case 0xA0: r = d ^ s; break;
    case 0xB0:
        if (off == 0) r = s;
        else if (off == 8 || off == 16 || (off == 32 && !is32)) r = sext(s, off);
        else return OR_EINVAL;
        break;
    case 0xC0:
        if (is32) r = (uint32_t)((int32_t)(uint32_t)d >> (s & 31));
        else r = (uint64_t)((int64_t)d >> (s & 63));
        break;
    default: return OR_EINVAL;
    }
    if (code != 0xB0 && code != 0x30 && code != 0x90 && off != 0) return OR_EINVAL;
    *out = is32 ? (r & 0xFFFFFFFFULL) : r;
    return OR_OK;
}

static int cond(uint8_t code, int is32, uint64_t d, uint64_t s, int *taken) {
    if (is32) {
        d &= 0xFFFFFFFFULL;
        s &= 0xFFFFFFFFULL;
    }
    int64_t sd = is32 ? (int64_t)(int32_t)(uint32_t)d : (int64_t)d;
    int64_t ss = is32 ? (int64_t)(int32_t)(uint32_t)s : (int64_t)s;
    switch (code) {
    case 0x10: *taken = d == s; break;
    case 0x20: *taken = d > s; break;
    case 0x30: *taken = d >= s; break;
    case 0x40: *taken = (d & s) != 0; break;
    case 0x50: *taken = d != s; break;
    case 0x60: *taken = sd > ss; break;
    case 0x70: *taken = sd >= ss; break;
    case 0xA0: *taken = d < s; break;
    case 0xB0: *taken = d <= s; break;
    case 0xC0: *taken = sd < ss; break;
    case 0xD0: *taken = sd <= ss; break;
    default: return OR_EINVAL;
    }
    return OR_OK;
}

typedef struct {
    or_map **maps;
    uint32_t n_maps;
    uint64_t event_idx;
    regions *g;
    region granted; /* the region the last helper call granted (size 0: none) */
    int strict_align;
    uint64_t helpers, mem; /* this event's helper calls and loads / stores / atomics */
    defer_t *defer;
} hctx;

static or_map *map_arg(const hctx *h, uint64_t v) {
    for (uint32_t i = 0; i < h->n_maps; i++)
        if ((uint64_t)(uintptr_t)h->maps[i] == v) return h->maps[i];
    return NULL;
}

static uint8_t *rb_reserve(or_map *m, uint64_t size, uint64_t event_idx) {
    uint64_t rec = 16 + ((size + 7) & ~7ULL);
    if (size == 0 || size > 0xFFFFFFFFULL) {
        m->dropped++;
        return NULL;
    }
    if (m->ring_closed || m->ring_used + rec > m->max_entries) {
        m->ring_closed = 1;
        m->dropped++;
        return NULL;
    }
    uint8_t *p = m->ring + m->ring_used;
    memset(p, 0, rec);
    store_le(p, 4, size);
    store_le(p + 4, 4, 0);
    store_le(p + 8, 8, event_idx);
    m->ring_used += rec;
    return p + 16;
}

/* header of the record whose payload starts at p, if p is one of this event's grants */
static int rb_finish(const hctx *h, uint64_t p, int discard) {
    for (uint32_t i = 0; i < h->n_maps; i++) {
        or_map *m = h->maps[i];
        if (m->type != MAP_RINGBUF) continue;
        uint64_t b = (uint64_t)(uintptr_t)m->ring;
        if (p >= b + 16 && p < b + m->ring_used) {
            uint8_t *hdr = (uint8_t *)(uintptr_t)(p - 16);
            store_le(hdr + 4, 4, discard ? 1 : 0);
            return OR_OK;
        }
    }
    return OR_EFAULT;
}

static int helper(hctx *h, int32_t id, uint64_t *R) {
    regions *g = h->g;
    uint64_t r0 = 0;
    switch (id) {
    case 1: { /* map_lookup_elem(map, key) */
        or_map *m = map_arg(h, R[1]);
        if (!m || m->type == MAP_RINGBUF) return OR_EFAULT;
        if (deferred(h->defer, R[2], m->key_size)) return OR_EDEFER;
        uint8_t *k = check(g, R[2], m->key_size, 0);
        if (!k) return OR_EFAULT;
        uint8_t *v = map_lookup(m, k);
        if (v) {
            grant(g, v, m->value_size, 1);
            h->granted = g->r[g->n - 1];
        }
        r0 = (uint64_t)(uintptr_t)v;
        break;
    }
    case 2: { /* map_update_elem(map, key, value, flags) */
        or_map *m = map_arg(h, R[1]);
        if (!m || m->type == MAP_RINGBUF) return OR_EFAULT;
        if (deferred(h->defer, R[2], m->key_size) || deferred(h->defer, R[3], m->value_size) ||
            (deferred_map(h->defer, m) && R[4] != 1))
            return OR_EDEFER; /* a deferred map may only gain keys (NOEXIST inserts) */
        uint8_t *k = check(g, R[2], m->key_size, 0);
        uint8_t *v = check(g, R[3], m->value_size, 0);
        if (!k || !v) return OR_EFAULT;
        uint8_t kb[512], vb[4096];
        if (m->key_size > sizeof kb || m->value_size > sizeof vb) return OR_EINVAL;
        memcpy(kb, k, m->key_size);
        memcpy(vb, v, m->value_size);
        r0 = (uint64_t)(int64_t)map_update(m, kb, vb, R[4]);
        break;
    }
    case 3: { /* map_delete_elem(map, key) */
        or_map *m = map_arg(h, R[1]);
        if (!m || m->type == MAP_RINGBUF) return OR_EFAULT;
        if (deferred_map(h->defer, m) || deferred(h->defer, R[2], m->key_size)) return OR_EDEFER;
        uint8_t *k = check(g, R[2], m->key_size, 0);
        if (!k) return OR_EFAULT;
        r0 = (uint64_t)(int64_t)map_delete(m, k);
        break;
    }
    case 130: { /* ringbuf_output(rb, data, size, flags) */
        or_map *m = map_arg(h, R[1]);
        if (!m || m->type != MAP_RINGBUF) return OR_EFAULT;
        if (R[4] & ~3ULL) {
            r0 = (uint64_t)(int64_t)OR_EINVAL;
            break;
        }
        if (deferred(h->defer, R[2], R[3])) return OR_EDEFER;
        uint8_t *src = check(g, R[2], R[3], 0);
        if (!src && R[3]) return OR_EFAULT;
        uint8_t tmp[4096];
        if (R[3] > sizeof tmp) return OR_EINVAL;
        if (R[3]) memcpy(tmp, src, R[3]); /* a zero-size output may name no memory at all */
        uint8_t *p = rb_reserve(m, R[3], h->event_idx);
        if (!p) {
            r0 = (uint64_t)(int64_t)OR_EAGAIN;
            break;
        }
        memcpy(p, tmp, R[3]);
        r0 = 0;
        break;
    }
    case 131: { /* ringbuf_reserve(rb, size, flags) */
        or_map *m = map_arg(h, R[1]);
        if (!m || m->type != MAP_RINGBUF) return OR_EFAULT;
        uint8_t *p = R[3] ? NULL : rb_reserve(m, R[2], h->event_idx);
        if (p) {
            grant(g, p, R[2], 1);
            h->granted = g->r[g->n - 1];
        }
        r0 = (uint64_t)(uintptr_t)p;
        break;
    }
    case 132: /* ringbuf_submit(data, flags) */
    case 133: /* ringbuf_discard(data, flags) */
        if (rb_finish(h, R[1], id == 133) != OR_OK) return OR_EFAULT;
        r0 = 0;
        break;
    case 0x10000: /* atomic_max_u64(ptr, v) */
    case 0x10001: { /* atomic_min_u64(ptr, v) */
        uint8_t *p = check(g, R[1], 8, 1);
        if (!p || (g->strict_align && R[1] % 8)) return OR_EFAULT;
        if (deferred(h->defer, R[1], 8)) {
            int rc = defer_log(h->defer, p, 8, id == 0x10000 ? DEFER_MAX : DEFER_MIN, R[2]);
            if (rc != OR_OK) return rc;
            r0 = 0;
            break;
        }
        uint64_t cur = load_le(p, 8);
        if (id == 0x10000 ? R[2] > cur : R[2] < cur) store_le(p, 8, R[2]);
        r0 = 0;
        break;
    }
    default: return OR_EINVAL;
    }
    R[0] = r0;
    for (int i = 1; i <= 5; i++) R[i] = 0;
    return OR_OK;
}


/* ------------------------------------------------------------------ one instruction, one lane */
/* ALU / ALU64 (RFC 9669 Sec. 4.1, byte swaps Sec. 4.2) on register file R */
static int ins_alu(uint64_t *R, uint8_t op, int dst, int src, int16_t off, int32_t imm) {
    int is32 = (op & 7) == 4;
    uint8_t code = op & 0xF0;
    if (dst == 10) return OR_EINVAL;
    if (code == 0xD0) { /* END */
        if (imm != 16 && imm != 32 && imm != 64) return OR_EINVAL;
        if (!is32 && (op & 0x08)) return OR_EINVAL;
        if (is32 && !(op & 0x08)) R[dst] = imm == 64 ? R[dst] : (R[dst] & ((1ULL << imm) - 1ULL));
        else R[dst] = bswap(R[dst], imm);
        return OR_OK;
    }
    uint64_t s;
    if (op & 0x08) s = R[src];
    else s = is32 ? (uint64_t)(uint32_t)imm : (uint64_t)(int64_t)imm;
    if (code == 0x80 && (op & 0x08)) return OR_EINVAL;
    if (code == 0xB0 && off != 0 && !(op & 0x08)) return OR_EINVAL;
    uint64_t r;
    if (alu(code, is32, off, R[dst], s, &r) != OR_OK) return OR_EINVAL;
    R[dst] = r;
    return OR_OK;
}

/* outcome of a conditional jump (JMP / JMP32 other than JA, CALL and EXIT; RFC 9669 Sec. 4.3) */
static int ins_cond(const uint64_t *R, uint8_t op, int dst, int src, int32_t imm, int *taken) {
    uint64_t s = (op & 0x08) ? R[src] : (uint64_t)(int64_t)imm;
    return cond(op & 0xF0, (op & 7) == 6, R[dst], s, taken);
}

/* 64-bit immediate load (RFC 9669 Sec. 5.4): a constant or a map handle */
static int ins_ld64(uint64_t *R, const hctx *h, const uint64_t *insns, uint32_t n, uint32_t pc) {
    uint64_t w = insns[pc];
    int dst = (int)((w >> 8) & 0xF), src = (int)((w >> 12) & 0xF);
    int32_t imm = (int32_t)(uint32_t)(w >> 32);
    if ((w & 0xFF) != 0x18 || pc + 1 >= n || dst == 10) return OR_EINVAL;
    uint64_t hi = insns[pc + 1] >> 32;
    if (src == 0) {
        R[dst] = ((uint64_t)(uint32_t)imm) | (hi << 32);
    } else if (src == 1) {
        if ((uint32_t)imm >= h->n_maps) return OR_EINVAL;
        R[dst] = (uint64_t)(uintptr_t)h->maps[(uint32_t)imm];
    } else {
        return OR_EINVAL;
    }
    return OR_OK;
}

/* LDX: MEM and MEMSX loads (RFC 9669 Sec. 5.1, 5.2) */
static int ins_ldx(uint64_t *R, const regions *g, uint8_t op, int dst, int src, int16_t off) {
    uint8_t mode = op & 0xE0;
    int sz = size_of(op);
    if (dst == 10 || (mode != 0x60 && mode != 0x80) || (mode == 0x80 && sz == 8)) return OR_EINVAL;
    uint64_t a = R[src] + (uint64_t)(int64_t)off;
    if (deferred(g->defer, a, (uint64_t)sz)) return OR_EDEFER;
    uint8_t *p = check(g, a, (uint64_t)sz, 0);
    if (!p || (g->strict_align && a % (uint64_t)sz)) return OR_EFAULT;
    uint64_t v = load_le(p, sz);
    R[dst] = mode == 0x80 ? sext(v, 8 * sz) : v;
    return OR_OK;
}

/* the address a ST / STX writes */
static uint64_t store_addr(const uint64_t *R, int dst, int16_t off) { return R[dst] + (uint64_t)(int64_t)off; }

/* ST / STX: plain stores (RFC 9669 Sec. 5.1) and atomics (Sec. 5.3) */
static int ins_store(uint64_t *R, const regions *g, uint8_t op, int dst, int src, int16_t off, int32_t imm) {
    uint8_t cls = op & 7, mode = op & 0xE0;
    int sz = size_of(op);
    uint64_t a = store_addr(R, dst, off);
    if (g->strict_align && a % (uint64_t)sz) return OR_EFAULT;
    if (deferred(g->defer, a, (uint64_t)sz)) { /* only a non-fetching ADD / OR / AND / XOR is deferred */
        const int base = imm & ~1;
        if (mode != 0xC0 || cls != 3 || (imm & 1) || (sz != 4 && sz != 8) ||
            !(base == 0x00 || base == 0x40 || base == 0x50 || base == 0xA0))
            return OR_EDEFER;
        uint8_t *p = check(g, a, (uint64_t)sz, 1);
        if (!p) return OR_EFAULT;
        return defer_log(g->defer, p, sz, base, R[src] & (sz == 4 ? 0xFFFFFFFFULL : ~0ULL));
    }
    if (mode == 0x60) {
        uint8_t *p = check(g, a, (uint64_t)sz, 1);
        if (!p) return OR_EFAULT;
        store_le(p, sz, cls == 2 ? (uint64_t)(int64_t)imm : R[src]);
        return OR_OK;
    }
    if (mode != 0xC0 || cls != 3 || (sz != 4 && sz != 8)) return OR_EINVAL;
    uint8_t *p = check(g, a, (uint64_t)sz, 1);
    if (!p) return OR_EFAULT;
    uint64_t mask = sz == 4 ? 0xFFFFFFFFULL : ~0ULL;
    uint64_t old = load_le(p, sz);
    uint64_t v = R[src] & mask;
    int fetch = imm & 1;
    switch (imm & ~1) {
    case 0x00: store_le(p, sz, (old + v) & mask); break;
    case 0x40: store_le(p, sz, old | v); break;
    case 0x50: store_le(p, sz, old & v); break;
    case 0xA0: store_le(p, sz, old ^ v); break;
    case 0xE0: /* XCHG */
        if (!fetch) return OR_EINVAL;
        store_le(p, sz, v);
        break;
    case 0xF0: /* CMPXCHG */
        if (!fetch) return OR_EINVAL;
        if (old == (R[0] & mask)) store_le(p, sz, v);
        R[0] = old;
        fetch = 0;
        break;
    default: return OR_EINVAL;
    }
    if (fetch) R[src] = old;
    return OR_OK;
}

/* ------------------------------------------------------------------ one event */
/* returns OR_OK and sets *ret, or an error */
static int run_one(const uint64_t *insns, uint32_t n, hctx *h, uint8_t *ctx, uint32_t ctx_size, uint64_t budget,
                   uint64_t *ret, uint64_t *count) {
    uint64_t R[11];
    uint8_t stack[STACK_BYTES];
    regions g;
    memset(R, 0, sizeof R);
    memset(stack, 0, sizeof stack);
    g.n = 0;
    g.strict_align = h->strict_align;
    g.defer = h->defer;
    grant(&g, ctx, ctx_size, 0);
    grant(&g, stack, STACK_BYTES, 1);
    h->g = &g;
    R[1] = (uint64_t)(uintptr_t)ctx;
    R[10] = (uint64_t)(uintptr_t)(stack + STACK_BYTES);
    uint64_t steps = 0;
    uint32_t pc = 0;
    for (;;) {
        if (pc >= n) return OR_EFAULT;
        if (++steps > budget) return OR_EBUDGET;
        uint64_t w = insns[pc];
        uint8_t op = (uint8_t)(w & 0xFF);
        int dst = (int)((w >> 8) & 0xF), src = (int)((w >> 12) & 0xF);
        int16_t off = (int16_t)(uint16_t)((w >> 16) & 0xFFFF);
        int32_t imm = (int32_t)(uint32_t)(w >> 32);
        uint8_t cls = op & 7;
        uint32_t next = pc + 1;
        int rc = OR_OK;
        if (dst > 10 || src > 10) return OR_EINVAL;
        switch (cls) {
        case 4: /* ALU */
        case 7: /* ALU64 */
            rc = ins_alu(R, op, dst, src, off, imm);
            break;
        case 5:   /* JMP */
        case 6: { /* JMP32 */
            uint8_t code = op & 0xF0;
            if (code == 0x00) { /* JA */
                next = (uint32_t)((int64_t)pc + 1 + (cls == 6 ? imm : off));
                break;
            }
            if (code == 0x80 && cls == 5) { /* CALL */
                if (src != 0) return OR_EINVAL;
                h->helpers++;
                rc = helper(h, imm, R);
                break;
            }
            if (code == 0x90 && cls == 5) { /* EXIT */
                *ret = R[0];
                *count += steps;
                return OR_OK;
            }
            int taken;
            if (ins_cond(R, op, dst, src, imm, &taken) != OR_OK) return OR_EINVAL;
            if (taken) next = (uint32_t)((int64_t)pc + 1 + off);
            break;
        }
        case 0: /* LD: only the 64-bit immediate form */
            rc = ins_ld64(R, h, insns, n, pc);
            next = pc + 2;
            break;
        case 1: /* LDX */
            h->mem++;
            rc = ins_ldx(R, &g, op, dst, src, off);
            break;
        case 2: /* ST */
        case 3: /* STX */
            h->mem++;
            rc = ins_store(R, &g, op, dst, src, off, imm);
            break;
        default: return OR_EINVAL;
        }
        if (rc != OR_OK) return rc;
        pc = next;
    }
}

/*
 * Run the program over n_events records of ctx_size bytes, sequentially.
 * r0_out (nullable): R0 per event.  insn_count (nullable): total executed instructions
 * (a 64-bit immediate load counts once).  budget: per-event instruction cap (0 = 2^20).
 * Returns 0 or the first error; *bad_event = the index of the event that failed.
 * or_run_flags: OR_STRICT_ALIGN also stops with OR_EFAULT at a load, store or atomic (the
 * max / min helpers included) whose address is not a multiple of its size, the engine's
 * reading that device accesses are naturally aligned; or_run leaves alignment free.
 * most (nullable): the most instructions, helper calls and loads / stores / atomics that
 * one event executed.  defer_mask: bit m defers map m's updates (see "deferred updates").
 */
#define OR_STRICT_ALIGN 1u
/* the deferred updates, in the order they were made */
static void defer_apply(const defer_t *d) {
    for (size_t i = 0; i < d->n; i++) {
        const dop *o = &d->log[i];
        uint64_t mask = o->size == 4 ? 0xFFFFFFFFULL : ~0ULL, old = load_le(o->p, o->size), r = old;
        switch (o->op) {
        case 0x00: r = (old + o->v) & mask; break;
        case 0x40: r = old | o->v; break;
        case 0x50: r = old & o->v; break;
        case 0xA0: r = old ^ o->v; break;
        case DEFER_MAX: r = o->v > old ? o->v : old; break;
        case DEFER_MIN: r = o->v < old ? o->v : old; break;
        }
        store_le(o->p, o->size, r);
    }
}

int or_run_flags(const uint64_t *insns, uint32_t n_insns, or_map **maps, uint32_t n_maps, const uint8_t *events,
                 uint64_t n_events, uint32_t ctx_size, uint64_t event_idx_base, int64_t *r0_out,
                 uint64_t *insn_count, uint64_t budget, uint64_t *bad_event, uint32_t flags, uint64_t *most,
                 uint32_t defer_mask) {
    hctx h;
    memset(&h, 0, sizeof h);
    h.strict_align = (flags & OR_STRICT_ALIGN) != 0;
    defer_t d;
    memset(&d, 0, sizeof d);
    d.mask = defer_mask;
    d.maps = maps;
    d.n_maps = n_maps;
    if (defer_mask) h.defer = &d;
    int rc = OR_OK;
    h.maps = maps;
    h.n_maps = n_maps;
    uint64_t count = 0;
    if (budget == 0) budget = 1ULL << 20;
    if (most) most[0] = most[1] = most[2] = 0;
    for (uint64_t i = 0; i < n_events && rc == OR_OK; i++) {
        uint64_t ret = 0, before = count;
        h.event_idx = event_idx_base + i;
        h.helpers = h.mem = 0;
        rc = run_one(insns, n_insns, &h, (uint8_t *)(uintptr_t)(events + i * (uint64_t)ctx_size), ctx_size,
                     budget, &ret, &count);
        if (rc != OR_OK) {
            if (bad_event) *bad_event = i;
            break;
        }
        if (most) {
            if (count - before > most[0]) most[0] = count - before;
            if (h.helpers > most[1]) most[1] = h.helpers;
            if (h.mem > most[2]) most[2] = h.mem;
        }
        if (r0_out) r0_out[i] = (int64_t)ret;
    }
    if (rc == OR_OK) defer_apply(&d);
    free(d.log);
    if (insn_count) *insn_count = count;
    return rc;
}

int or_run(const uint64_t *insns, uint32_t n_insns, or_map **maps, uint32_t n_maps, const uint8_t *events,
           uint64_t n_events, uint32_t ctx_size, uint64_t event_idx_base, int64_t *r0_out, uint64_t *insn_count,
           uint64_t budget, uint64_t *bad_event) {
    return or_run_flags(insns, n_insns, maps, n_maps, events, n_events, ctx_size, event_idx_base, r0_out, insn_count,
                        budget, bad_event, 0, NULL, 0);
}

/* ------------------------------------------------------------------ one warp, in lockstep */
/*
 * The warp-level execution of device handlers (Sec. 4.4.1, Sec. 4.4.2): the lanes of a
 * warp run the handler together.  Values may differ between lanes, but they may not
 * decide control flow or reach state outside the warp; the warp's side effects happen
 * once, and their results reach every lane.  This is that definition written out: the
 * lanes step in lockstep, and wherever they must agree the run checks that they do.
 * A disagreement stops the run with OR_EDIVERGE at that instruction.
 *
 * Per lane: registers, a 512-byte stack, its own ctx record.  Shared: maps and rings.
 *   - ALU, 64-bit immediates, loads, and stores and atomics on the lane's own stack:
 *     every lane on its own.
 *   - Conditional jumps: every lane evaluates; all must agree.
 *   - Stores and atomics elsewhere (map values, ring-buffer records): every lane names
 *     the same address and operand (and R0 for CMPXCHG); the leader executes it once
 *     and a fetched old value goes to every lane.
 *   - Warp helpers (GX_HELPER_WARP_*, 0x10010..0x10015) reduce R1 over the warp's lanes
 *     into every lane's R0: sum mod 2^64, unsigned max, unsigned min, OR, AND, and the
 *     number of lanes with R1 != 0.
 *   - Other helpers: every argument the helper reads must agree (a pointer into the
 *     lane's own stack or ctx compares by its offset there), and so must the bytes
 *     behind a key, value or payload pointer; the leader calls it once, and R0 and any
 *     region it grants go to every lane.  Atomic max / min on the lane's own stack runs
 *     per lane.
 *   - EXIT: every lane's R0 must agree.
 * The leader is the warp's first lane: ring-buffer records carry its event index.
 */
#define OR_EDIVERGE (-1003)
#define WARP_MAX 32

typedef struct {
    uint64_t R[11];
    uint8_t stack[STACK_BYTES];
    regions g;
    uint8_t *ctx;
} lane;

/* a register value as every lane would see it: pointers into the lane's own stack or ctx by offset */
static void lane_norm(const lane *l, uint32_t ctx_size, uint64_t v, int *kind, uint64_t *x) {
    uint64_t sb = (uint64_t)(uintptr_t)l->stack, cb = (uint64_t)(uintptr_t)l->ctx;
    if (v >= sb && v - sb <= STACK_BYTES) {
        *kind = 1;
        *x = v - sb;
    } else if (v >= cb && v - cb <= ctx_size) {
        *kind = 2;
        *x = v - cb;
    } else {
        *kind = 0;
        *x = v;
    }
}

static int lanes_agree_reg(const lane *L, uint32_t nl, uint32_t ctx_size, int r) {
    int k0, k;
    uint64_t x0, x;
    lane_norm(&L[0], ctx_size, L[0].R[r], &k0, &x0);
    for (uint32_t i = 1; i < nl; i++) {
        lane_norm(&L[i], ctx_size, L[i].R[r], &k, &x);
        if (k != k0 || x != x0) return 0;
    }
    return 1;
}

/* the `size` bytes at each lane's R[r] are readable and the same in every lane; -1 unreadable */
static int lanes_agree_bytes(const lane *L, uint32_t nl, int r, uint64_t size) {
    const uint8_t *p0 = check(&L[0].g, L[0].R[r], size, 0);
    if (!p0) return -1;
    for (uint32_t i = 1; i < nl; i++) {
        const uint8_t *p = check(&L[i].g, L[i].R[r], size, 0);
        if (!p) return -1;
        if (memcmp(p, p0, size)) return 0;
    }
    return 1;
}

static int in_own_stack(const lane *l, uint64_t a) {
    uint64_t sb = (uint64_t)(uintptr_t)l->stack;
    return a >= sb && a - sb < STACK_BYTES;
}

static int helper_nargs(int32_t id) {
    switch (id) {
    case 1: case 3: case 132: case 133: case 0x10000: case 0x10001: return 2;
    case 2: case 130: return 4;
    case 131: return 3;
    }
    return 0;
}

/* a helper call by the whole warp */
static int warp_call(hctx *h, lane *L, uint32_t nl, uint32_t ctx_size, int32_t id) {
    if (id >= 0x10010 && id <= 0x10015) { /* warp helpers: a reduction over the lanes */
        uint64_t acc = id == 0x10012 || id == 0x10014 ? ~0ULL : 0;
        for (uint32_t i = 0; i < nl; i++) {
            uint64_t v = L[i].R[1];
            switch (id) {
            case 0x10010: acc += v; break;
            case 0x10011: if (v > acc) acc = v; break;
            case 0x10012: if (v < acc) acc = v; break;
            case 0x10013: acc |= v; break;
            case 0x10014: acc &= v; break;
            case 0x10015: acc += v != 0; break;
            }
        }
        for (uint32_t i = 0; i < nl; i++) {
            L[i].R[0] = acc;
            for (int r = 1; r <= 5; r++) L[i].R[r] = 0;
        }
        return OR_OK;
    }
    if ((id == 0x10000 || id == 0x10001) && in_own_stack(&L[0], L[0].R[1])) { /* lane-private memory */
        for (uint32_t i = 0; i < nl; i++) {
            if (!in_own_stack(&L[i], L[i].R[1])) return OR_EDIVERGE;
            h->g = &L[i].g;
            int rc = helper(h, id, L[i].R);
            if (rc != OR_OK) return rc;
        }
        return OR_OK;
    }
    for (int r = 1; r <= helper_nargs(id); r++)
        if (!lanes_agree_reg(L, nl, ctx_size, r)) return OR_EDIVERGE;
    or_map *m = map_arg(h, L[0].R[1]);
    if (m && m->type != MAP_RINGBUF && (id == 1 || id == 2 || id == 3)) {
        int a = lanes_agree_bytes(L, nl, 2, m->key_size);
        if (a == 1 && id == 2) a = lanes_agree_bytes(L, nl, 3, m->value_size);
        if (a < 0) return OR_EFAULT;
        if (a == 0) return OR_EDIVERGE;
    }
    if (m && m->type == MAP_RINGBUF && id == 130 && L[0].R[3] <= 4096) {
        int a = lanes_agree_bytes(L, nl, 2, L[0].R[3]);
        if (a < 0) return OR_EFAULT;
        if (a == 0) return OR_EDIVERGE;
    }
    h->g = &L[0].g;
    h->granted.size = 0;
    int rc = helper(h, id, L[0].R);
    if (rc != OR_OK) return rc;
    for (uint32_t i = 1; i < nl; i++) {
        if (h->granted.size) grant(&L[i].g, h->granted.base, h->granted.size, h->granted.writable);
        L[i].R[0] = L[0].R[0];
        for (int r = 1; r <= 5; r++) L[i].R[r] = 0;
    }
    return OR_OK;
}

/* a store or atomic by the whole warp */
static int warp_store(lane *L, uint32_t nl, uint8_t op, int dst, int src, int16_t off, int32_t imm) {
    uint8_t cls = op & 7, mode = op & 0xE0;
    int own = in_own_stack(&L[0], store_addr(L[0].R, dst, off));
    for (uint32_t i = 1; i < nl; i++)
        if (in_own_stack(&L[i], store_addr(L[i].R, dst, off)) != own) return OR_EDIVERGE;
    if (own) {
        for (uint32_t i = 0; i < nl; i++) {
            int rc = ins_store(L[i].R, &L[i].g, op, dst, src, off, imm);
            if (rc != OR_OK) return rc;
        }
        return OR_OK;
    }
    /* outside the lanes' stacks: one address, one operand, executed once */
    uint64_t a = store_addr(L[0].R, dst, off);
    int cmpx = mode == 0xC0 && imm == 0xF1;
    for (uint32_t i = 1; i < nl; i++) {
        if (store_addr(L[i].R, dst, off) != a) return OR_EDIVERGE;
        if (cls == 3 && L[i].R[src] != L[0].R[src]) return OR_EDIVERGE;
        if (cmpx && L[i].R[0] != L[0].R[0]) return OR_EDIVERGE;
        if (!check(&L[i].g, a, (uint64_t)size_of(op), 1)) return OR_EFAULT;
    }
    int rc = ins_store(L[0].R, &L[0].g, op, dst, src, off, imm);
    if (rc != OR_OK) return rc;
    if (mode == 0xC0)
        for (uint32_t i = 1; i < nl; i++) {
            if (cmpx) L[i].R[0] = L[0].R[0];
            else if (imm & 1) L[i].R[src] = L[0].R[src];
        }
    return OR_OK;
}

static int run_warp(const uint64_t *insns, uint32_t n, hctx *h, lane *L, uint32_t nl, uint32_t ctx_size,
                    uint64_t budget, uint64_t *ret, uint64_t *count, uint32_t *bad_pc) {
    for (uint32_t i = 0; i < nl; i++) {
        memset(L[i].R, 0, sizeof L[i].R);
        memset(L[i].stack, 0, sizeof L[i].stack);
        L[i].g.n = 0;
        L[i].g.strict_align = h->strict_align;
        L[i].g.defer = NULL;
        grant(&L[i].g, L[i].ctx, ctx_size, 0);
        grant(&L[i].g, L[i].stack, STACK_BYTES, 1);
        L[i].R[1] = (uint64_t)(uintptr_t)L[i].ctx;
        L[i].R[10] = (uint64_t)(uintptr_t)(L[i].stack + STACK_BYTES);
    }
    uint64_t steps = 0;
    uint32_t pc = 0;
    for (;;) {
        *bad_pc = pc;
        if (pc >= n) return OR_EFAULT;
        if (++steps > budget) return OR_EBUDGET;
        uint64_t w = insns[pc];
        uint8_t op = (uint8_t)(w & 0xFF);
        int dst = (int)((w >> 8) & 0xF), src = (int)((w >> 12) & 0xF);
        int16_t off = (int16_t)(uint16_t)((w >> 16) & 0xFFFF);
        int32_t imm = (int32_t)(uint32_t)(w >> 32);
        uint8_t cls = op & 7;
        uint32_t next = pc + 1;
        int rc = OR_OK;
        if (dst > 10 || src > 10) return OR_EINVAL;
        switch (cls) {
        case 4:
        case 7:
            for (uint32_t i = 0; i < nl && rc == OR_OK; i++) rc = ins_alu(L[i].R, op, dst, src, off, imm);
            break;
        case 5:
        case 6: {
            uint8_t code = op & 0xF0;
            if (code == 0x00) {
                next = (uint32_t)((int64_t)pc + 1 + (cls == 6 ? imm : off));
                break;
            }
            if (code == 0x80 && cls == 5) {
                if (src != 0) return OR_EINVAL;
                rc = warp_call(h, L, nl, ctx_size, imm);
                break;
            }
            if (code == 0x90 && cls == 5) {
                for (uint32_t i = 1; i < nl; i++)
                    if (L[i].R[0] != L[0].R[0]) return OR_EDIVERGE;
                for (uint32_t i = 0; i < nl; i++) ret[i] = L[i].R[0];
                *count += steps;
                return OR_OK;
            }
            int t0 = 0, t;
            for (uint32_t i = 0; i < nl; i++) {
                if (ins_cond(L[i].R, op, dst, src, imm, &t) != OR_OK) return OR_EINVAL;
                if (i == 0) t0 = t;
                else if (t != t0) return OR_EDIVERGE;
            }
            if (t0) next = (uint32_t)((int64_t)pc + 1 + off);
            break;
        }
        case 0:
            for (uint32_t i = 0; i < nl && rc == OR_OK; i++) rc = ins_ld64(L[i].R, h, insns, n, pc);
            next = pc + 2;
            break;
        case 1:
            for (uint32_t i = 0; i < nl && rc == OR_OK; i++) rc = ins_ldx(L[i].R, &L[i].g, op, dst, src, off);
            break;
        case 2:
        case 3:
            rc = warp_store(L, nl, op, dst, src, off, imm);
            break;
        default: return OR_EINVAL;
        }
        if (rc != OR_OK) return rc;
        pc = next;
    }
}

/*
 * Run the program over n_events records as warps of `lanes` consecutive events (1..32;
 * the last warp may be shorter), one warp after another (see run_warp above).  uniform
 * (nullable): ctx_size flags, nonzero marking a warp-uniform ctx byte; every lane of a
 * warp must carry the same value there (else OR_EINVAL for that warp).  r0_out, insn_count
 * (instructions per warp, summed), budget: as or_run.  Returns 0 or the first error with
 * *bad_event = the first event of the failing warp and *bad_pc = the instruction.
 */
int or_run_warps(const uint64_t *insns, uint32_t n_insns, or_map **maps, uint32_t n_maps, const uint8_t *events,
                 uint64_t n_events, uint32_t ctx_size, const uint8_t *uniform, uint32_t lanes, uint64_t event_idx_base,
                 int64_t *r0_out, uint64_t *insn_count, uint64_t budget, uint64_t *bad_event, uint32_t *bad_pc) {
    if (lanes < 1 || lanes > WARP_MAX) return OR_EINVAL;
    lane *L = (lane *)calloc(WARP_MAX, sizeof(lane));
    if (!L) return OR_ENOMEM;
    hctx h;
    memset(&h, 0, sizeof h);
    h.maps = maps;
    h.n_maps = n_maps;
    uint64_t count = 0, ret[WARP_MAX];
    uint32_t pc = 0;
    if (budget == 0) budget = 1ULL << 20;
    int rc = OR_OK;
    for (uint64_t w0 = 0; w0 < n_events && rc == OR_OK; w0 += lanes) {
        uint32_t nl = (uint32_t)(n_events - w0 < lanes ? n_events - w0 : lanes);
        for (uint32_t i = 0; i < nl; i++) L[i].ctx = (uint8_t *)(uintptr_t)(events + (w0 + i) * (uint64_t)ctx_size);
        for (uint32_t b = 0; uniform && b < ctx_size && rc == OR_OK; b++)
            for (uint32_t i = 1; uniform[b] && i < nl; i++)
                if (L[i].ctx[b] != L[0].ctx[b]) rc = OR_EINVAL;
        h.event_idx = event_idx_base + w0;
        if (rc == OR_OK) rc = run_warp(insns, n_insns, &h, L, nl, ctx_size, budget, ret, &count, &pc);
        if (rc != OR_OK) {
            if (bad_event) *bad_event = w0;
            if (bad_pc) *bad_pc = pc;
        } else if (r0_out) {
            for (uint32_t i = 0; i < nl; i++) r0_out[w0 + i] = (int64_t)ret[i];
        }
    }
    free(L);
    if (insn_count) *insn_count = count;
    return rc;
}
