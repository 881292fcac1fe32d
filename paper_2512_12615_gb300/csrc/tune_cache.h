/*
 * The autotuner's choices on disk (GX_TUNE_CACHE=<dir>): one small text file per
 * (program, size bucket, device, engine build), so that a later process running the same
 * program at the same size on the same kind of GPU reuses the choice instead of timing
 * the candidates again.  Host-only and header-only; gx_autotune uses it, and
 * tests/host/tune_cache_check.cpp checks it without a device.
 *
 * A record is one line: "gx-tune 1 <block> <ept> <grid> <shards> <variant>".  A file that
 * is missing, truncated, from another format version or holding a shape the engine would
 * refuse is ignored (the tuner then runs as without a cache).  Files are written to a
 * temporary name and renamed, so readers never see half a record.
 */
#ifndef GX_TUNE_CACHE_H
#define GX_TUNE_CACHE_H

#include <stdint.h>
#include <stdio.h>
#include <string.h>
#include <sys/stat.h>
#include <unistd.h>

#include <string>

#include "../../include/gx.h"

namespace gx {

/* FNV-1a (64-bit) over bytes, chained: start from the offset basis, or from an earlier hash */
inline uint64_t tune_fnv(const void *data, size_t n, uint64_t h = 0xcbf29ce484222325ull) {
    const uint8_t *p = (const uint8_t *)data;
    for (size_t i = 0; i < n; i++) {
        h ^= p[i];
        h *= 0x100000001b3ull; /* the 64-bit FNV prime */
    }
    return h;
}

/* file name of a record: the identity hash and the size bucket, in hex and decimal */
inline std::string tune_cache_path(const std::string &dir, uint64_t identity, int bucket, bool policy_only) {
    char name[64];
    snprintf(name, sizeof name, "/%016llx-%02d%s.tune", (unsigned long long)identity, bucket, policy_only ? "p" : "");
    return dir + name;
}

/* a shape the engine accepts (gx_run_batch_ex's checks, before the device ones) */
inline bool tune_shape_valid(const gx_launch &l) {
    const uint32_t w = l.shards & 0xFFu;
    const bool shards_ok =
        l.shards == GX_SHARDS_OFF || ((l.shards & ~(0xFFu | GX_SHARDS_AGG)) == 0 && (w == 0 || (w >= 2 && w <= 10)));
    return l.block >= 64 && l.block <= 256 && l.block % 32 == 0 && l.ept >= 1 && l.ept <= 64 && l.reserved == 0 &&
           l.variant <= GX_VARIANT_4 && shards_ok;
}

inline bool tune_cache_load(const std::string &path, gx_launch *out) {
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return false;
    char line[128] = {0};
    const bool got = fgets(line, sizeof line, f) != nullptr;
    fclose(f);
    if (!got) return false;
    unsigned v = 0, b = 0, e = 0, g = 0, s = 0, var = 0;
    char tail = 0;
    if (sscanf(line, "gx-tune %u %u %u %u %u %u%c", &v, &b, &e, &g, &s, &var, &tail) < 6 || v != 1) return false;
    if (tail != 0 && tail != '\n') return false;
    gx_launch l;
    memset(&l, 0, sizeof l);
    l.block = b;
    l.ept = e;
    l.grid = g;
    l.shards = s;
    l.variant = var;
    if (!tune_shape_valid(l)) return false;
    *out = l;
    return true;
}

inline bool tune_cache_store(const std::string &path, const gx_launch &l) {
    if (!tune_shape_valid(l)) return false;
    const std::string tmp = path + ".tmp" + std::to_string((long)getpid());
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return false;
    const bool ok = fprintf(f, "gx-tune 1 %u %u %u %u %u\n", l.block, l.ept, l.grid, l.shards, l.variant) > 0;
    if (fclose(f) != 0 || !ok || rename(tmp.c_str(), path.c_str()) != 0) {
        remove(tmp.c_str());
        return false;
    }
    return true;
}

} // namespace gx

#endif
