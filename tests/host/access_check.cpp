/*
 * Host check of the checked interpreter's region tests (gx_layout.h: gx_value_bytes,
 * gx_range_ok, gx_access_ok): every edge of the stack and of each kind of map region,
 * misalignment, empty and wrapping ranges.  Prints OK or the failing line.
 */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "gx_layout.h"

static int fails = 0;
#define CHECK(c)                                            \
    do {                                                    \
        if (!(c)) {                                         \
            printf("FAIL line %d: %s\n", __LINE__, #c);     \
            fails++;                                        \
        }                                                   \
    } while (0)

int main() {
    gx_dmap m[3];
    memset(m, 0, sizeof m);
    m[0].type = 2; /* array: 4 entries of stride 8 -> 32 bytes */
    m[0].max_entries = 4;
    m[0].vstride = 8;
    m[0].values = (uint8_t *)(uintptr_t)0x100000;
    m[1].type = 1; /* hash: 8 slots (mask 7) of stride 16 -> 128 bytes of values */
    m[1].max_entries = 3;
    m[1].mask = 7;
    m[1].vstride = 16;
    m[1].values = (uint8_t *)(uintptr_t)0x200000;
    m[2].type = 27; /* ring buffer: 4096 data bytes */
    m[2].mask = 4096;
    m[2].values = (uint8_t *)(uintptr_t)0x300000;
    const uint64_t stk = 0x400000;
    const uint32_t sb = 512;

    CHECK(gx_value_bytes(&m[0]) == 32 && gx_value_bytes(&m[1]) == 128 && gx_value_bytes(&m[2]) == 4096);
    /* the stack: [stk, stk + 512) */
    CHECK(gx_access_ok(m, 3, stk, sb, stk, 8));
    CHECK(gx_access_ok(m, 3, stk, sb, stk + 504, 8));
    CHECK(!gx_access_ok(m, 3, stk, sb, stk + 505, 8));  /* misaligned */
    CHECK(!gx_access_ok(m, 3, stk, sb, stk + 508, 8));  /* straddles the end, and misaligned */
    CHECK(gx_access_ok(m, 3, stk, sb, stk + 511, 1));
    CHECK(!gx_access_ok(m, 3, stk, sb, stk + 512, 1));  /* one past the end */
    CHECK(!gx_access_ok(m, 3, stk, sb, stk - 1, 1));    /* one before */
    CHECK(!gx_access_ok(m, 3, stk, sb, stk + 2, 4));    /* misaligned */
    CHECK(gx_access_ok(m, 3, stk, sb, stk + 2, 2));
    /* the array's values: [0x100000, 0x100020) */
    CHECK(gx_access_ok(m, 3, stk, sb, 0x100018, 8));
    CHECK(!gx_access_ok(m, 3, stk, sb, 0x100020, 1));
    CHECK(!gx_access_ok(m, 3, stk, sb, 0x100020 - 4, 8)); /* misaligned and past the end */
    CHECK(gx_access_ok(m, 3, stk, sb, 0x10001C, 4));
    /* the hash map's values: [0x200000, 0x200080) */
    CHECK(gx_access_ok(m, 3, stk, sb, 0x200078, 8));
    CHECK(!gx_access_ok(m, 3, stk, sb, 0x200080, 8));
    /* the ring's data: [0x300000, 0x301000) */
    CHECK(gx_access_ok(m, 3, stk, sb, 0x300FF8, 8));
    CHECK(!gx_access_ok(m, 3, stk, sb, 0x301000, 4));
    /* a region a map does not own, and maps left out of the count */
    CHECK(!gx_access_ok(m, 3, stk, sb, 0x250000, 8));
    CHECK(!gx_access_ok(m, 2, stk, sb, 0x300000, 8));
    CHECK(!gx_access_ok(m, 0, stk, sb, 0x100000, 8));
    /* ranges (helper buffers): no alignment, no empty range, no wrap-around */
    CHECK(gx_range_ok(m, 3, stk, sb, stk + 505, 7));
    CHECK(!gx_range_ok(m, 3, stk, sb, stk + 505, 8));
    CHECK(!gx_range_ok(m, 3, stk, sb, stk, 0));
    CHECK(!gx_range_ok(m, 3, stk, sb, ~(uint64_t)0 - 3, 8));
    CHECK(gx_range_ok(m, 3, stk, sb, 0x100001, 31));
    CHECK(!gx_range_ok(m, 3, stk, sb, 0x100001, 32));
    if (fails) return 1;
    printf("OK\n");
    return 0;
}
