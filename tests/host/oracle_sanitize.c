/*
 * The oracle built with AddressSanitizer and UndefinedBehaviorSanitizer by
 * tests/test_host_sanitize.py and run over a corpus of programs and seeded mutants of them,
 * verified or not: the oracle checks every memory access itself, so it must stay safe on
 * any program.  Each program runs on fresh maps over random events per event (plain and
 * strict-alignment) and as warps (random uniform ctx words).  A memory error or undefined
 * behaviour aborts with the sanitizer's report; a clean run prints "OK" and the counts.
 *
 * Corpus: as tests/host/verify_sanitize.cpp reads it.
 */
#include "../../oracle/gx_oracle.c"

#include <stdio.h>

typedef struct {
    uint32_t type, key_size, value_size, max_entries, flags, reserved;
} spec_t;

static uint64_t rng_state = 0x0dd5eedull;
static uint64_t next_rand(void) { /* splitmix64 */
    uint64_t z = (rng_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void mutate(uint64_t *v, uint32_t *n) {
    if (*n == 0) return;
    const uint32_t at = (uint32_t)(next_rand() % *n);
    switch (next_rand() % 3) {
    case 0: v[at] ^= 1ull << (next_rand() % 64); break;
    case 1: v[at] = next_rand(); break;
    default:
        memmove(v + at, v + at + 1, (size_t)(*n - at - 1) * 8);
        (*n)--;
        break;
    }
}

static int run_program(const uint64_t *insns, uint32_t n, const spec_t *specs, uint32_t n_maps, uint32_t ctx) {
    or_map *maps[16];
    uint32_t made = 0;
    int ok = 1;
    for (; made < n_maps; made++) {
        maps[made] = or_map_create(specs[made].type, specs[made].key_size, specs[made].value_size,
                                   specs[made].max_entries);
        if (!maps[made]) {
            ok = 0;
            break;
        }
    }
    if (ok) {
        enum { EV = 64 };
        uint8_t *ev = (uint8_t *)malloc((size_t)EV * ctx);
        int64_t r0[EV];
        uint8_t uni[256];
        for (uint32_t i = 0; i < EV * ctx; i++) ev[i] = (uint8_t)(next_rand() & ((i & 8) ? 0xFF : 0x0F));
        for (uint32_t w = 0; w * 8 < ctx; w++) {
            const uint8_t u = (uint8_t)(next_rand() & 1);
            for (uint32_t b = w * 8; b < ctx && b < w * 8 + 8; b++) uni[b] = u;
        }
        uint64_t count = 0, bad = 0, most[3];
        uint32_t bad_pc = 0;
        or_run_flags(insns, n, maps, n_maps, ev, 16, ctx, 0, r0, &count, 1u << 12, &bad, 0, most, 0);
        or_run_flags(insns, n, maps, n_maps, ev, 16, ctx, 16, r0, &count, 1u << 12, &bad, OR_STRICT_ALIGN, most, 0);
        or_run_warps(insns, n, maps, n_maps, ev, EV, ctx, uni, 32, 0, r0, &count, 1u << 12, &bad, &bad_pc);
        free(ev);
    }
    for (uint32_t i = 0; i < made; i++) or_map_destroy(maps[i]);
    return ok;
}

int main(int argc, char **argv) {
    if (argc < 3) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    const int mutants = atoi(argv[2]);
    char magic[4];
    uint32_t count = 0, runs = 0;
    if (fread(magic, 1, 4, f) != 4 || memcmp(magic, "GXCP", 4) != 0 || fread(&count, 4, 1, f) != 1) return 2;
    static uint64_t insns[4096], work[4096];
    spec_t specs[16];
    for (uint32_t p = 0; p < count; p++) {
        uint32_t h[4];
        if (fread(h, 4, 4, f) != 4 || h[0] > 4096 || h[1] > 16 || h[2] < 8 || h[2] > 256) return 2;
        if ((h[1] && fread(specs, sizeof(spec_t), h[1], f) != h[1]) || (h[0] && fread(insns, 8, h[0], f) != h[0]))
            return 2;
        for (int m = 0; m <= mutants; m++) {
            uint32_t n = h[0];
            memcpy(work, insns, (size_t)n * 8);
            if (m) mutate(work, &n);
            run_program(work, n, specs, h[1], h[2]);
            runs++;
        }
    }
    fclose(f);
    printf("OK runs=%u\n", runs);
    return 0;
}
