/*
 * Host-only checks of the autotuner's on-disk cache (csrc/tune_cache.h): the FNV-1a hash
 * against published test vectors, the record round trip, and that every malformed or
 * refused record is ignored rather than used.  Run in a scratch directory given as argv[1]
 * by tests/test_host_tune_cache.py.  Prints OK or the failed checks.
 */
#include "tune_cache.h"

#include <dirent.h>

static int fails = 0;
#define CHECK(c)                                                          \
    do {                                                                  \
        if (!(c)) {                                                       \
            printf("FAIL line %d: %s\n", __LINE__, #c);                   \
            fails++;                                                      \
        }                                                                 \
    } while (0)

static void write(const std::string &path, const char *text) {
    FILE *f = fopen(path.c_str(), "w");
    if (f) {
        fputs(text, f);
        fclose(f);
    }
}

int main(int argc, char **argv) {
    if (argc < 2) return 2;
    const std::string dir = argv[1];
    /* FNV-1a 64: the offset basis for no bytes; published vectors for "a" and "foobar" */
    CHECK(gx::tune_fnv("", 0) == 0xcbf29ce484222325ull);
    CHECK(gx::tune_fnv("a", 1) == 0xaf63dc4c8601ec8cull);
    CHECK(gx::tune_fnv("foobar", 6) == 0x85944171f73967e8ull);
    CHECK(gx::tune_fnv("bar", 3, gx::tune_fnv("foo", 3)) == gx::tune_fnv("foobar", 6)); /* chaining */

    const std::string p = gx::tune_cache_path(dir, 0x0123456789abcdefull, 26, false);
    CHECK(p == dir + "/0123456789abcdef-26.tune");
    CHECK(gx::tune_cache_path(dir, 1, 7, true) == dir + "/0000000000000001-07p.tune");

    gx_launch l = {256, 8, 0, 8 | GX_SHARDS_AGG, GX_VARIANT_CAPPED, 0}, r;
    CHECK(gx::tune_cache_store(p, l));
    memset(&r, 0xFF, sizeof r);
    CHECK(gx::tune_cache_load(p, &r));
    CHECK(memcmp(&l, &r, sizeof l) == 0);
    gx_launch off = {128, 2, 0, GX_SHARDS_OFF, GX_VARIANT_WIDE, 0};
    CHECK(gx::tune_cache_store(p, off) && gx::tune_cache_load(p, &r) && memcmp(&off, &r, sizeof off) == 0);
    /* no temporary file is left behind */
    unsigned files = 0;
    if (DIR *d = opendir(dir.c_str())) {
        while (dirent *e = readdir(d)) files += e->d_name[0] != '.';
        closedir(d);
    }
    CHECK(files == 1);

    /* refused shapes are neither stored nor loaded */
    const gx_launch bad[] = {{48, 4, 0, 0, 0, 0},   {256, 0, 0, 0, 0, 0},  {256, 65, 0, 0, 0, 0},
                             {256, 4, 0, 1, 0, 0},   {256, 4, 0, 11, 0, 0}, {256, 4, 0, 0x200, 0, 0},
                             {256, 4, 0, 0, 5, 0},   {256, 4, 0, 0, 0, 1},  {100, 4, 0, 0, 0, 0}};
    for (const gx_launch &b : bad) CHECK(!gx::tune_shape_valid(b) && !gx::tune_cache_store(dir + "/bad.tune", b));
    const char *garbled[] = {"", "gx-tune 2 256 8 0 8 2\n", "gx-tune 1 256 8 0\n", "gx-tune 1 48 8 0 8 2\n",
                             "gx-tune 1 256 8 0 8 2 extra\n", "tune 1 256 8 0 8 2\n", "gx-tune 1 256 8 0 8 9\n"};
    for (const char *g : garbled) {
        write(dir + "/g.tune", g);
        memset(&r, 0, sizeof r);
        CHECK(!gx::tune_cache_load(dir + "/g.tune", &r));
    }
    CHECK(!gx::tune_cache_load(dir + "/missing.tune", &r));
    if (fails) return 1;
    printf("OK\n");
    return 0;
}
