/*
 * The engine's host code that parses untrusted bytecode (verifier.cpp, decode.cpp), built
 * with AddressSanitizer and UndefinedBehaviorSanitizer by tests/test_host_sanitize.py and
 * run over a corpus of programs and seeded mutants of them.  Each program is verified
 * per lane (plain and deterministic) and in SIMT mode (random uniform ctx words and
 * budgets), and every accepted one is decoded.  A memory error or undefined behaviour
 * aborts with the sanitizer's report; a clean run prints "OK" and the counts.
 *
 * Corpus (little-endian): "GXCP", u32 count, then per program u32 n_insns, u32 n_maps,
 * u32 ctx_size, u32 0, n_maps x gx_map_spec (6 x u32), n_insns x u64.
 */
#include <stdio.h>
#include <string.h>

#include <random>
#include <string>
#include <vector>

#include "gx_internal.h"

struct Prog {
    std::vector<uint64_t> insns;
    std::vector<gx_map_spec> maps;
    uint32_t ctx_size = 8;
};

static bool read_corpus(const char *path, std::vector<Prog> &out) {
    FILE *f = fopen(path, "rb");
    if (!f) return false;
    char magic[4];
    uint32_t count = 0;
    bool ok = fread(magic, 1, 4, f) == 4 && memcmp(magic, "GXCP", 4) == 0 && fread(&count, 4, 1, f) == 1;
    for (uint32_t i = 0; ok && i < count; i++) {
        uint32_t h[4];
        ok = fread(h, 4, 4, f) == 4 && h[0] <= GX_MAX_INSNS && h[1] <= GX_MAX_MAPS;
        if (!ok) break;
        Prog p;
        p.ctx_size = h[2];
        p.maps.resize(h[1]);
        p.insns.resize(h[0]);
        ok = (h[1] == 0 || fread(p.maps.data(), sizeof(gx_map_spec), h[1], f) == h[1]) &&
             (h[0] == 0 || fread(p.insns.data(), 8, h[0], f) == h[0]);
        if (ok) out.push_back(std::move(p));
    }
    fclose(f);
    return ok;
}

/* a seeded mutant: a few bit flips, a random word, a duplicated or dropped instruction */
static std::vector<uint64_t> mutate(const std::vector<uint64_t> &in, std::mt19937_64 &rng) {
    std::vector<uint64_t> v = in;
    if (v.empty()) return v;
    const int kind = (int)(rng() % 4);
    const size_t at = rng() % v.size();
    switch (kind) {
    case 0:
        for (int k = 0; k < 1 + (int)(rng() % 3); k++) v[rng() % v.size()] ^= 1ull << (rng() % 64);
        break;
    case 1: v[at] = rng(); break;
    case 2:
        if (v.size() < GX_MAX_INSNS) v.insert(v.begin() + (long)at, v[at]);
        break;
    default:
        v.erase(v.begin() + (long)at);
        break;
    }
    return v;
}

int main(int argc, char **argv) {
    if (argc < 3) return 2;
    std::vector<Prog> corpus;
    if (!read_corpus(argv[1], corpus)) {
        printf("bad corpus\n");
        return 2;
    }
    const int mutants = atoi(argv[2]);
    std::mt19937_64 rng(0x5eed);
    unsigned runs = 0, accepted = 0, simt_accepted = 0;
    for (const Prog &p : corpus) {
        for (int m = 0; m <= mutants; m++) {
            const std::vector<uint64_t> insns = m ? mutate(p.insns, rng) : p.insns;
            for (uint32_t det = 0; det < 2; det++) {
                gx_prog_opts opts;
                memset(&opts, 0, sizeof opts);
                opts.ctx_size = p.ctx_size;
                opts.deterministic = det;
                opts.insn_budget = 1u << 12;
                gx::VerifyOut v;
                const int rc = gx::verify_program(insns.data(), (uint32_t)insns.size(), p.maps.data(),
                                                  (uint32_t)p.maps.size(), opts, v);
                runs++;
                if (rc != GX_OK) continue;
                accepted++;
                std::vector<uint64_t> uops;
                std::string log;
                gx::decode_program(insns.data(), (uint32_t)insns.size(), v, uops, log);
            }
            gx::SimtIn in;
            in.uniform.assign(p.ctx_size, 0);
            for (uint32_t w = 0; w * 8 < p.ctx_size; w++) {
                const uint8_t u = (uint8_t)(rng() & 1);
                for (uint32_t b = w * 8; b < p.ctx_size && b < w * 8 + 8; b++) in.uniform[b] = u;
            }
            if (rng() & 1) {
                in.max_insns = (uint32_t)(rng() % 64);
                in.max_helpers = (uint32_t)(rng() % 4);
                in.max_mem = (uint32_t)(rng() % 16);
            }
            gx_prog_opts opts;
            memset(&opts, 0, sizeof opts);
            opts.ctx_size = p.ctx_size;
            opts.deterministic = (uint32_t)(rng() & 1);
            gx::VerifyOut v;
            if (gx::verify_program(insns.data(), (uint32_t)insns.size(), p.maps.data(), (uint32_t)p.maps.size(), opts,
                                   v, &in) == GX_OK)
                simt_accepted++;
            runs++;
        }
    }
    printf("OK runs=%u accepted=%u simt_accepted=%u\n", runs, accepted, simt_accepted);
    return 0;
}
