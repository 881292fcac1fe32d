/*
 * The load-time code generator (jit.cpp: jit_source) built with AddressSanitizer and
 * UndefinedBehaviorSanitizer by tests/test_host_sanitize.py and run over the corpus that
 * tests/host/verify_sanitize.cpp reads, with seeded mutants.  Every program the verifier
 * accepts is generated as per-lane code, in groups of three as one multi-program kernel,
 * and with a scheduling program as the work-stealing kernel; every program SIMT
 * verification accepts is generated in the warp-level form.  Each source must balance its
 * braces and parentheses.  Nothing is compiled or run on a device.  Prints "OK" and the
 * counts, or the failed checks.
 */
#include <stdio.h>
#include <string.h>

#include <random>
#include <string>
#include <vector>

#include "gx_jit.h"

namespace gx {
std::string jit_source(const std::vector<const JitProgram *> &progs, std::string &log, int &rc,
                       const JitProgram *sched);
}

static int fails = 0;
#define CHECK(c)                                                  \
    do {                                                          \
        if (!(c)) {                                               \
            if (fails < 20) printf("FAIL line %d: %s\n", __LINE__, #c); \
            fails++;                                              \
        }                                                         \
    } while (0)

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

static std::vector<uint64_t> mutate(const std::vector<uint64_t> &in, std::mt19937_64 &rng) {
    std::vector<uint64_t> v = in;
    if (v.empty()) return v;
    const size_t at = rng() % v.size();
    switch (rng() % 3) {
    case 0: v[at] ^= 1ull << (rng() % 64); break;
    case 1: v[at] = rng(); break;
    default: v.erase(v.begin() + (long)at); break;
    }
    return v;
}

static void check_source(const std::string &src) {
    long braces = 0, parens = 0;
    bool neg = false;
    for (char c : src) {
        braces += c == '{' ? 1 : c == '}' ? -1 : 0;
        parens += c == '(' ? 1 : c == ')' ? -1 : 0;
        neg = neg || braces < 0 || parens < 0;
    }
    CHECK(braces == 0 && parens == 0 && !neg);
    CHECK(src.find("__global__") != std::string::npos);
}

static gx::JitProgram jit_program(const std::vector<uint64_t> &insns, const Prog &p, const gx::VerifyOut &v,
                                  bool warp) {
    gx::JitProgram jp;
    jp.insns = insns;
    jp.info = v.info;
    jp.maps = p.maps;
    jp.use = v.map_use;
    jp.ctx_size = p.ctx_size;
    jp.warp = warp;
    return jp;
}

int main(int argc, char **argv) {
    if (argc < 3) return 2;
    std::vector<Prog> corpus;
    if (!read_corpus(argv[1], corpus)) {
        printf("bad corpus\n");
        return 2;
    }
    const int mutants = atoi(argv[2]);
    /* optional "part of": this run takes programs part, part + of, ... (runs in parallel) */
    const unsigned part = argc > 4 ? (unsigned)atoi(argv[3]) : 0u, of = argc > 4 ? (unsigned)atoi(argv[4]) : 1u;
    std::mt19937_64 rng(0x11e7 + part);
    /* the scheduling program: the first one in the corpus that qualifies */
    gx::JitProgram hook;
    bool have_hook = false;
    for (const Prog &p : corpus) {
        gx_prog_opts o;
        memset(&o, 0, sizeof o);
        o.ctx_size = p.ctx_size;
        gx::VerifyOut v;
        if (p.ctx_size == GX_SCHED_CTX && gx::check_sched_program(p.insns.data(), (uint32_t)p.insns.size(),
                                                                   p.maps.data(), (uint32_t)p.maps.size(), o,
                                                                   nullptr, v) == GX_OK) {
            hook = jit_program(p.insns, p, v, false);
            have_hook = true;
            break;
        }
    }
    CHECK(have_hook);
    unsigned lane = 0, warp = 0, multi = 0, sched = 0;
    std::vector<gx::JitProgram> group;
    for (size_t pi = part; pi < corpus.size(); pi += of) {
        const Prog &p = corpus[pi];
        for (int m = 0; m <= mutants; m++) {
            const std::vector<uint64_t> insns = m ? mutate(p.insns, rng) : p.insns;
            gx_prog_opts opts;
            memset(&opts, 0, sizeof opts);
            opts.ctx_size = p.ctx_size;
            opts.deterministic = (uint32_t)(rng() & 1);
            gx::VerifyOut v;
            if (gx::verify_program(insns.data(), (uint32_t)insns.size(), p.maps.data(), (uint32_t)p.maps.size(), opts,
                                   v) == GX_OK) {
                gx::JitProgram jp = jit_program(insns, p, v, false);
                std::string log;
                int rc = 0;
                std::string src = gx::jit_source({&jp}, log, rc, nullptr);
                if (rc == GX_OK) check_source(src);
                lane++;
                if (have_hook && (rng() & 3) == 0) {
                    src = gx::jit_source({&jp}, log, rc, &hook);
                    if (rc == GX_OK) check_source(src);
                    sched++;
                }
                group.push_back(std::move(jp));
                if (group.size() == 3) {
                    src = gx::jit_source({&group[0], &group[1], &group[2]}, log, rc, nullptr);
                    if (rc == GX_OK) check_source(src);
                    group.clear();
                    multi++;
                }
            }
            gx::SimtIn in;
            in.uniform.assign(p.ctx_size, 0);
            for (uint32_t w = 0; w * 8 < p.ctx_size; w++) {
                const uint8_t u = (uint8_t)((rng() % 4) != 0);
                for (uint32_t b = w * 8; b < p.ctx_size && b < w * 8 + 8; b++) in.uniform[b] = u;
            }
            gx::VerifyOut sv;
            if (gx::verify_program(insns.data(), (uint32_t)insns.size(), p.maps.data(), (uint32_t)p.maps.size(), opts,
                                   sv, &in) == GX_OK) {
                gx::JitProgram jp = jit_program(insns, p, sv, true);
                std::string log;
                int rc = 0;
                const std::string src = gx::jit_source({&jp}, log, rc, nullptr);
                if (rc == GX_OK) check_source(src);
                warp++;
            }
        }
    }
    if (fails) return 1;
    printf("OK lane=%u warp=%u multi=%u sched=%u\n", lane, warp, multi, sched);
    return 0;
}
