/*
 * Host-only checks of the work-stealing walk (gx_steal.cuh: steal_walk), the claim loop of
 * the persistent kernel steered by a `should_try_steal` program (Sec. 4.3.2; the FixedWork,
 * Greedy and LatencyBudget policies of Sec. 6).  Blocks are host threads (or, for the
 * exact pins, calls made one after another); a claim is an atomic add, as on the device.
 * What must hold whatever the policy answers and however the blocks interleave:
 *   - every chunk runs exactly once;
 *   - a policy that never steals leaves each block exactly its own share;
 *   - the counters agree: asked >= granted >= stolen, owned + stolen summed = chunks;
 *   - every walk ends, within its own share + one failed claim per share of claims.
 * The same for the walk of one block per chunk (cancel_walk) over a model of the launcher:
 * a cancelled block never starts, and no block cancels again after a failed cancel.
 * Prints OK or the failed checks.
 */
#include "gx_steal.cuh" /* compiled with the engine's csrc/ (or a mutant copy) on the include path */

#include <atomic>
#include <cstdio>
#include <deque>
#include <memory>
#include <mutex>
#include <random>
#include <thread>
#include <vector>

static int fails = 0;
#define CHECK(c)                                                          \
    do {                                                                  \
        if (!(c)) {                                                       \
            std::printf("FAIL line %d: %s\n", __LINE__, #c);              \
            fails++;                                                      \
        }                                                                 \
    } while (0)

enum Policy { NEVER, ALWAYS, RANDOM, FIRST_K };

struct Run {
    uint32_t n, shares;
    std::unique_ptr<std::atomic<uint32_t>[]> next, runs;
    std::vector<uint32_t> t; /* shares x GX_STEAL_WORDS */
    std::vector<uint32_t> claims;
    Run(uint32_t n_, uint32_t s_)
        : n(n_), shares(s_), next(new std::atomic<uint32_t>[s_]), runs(new std::atomic<uint32_t>[n_ ? n_ : 1]),
          t(s_ * GX_STEAL_WORDS, 0), claims(s_, 0) {
        for (uint32_t i = 0; i < s_; i++) next[i] = 0;
        for (uint32_t i = 0; i < (n_ ? n_ : 1); i++) runs[i] = 0;
    }
    uint32_t size(uint32_t s) const { return gx::share_lo(s + 1, shares, n) - gx::share_lo(s, shares, n); }

    void walk(uint32_t self, Policy pol, uint64_t seed, bool yield) {
        std::mt19937_64 rng(seed);
        uint32_t *tt = &t[self * GX_STEAL_WORDS];
        auto claim = [&](uint32_t s) {
            claims[self]++;
            if (yield && (rng() & 3) == 0) std::this_thread::yield();
            return next[s].fetch_add(1);
        };
        auto left = [&](uint32_t s, uint32_t size) {
            const uint32_t k = next[s].load();
            return k < size ? size - k : 0u;
        };
        auto ask = [&](uint32_t, uint32_t l, uint32_t done) {
            CHECK(l > 0);
            CHECK(done == tt[GX_STEAL_OWNED] + tt[GX_STEAL_STOLEN]);
            switch (pol) {
            case NEVER: return false;
            case ALWAYS: return true;
            case RANDOM: return (rng() & 1) != 0;
            case FIRST_K: return tt[GX_STEAL_ASKED] <= 3; /* a budget: the first three asks */
            }
            return false;
        };
        auto run = [&](uint32_t c) {
            CHECK(c < n);
            if (c < n) runs[c].fetch_add(1);
        };
        uint32_t last = 0;
        auto find = [&](uint32_t after) {
            CHECK(after == last); /* one forward pass over the other shares */
            for (uint32_t o = after + 1; o < shares; o++)
                if (next[gx::share_after(self, o, shares)].load() < size(gx::share_after(self, o, shares)))
                    return last = o;
            return last = shares;
        };
        gx::steal_walk(self, shares, n, claim, left, find, ask, run, tt);
    }

    void check_common(Policy pol) {
        uint64_t done = 0;
        for (uint32_t c = 0; c < n; c++) CHECK(runs[c].load() == 1);
        for (uint32_t b = 0; b < shares; b++) {
            const uint32_t *tt = &t[b * GX_STEAL_WORDS];
            done += tt[GX_STEAL_OWNED] + tt[GX_STEAL_STOLEN];
            CHECK(tt[GX_STEAL_OWNED] <= size(b));
            CHECK(tt[GX_STEAL_ASKED] >= tt[GX_STEAL_GRANTED] && tt[GX_STEAL_GRANTED] >= tt[GX_STEAL_STOLEN]);
            /* a grant that finds the share empty ends that share's visit: at most one per other share */
            CHECK(tt[GX_STEAL_GRANTED] - tt[GX_STEAL_STOLEN] <= shares - 1);
            /* claims: own share plus one failed claim, then one per grant */
            CHECK(claims[b] == tt[GX_STEAL_OWNED] + 1 + tt[GX_STEAL_GRANTED]);
            if (pol == NEVER) {
                CHECK(tt[GX_STEAL_OWNED] == size(b));
                CHECK(tt[GX_STEAL_STOLEN] == 0 && tt[GX_STEAL_GRANTED] == 0);
                CHECK(tt[GX_STEAL_ASKED] <= 1);
            }
        }
        CHECK(done == n);
    }
};

/*
 * Mode 3: one block per chunk.  The launcher model keeps the blocks not yet started in a
 * queue; idle workers (the SMs) launch the next one, and a cancel takes one out of the
 * queue (the last, as a scheduler that launches in order would have started the others
 * first), so a cancelled block never runs.
 */
struct Launch {
    uint32_t n, grid;
    std::mutex mu;
    std::deque<uint32_t> pending;
    std::vector<uint8_t> cancelled;
    std::atomic<uint32_t> started{0};
    std::unique_ptr<std::atomic<uint32_t>[]> runs;
    std::vector<uint32_t> t;
    explicit Launch(uint32_t n_)
        : n(n_), grid(n_ ? n_ : 1), cancelled(grid, 0), runs(new std::atomic<uint32_t>[grid]), t(grid * GX_STEAL_WORDS, 0) {
        for (uint32_t b = 0; b < grid; b++) {
            pending.push_back(b);
            runs[b] = 0;
        }
    }
    uint32_t launch_next() {
        std::lock_guard<std::mutex> g(mu);
        if (pending.empty()) return ~0u;
        const uint32_t b = pending.front();
        pending.pop_front();
        return b;
    }
    uint32_t cancel_one() {
        std::lock_guard<std::mutex> g(mu);
        if (pending.empty()) return ~0u;
        const uint32_t b = pending.back();
        pending.pop_back();
        cancelled[b] = 1;
        return b;
    }
    void walk(uint32_t self, Policy pol, uint64_t seed, bool yield) {
        std::mt19937_64 rng(seed);
        uint32_t *tt = &t[self * GX_STEAL_WORDS];
        bool failed = false;
        auto left = [&]() {
            const uint32_t k = started.load();
            return k < n ? n - k : 0u;
        };
        auto ask = [&](uint32_t l, uint32_t done) {
            CHECK(l > 0);
            CHECK(done == tt[GX_STEAL_OWNED] + tt[GX_STEAL_STOLEN]);
            if (tt[GX_STEAL_ASKED] > n + 64) { /* a walk that keeps asking */
                CHECK(!"the walk does not end");
                return false;
            }
            switch (pol) {
            case NEVER: return false;
            case ALWAYS: return true;
            case RANDOM: return (rng() & 1) != 0;
            case FIRST_K: return tt[GX_STEAL_ASKED] <= 3;
            }
            return false;
        };
        auto cancel = [&]() {
            CHECK(!failed); /* a cancel after a failed one */
            if (yield && (rng() & 3) == 0) std::this_thread::yield();
            const uint32_t c = cancel_one();
            failed = c >= n;
            return c;
        };
        auto run = [&](uint32_t c) {
            CHECK(c < n);
            if (c >= n) return;
            CHECK(c == self || cancelled[c]);
            started.fetch_add(1);
            runs[c].fetch_add(1);
        };
        CHECK(!cancelled[self]); /* a cancelled block never starts */
        gx::cancel_walk(self, n, left, ask, cancel, run, tt);
    }
    void check_common(Policy pol) {
        uint64_t done = 0;
        for (uint32_t c = 0; c < n; c++) CHECK(runs[c].load() == 1);
        for (uint32_t b = 0; b < grid; b++) {
            const uint32_t *tt = &t[b * GX_STEAL_WORDS];
            done += tt[GX_STEAL_OWNED] + tt[GX_STEAL_STOLEN];
            CHECK(tt[GX_STEAL_OWNED] == (cancelled[b] || b >= n ? 0u : 1u));
            if (cancelled[b]) CHECK(tt[GX_STEAL_ASKED] == 0);
            CHECK(tt[GX_STEAL_ASKED] >= tt[GX_STEAL_GRANTED] && tt[GX_STEAL_GRANTED] >= tt[GX_STEAL_STOLEN]);
            CHECK(tt[GX_STEAL_GRANTED] - tt[GX_STEAL_STOLEN] <= 1); /* one failed cancel ends the walk */
            if (pol == NEVER) CHECK(tt[GX_STEAL_STOLEN] == 0 && tt[GX_STEAL_ASKED] <= 1);
        }
        CHECK(done == n);
    }
};

static void launched(uint32_t n, uint32_t workers, Policy pol, uint64_t seed) {
    Launch L(n);
    std::vector<std::thread> th;
    for (uint32_t w = 0; w < workers; w++)
        th.emplace_back([&L, w, pol, seed] {
            for (uint32_t b; (b = L.launch_next()) != ~0u;) L.walk(b, pol, seed * 7919u + w * 131u + b, true);
        });
    for (auto &x : th) x.join();
    L.check_common(pol);
}

/* blocks as threads, interleaved by the OS (and random yields) */
static void threaded(uint32_t n, uint32_t shares, Policy pol, uint64_t seed) {
    Run r(n, shares);
    std::vector<std::thread> th;
    for (uint32_t b = 0; b < shares; b++)
        th.emplace_back([&r, b, pol, seed] { r.walk(b, pol, seed * 1000003u + b, true); });
    for (auto &x : th) x.join();
    r.check_common(pol);
}

int main() {
    /* share cut: contiguous, covering [0, n), sizes differing by at most one */
    for (uint32_t n : {0u, 1u, 5u, 152u, 1000u, 4097u})
        for (uint32_t s : {1u, 2u, 7u, 152u, 760u}) {
            uint32_t lo = 0, mn = ~0u, mx = 0;
            for (uint32_t b = 0; b < s; b++) {
                CHECK(gx::share_lo(b, s, n) == lo);
                const uint32_t z = gx::share_lo(b + 1, s, n) - lo;
                mn = z < mn ? z : mn;
                mx = z > mx ? z : mx;
                lo += z;
            }
            CHECK(lo == n && mx - mn <= 1);
        }
    CHECK(gx::share_lo(760, 760, 0xFFFFFFFFu) == 0xFFFFFFFFu); /* no overflow at the largest table */

    /* exact pins, blocks one after another: block 0 first takes every chunk when it always steals */
    {
        Run r(1000, 8);
        r.walk(0, ALWAYS, 1, false);
        for (uint32_t b = 1; b < 8; b++) r.walk(b, ALWAYS, 1, false);
        r.check_common(ALWAYS);
        CHECK(r.t[GX_STEAL_OWNED] == 125 && r.t[GX_STEAL_STOLEN] == 875);
        CHECK(r.t[GX_STEAL_ASKED] == 875 && r.t[GX_STEAL_GRANTED] == 875); /* `left` is exact here: no failed grant */
        for (uint32_t b = 1; b < 8; b++) {
            CHECK(r.t[b * GX_STEAL_WORDS + GX_STEAL_OWNED] == 0);
            CHECK(r.t[b * GX_STEAL_WORDS + GX_STEAL_ASKED] == 0);
        }
    }
    {
        /* never stealing: each block exactly its share, in any order */
        Run r(1001, 7);
        for (uint32_t b = 7; b-- > 0;) r.walk(b, NEVER, 2, false);
        r.check_common(NEVER);
        /* the last block walked (block 0) found every other share drained: it never asked */
        CHECK(r.t[GX_STEAL_ASKED] == 0);
        CHECK(r.t[6 * GX_STEAL_WORDS + GX_STEAL_ASKED] == 1); /* the first one asked once and stopped */
    }
    {
        /* a budget of three grants: block 0 steals three chunks from share 1, then stops */
        Run r(80, 4);
        r.walk(0, FIRST_K, 3, false);
        CHECK(r.t[GX_STEAL_OWNED] == 20 && r.t[GX_STEAL_STOLEN] == 3 && r.t[GX_STEAL_ASKED] == 4);
        CHECK(r.next[1].load() == 3 && r.next[2].load() == 0);
        for (uint32_t b = 1; b < 4; b++) r.walk(b, NEVER, 3, false);
        r.check_common(FIRST_K);
        CHECK(r.t[1 * GX_STEAL_WORDS + GX_STEAL_OWNED] == 17);
    }
    {
        /* empty table, more shares than chunks */
        Run r0(0, 5);
        for (uint32_t b = 0; b < 5; b++) r0.walk(b, ALWAYS, 4, false);
        r0.check_common(ALWAYS);
        Run r1(3, 8);
        for (uint32_t b = 0; b < 8; b++) r1.walk(b, ALWAYS, 5, false);
        r1.check_common(ALWAYS);
    }

    /* mode 3, one worker: block 0 runs its chunk, then cancels every other block and runs its chunk */
    {
        Launch L(10);
        for (uint32_t b; (b = L.launch_next()) != ~0u;) L.walk(b, ALWAYS, 6, false);
        L.check_common(ALWAYS);
        CHECK(L.t[GX_STEAL_OWNED] == 1 && L.t[GX_STEAL_STOLEN] == 9 && L.t[GX_STEAL_ASKED] == 9);
    }
    {
        /* a block launched but not yet started keeps `left` above zero; the cancel that finds
           no block waiting ends the walk (a second cancel would be an error) */
        Launch L(6);
        const uint32_t first = L.launch_next(), second = L.launch_next(); /* blocks 0 and 1 launched */
        CHECK(first == 0 && second == 1);
        L.walk(0, ALWAYS, 7, false); /* cancels 5, 4, 3, 2; then block 1 has not started */
        CHECK(L.t[GX_STEAL_STOLEN] == 4 && L.t[GX_STEAL_GRANTED] == 5 && L.t[GX_STEAL_ASKED] == 5);
        L.walk(1, ALWAYS, 8, false);
        L.check_common(ALWAYS);
    }
    {
        Launch L(0); /* an empty table still launches one block, which does nothing */
        L.walk(L.launch_next(), ALWAYS, 9, false);
        L.check_common(ALWAYS);
        CHECK(L.t[GX_STEAL_ASKED] == 0);
    }
    for (Policy pol : {NEVER, ALWAYS, RANDOM, FIRST_K})
        for (uint32_t n : {0u, 1u, 7u, 300u, 3000u})
            for (uint32_t w : {1u, 4u, 16u}) launched(n, w, pol, n * 31u + w);

    /* interleaved: every policy, sizes around the share count */
    uint64_t seed = 11;
    for (Policy pol : {NEVER, ALWAYS, RANDOM, FIRST_K})
        for (uint32_t n : {0u, 1u, 63u, 64u, 1000u, 5000u})
            for (uint32_t s : {1u, 3u, 64u, 152u}) threaded(n, s, pol, seed++);

    if (fails) return 1;
    std::printf("OK\n");
    return 0;
}
