/*
 * Host-only checks of the batch planner's chunk cutting (batch.cpp: make_chunks), the step
 * that turns a batch of (program, events) items into the chunk table the persistent kernel
 * claims from (Sec. 4.3.2, Sec. 5.3: persistent workers claiming logical work units).
 * Compiled by tests/test_host_planner.py against the engine's sources; prints OK or the
 * failed checks.  No device is touched: the programs are host-side stand-ins.
 */
#include "../../paper_2512_12615_gb300/csrc/batch.cpp"

#include <cstdio>

static int fails = 0;
#define CHECK(c)                                                          \
    do {                                                                  \
        if (!(c)) {                                                       \
            std::printf("FAIL line %d: %s\n", __LINE__, #c);              \
            fails++;                                                      \
        }                                                                 \
    } while (0)

static gx_prog *fake_prog(uintptr_t image, uint32_t image_bytes, uint32_t ctx_size) {
    gx_prog *p = new gx_prog();
    p->dmem = (void *)image;
    p->image_bytes = image_bytes;
    p->opts.ctx_size = ctx_size;
    return p;
}

/* every item's events [0, n) covered once, in order, by chunks of at most `ce` events */
static void check_cover(const std::vector<Item> &items, const std::vector<gx_chunk> &ch, uint64_t ce) {
    for (const Item &it : items) {
        uint64_t next = 0;
        for (const gx_chunk &c : ch) {
            if (c.events != (const uint8_t *)it.events) continue;
            CHECK(c.begin == next);
            CHECK(c.end > c.begin && c.end - c.begin <= ce && c.end <= it.n);
            CHECK(c.begin % ce == 0);
            CHECK(c.image == (const uint8_t *)it.prog->dmem && c.image_bytes == it.prog->image_bytes);
            CHECK(c.ctx_size == it.prog->opts.ctx_size && c.ret_out == (long long *)it.ret_out && c.idx_base == 0);
            next = c.end;
        }
        CHECK(next == it.n);
    }
}

int main() {
    gx_prog *a = fake_prog(0x10000, 512, 32), *b = fake_prog(0x20000, 768, 64);
    static uint8_t ev[8][16];
    static int64_t ret[8][4];
    /* sizes around the chunk: empty, 1, one short, exact, one over, many and ragged */
    const uint64_t ns[] = {0, 1, 1023, 1024, 1025, 7 * 1024 + 9, 33, 2048};
    std::vector<Item> items;
    for (int i = 0; i < 8; i++) items.push_back(Item{i % 2 ? b : a, ev[i], ns[i], ret[i]});
    std::vector<gx_chunk> ch;

    make_chunks(items, 1024, ch);
    check_cover(items, ch, 1024);
    uint64_t total = 0;
    for (uint64_t n : ns) total += (n + 1023) / 1024;
    CHECK(ch.size() == total);
    /* largest item first, ties in item order (stable) */
    for (size_t k = 1; k < ch.size(); k++) {
        const Item *p = nullptr, *q = nullptr;
        for (const Item &it : items) {
            if (ch[k - 1].events == (const uint8_t *)it.events) p = &it;
            if (ch[k].events == (const uint8_t *)it.events) q = &it;
        }
        CHECK(p && q && (p == q || p->n >= q->n));
        if (p && q && p != q && p->n == q->n) CHECK(p < q);
    }
    for (const gx_chunk &c : ch) CHECK(c.pad == 0); /* no slots, no per-program choice */

    /* a multi-program kernel: each chunk carries its program's slot */
    std::map<gx_prog *, uint32_t> slots{{a, 0}, {b, 1}};
    make_chunks(items, 256, ch, &slots);
    check_cover(items, ch, 256);
    for (const gx_chunk &c : ch) CHECK(c.pad == (c.image == (const uint8_t *)a->dmem ? 0u : 1u));

    /* a tuned sharding choice travels on its program's chunks, never wider than the area */
    a->pref_tuned = true;
    a->pref_shards = 9 | GX_SHARDS_AGG; /* wider than an 8-entry-bit area */
    b->pref_tuned = true;
    b->pref_shards = GX_SHARDS_OFF;
    make_chunks(items, 1024, ch, &slots, /*pref_bits=*/8, /*alloc_bits=*/8);
    for (const gx_chunk &c : ch) {
        const bool is_a = c.image == (const uint8_t *)a->dmem;
        CHECK((c.pad >> 63) == 1);
        const uint32_t wc = (uint32_t)((c.pad >> 32) & 0x7FFFFFFFu);
        CHECK(is_a ? wc == (8u | 0x100u) : wc == 0u); /* 9 clamped to 8, the miss policy kept; OFF = 0 */
        CHECK((c.pad & 0xFFFFFFFFu) == (is_a ? 0u : 1u));
    }
    /* the default choice (0) takes the kernel's width */
    a->pref_shards = GX_SHARDS_AGG;
    make_chunks(items, 1024, ch, &slots, 6, 8);
    for (const gx_chunk &c : ch)
        if (c.image == (const uint8_t *)a->dmem) CHECK(((c.pad >> 32) & 0x7FFFFFFFu) == (6u | 0x100u));
    /* untuned programs, or no per-program choice asked for, carry nothing */
    a->pref_tuned = b->pref_tuned = false;
    make_chunks(items, 1024, ch, &slots, 8, 8);
    for (const gx_chunk &c : ch) CHECK((c.pad >> 63) == 0);
    a->pref_tuned = true;
    make_chunks(items, 1024, ch, &slots, 0, 8);
    for (const gx_chunk &c : ch) CHECK((c.pad >> 63) == 0);

    /* the cache width a launch's shards value runs with, and the area a kernel allocates */
    CHECK(bits_of(GX_SHARDS_OFF, 8) == 0 && bits_of(0, 8) == 8 && bits_of(5 | GX_SHARDS_AGG, 8) == 5);

    delete a;
    delete b;
    if (fails) return 1;
    std::printf("OK\n");
    return 0;
}
