/*
 * Work stealing between the blocks of the persistent kernel, steered by a scheduling
 * program: the `should_try_steal` hook over a block context (Sec. 4.3.2), with the
 * FixedWork / Greedy / LatencyBudget policies of Sec. 6.
 *
 * The chunk table is cut into one contiguous share per block.  A block first drains its
 * own share, then visits the other shares in turn.  Before each chunk it would take from
 * another share it runs the hook on a 32-byte context
 *     {u32 block @0, u32 SM @4, u32 chunks done @8, u32 chunks left in that share @12,
 *      u64 ns since the block started @16, u64 budget ns @24};
 * R0 != 0 takes the chunk, R0 == 0 ends the block's work.
 *
 * Every claim, the owner's and a thief's alike, is one atomic add on the share's counter,
 * so each chunk is handed out once.  Every owner drains its own share whatever the hook
 * answers, so every chunk runs: the policy decides only which block runs it.  Nothing
 * waits on another block.  A block's work is bounded by the chunks it runs, plus one
 * failed claim and one counter read per share.
 *
 * The walk (steal_walk) is plain C++ over four callbacks, so the host can check it; the
 * device skeleton (exec_steal) gives the callbacks block-wide meaning.  Only programs
 * compiled for a batch with a scheduling program include this header.
 */
#ifndef GX_STEAL_CUH
#define GX_STEAL_CUH

#include "gx.h"
#include "gx_layout.h"

#ifdef __CUDACC__
#define GX_STEAL_FN __device__ __forceinline__
#else
#define GX_STEAL_FN inline
#endif

/* ExecParams.mode 2 and 3: ExecParams.cursor points at this header (the persistent header block) */
typedef struct gx_steal_hdr {
    uint32_t unused;        /* the claim cursor of mode 1 */
    uint32_t nchunks;       /* chunks in the table (where mode 1 keeps its count) */
    uint32_t shares;        /* one share per block of the launch */
    uint32_t hook_ctx_size; /* GX_SCHED_CTX */
    uint64_t budget_ns;     /* the context's budget field */
    const uint8_t *hook;    /* the scheduling program's device image */
    uint32_t *next;         /* mode 2: per share, claims so far; mode 3: next[0] = chunks started;
                               zeroed before each launch */
    uint32_t *tally;        /* per block of the launch: GX_STEAL_WORDS counters; zeroed before each launch */
    uint64_t pad[26];
} gx_steal_hdr;

#ifdef __cplusplus
static_assert(sizeof(gx_steal_hdr) == 256, "the persistent header block is 256 bytes");
/* exec_steal packs the context as four words: block | SM << 32, done | left << 32, elapsed, budget */
static_assert(GX_SCHED_CTX == 32 && GX_SCHED_OFF_BLOCK == 0 && GX_SCHED_OFF_SM == 4 && GX_SCHED_OFF_DONE == 8 &&
                  GX_SCHED_OFF_LEFT == 12 && GX_SCHED_OFF_ELAPSED == 16 && GX_SCHED_OFF_BUDGET == 24,
              "scheduling context layout");
#endif

namespace gx {

/* first chunk of share s when n chunks are cut into `shares` contiguous shares */
GX_STEAL_FN uint32_t share_lo(uint32_t s, uint32_t shares, uint32_t n) {
    return (uint32_t)((uint64_t)s * n / shares);
}

/* the share `o` places after share `self` (cyclically) */
GX_STEAL_FN uint32_t share_after(uint32_t self, uint32_t o, uint32_t shares) {
    return self + o < shares ? self + o : self + o - shares;
}

/*
 * One block's walk over the shares.  claim(s): the share's next offset (one atomic add);
 * left(s, size): chunks of share s not yet handed out (an advisory read, possibly stale);
 * find(after): the smallest o in (after, shares) whose share share_after(self, o) showed
 * chunks left, else `shares` (advisory too); ask(s, left, done): the hook's answer;
 * run(c): run chunk c.  t[GX_STEAL_*] counts what the block did.  The other shares are
 * visited once each, in order after the block's own.
 */
template <class Claim, class Left, class Find, class Ask, class Run>
GX_STEAL_FN void steal_walk(uint32_t self, uint32_t shares, uint32_t n, Claim claim, Left left, Find find, Ask ask,
                            Run run, uint32_t *t) {
    uint32_t lo = share_lo(self, shares, n), size = share_lo(self + 1, shares, n) - lo;
    for (;;) {
        const uint32_t k = claim(self);
        if (k >= size) break;
        run(lo + k);
        t[GX_STEAL_OWNED]++;
    }
    for (uint32_t o = find(0u); o < shares; o = find(o)) {
        const uint32_t v = share_after(self, o, shares);
        lo = share_lo(v, shares, n);
        size = share_lo(v + 1, shares, n) - lo;
        for (;;) {
            const uint32_t l = left(v, size);
            if (l == 0) break;
            t[GX_STEAL_ASKED]++;
            if (!ask(v, l, t[GX_STEAL_OWNED] + t[GX_STEAL_STOLEN])) return;
            t[GX_STEAL_GRANTED]++;
            const uint32_t k = claim(v);
            if (k >= size) break;
            run(lo + k);
            t[GX_STEAL_STOLEN]++;
        }
    }
}

/*
 * One block's walk when every chunk has a block of its own (mode 3): run the block's own
 * chunk, then, while left() (chunks not yet started) is nonzero and ask(left, done) says
 * yes, cancel() a block that has not started and run its chunk.  cancel() returns that
 * block's index, or a value >= n when no block was cancelled; after that the walk never
 * cancels again.
 */
template <class Left, class Ask, class Cancel, class Run>
GX_STEAL_FN void cancel_walk(uint32_t self, uint32_t n, Left left, Ask ask, Cancel cancel, Run run, uint32_t *t) {
    if (self < n) {
        run(self);
        t[GX_STEAL_OWNED]++;
    }
    for (;;) {
        const uint32_t l = left();
        if (l == 0) break;
        t[GX_STEAL_ASKED]++;
        if (!ask(l, t[GX_STEAL_OWNED] + t[GX_STEAL_STOLEN])) break;
        t[GX_STEAL_GRANTED]++;
        const uint32_t c = cancel();
        if (c >= n) break;
        run(c);
        t[GX_STEAL_STOLEN]++;
    }
}

} // namespace gx

#ifdef __CUDACC__
#include "gx_device.cuh"

namespace gx {

__device__ __forceinline__ u64 steal_now_ns() {
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ u32 steal_smid() {
    u32 s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}

/*
 * Bounded wait on phase `parity` of a shared-memory mbarrier; false if it gave up.
 */
__device__ __forceinline__ bool steal_mbar_wait(u32 mbar, u32 parity) {
    for (u32 i = 0; i < WAIT_SPINS; i++) {
        u32 ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok)
                     : "r"(mbar), "r"(parity)
                     : "memory");
        if (ok) return true;
    }
    return false;
}

/*
 * Ask the hardware to cancel one block of this launch that has not started (cluster launch
 * control; every block is a cluster of one).  Thread 0 only.  Returns the cancelled block's
 * index, GX_STEAL_NONE if none was left, or GX_STEAL_STUCK if the response did not arrive
 * within the wait bound.  After a GX_STEAL_NONE the block must not ask again.
 */
#define GX_STEAL_NONE 0xFFFFFFFFu
#define GX_STEAL_STUCK 0xFFFFFFFEu
__device__ __forceinline__ u32 steal_cancel_one(u32 resp, u32 mbar, u32 parity) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], 16;\n}" ::"r"(mbar)
                 : "memory");
    asm volatile("clusterlaunchcontrol.try_cancel.async.shared::cta.mbarrier::complete_tx::bytes.b128 [%0], [%1];" ::"r"(
                     resp),
                 "r"(mbar)
                 : "memory");
    if (!steal_mbar_wait(mbar, parity)) return GX_STEAL_STUCK;
    u32 ok, x = GX_STEAL_NONE;
    asm volatile("{\n .reg .b128 r;\n .reg .pred p;\n ld.shared.b128 r, [%1];\n"
                 " clusterlaunchcontrol.query_cancel.is_canceled.pred.b128 p, r;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(resp)
                 : "memory");
    if (ok)
        asm volatile("{\n .reg .b128 r;\n ld.shared.b128 r, [%1];\n"
                     " clusterlaunchcontrol.query_cancel.get_first_ctaid::x.b32.b128 %0, r;\n}"
                     : "=r"(x)
                     : "r"(resp)
                     : "memory");
    return x;
}

/*
 * The skeleton of modes 2 and 3: exec_tiles' chunk handling (restaging on a program
 * change, the combining area kept open across a program's consecutive chunks) driven by
 * one of two walks.
 *   mode 2 (persistent, one share per block): steal_walk.
 *   mode 3 (one block per chunk, cluster launch control): block b runs chunk b; then,
 *     while chunks have not all started and the hook says yes, it cancels a block that
 *     has not launched and runs that block's chunk.  A cancelled block never runs, and
 *     each is handed to one canceller, so every chunk runs once.  The first failed
 *     cancel ends the block's stealing.
 * Every callback's result is taken by thread 0 (the hook's by warp 0, with lane 0 the
 * only valid lane) and handed to the block through shared memory between two barriers,
 * so every thread takes the same path.  `hook(env, ctxw, valid, idx)` runs the scheduling
 * program's per-event code on a transposed one-record tile.
 */
template <typename RunChunk, typename Init, typename Flush, typename Hook>
__device__ __forceinline__ void exec_steal(const ExecParams &P, RunChunk run_chunk, Init wc_init, Flush wc_flush,
                                           Hook hook) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ u32 s_word;
    __shared__ const uint8_t *s_image;
    __shared__ u64 s_hctx[GX_SCHED_CTX / 8 * GX_CTX_ROW(GX_SCHED_CTX / 8)];
    __shared__ __align__(16) uint4 s_resp;  /* mode 3: the cancel response */
    __shared__ __align__(8) u64 s_mbar;     /* mode 3: its completion barrier */
    const gx_steal_hdr *H = (const gx_steal_hdr *)P.cursor;
    const u32 n = H->nchunks, shares = H->shares, self = blockIdx.x;
    const u32 row = GX_CTX_ROW(GX_SCHED_CTX / 8);
    u64 *ctx_all = (u64 *)(smem + P.image_area);
    const u32 resp = (u32)__cvta_generic_to_shared(&s_resp), mbar = (u32)__cvta_generic_to_shared(&s_mbar);
    if (threadIdx.x == 0) {
        s_image = nullptr;
        if (P.mode == 3) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    for (u32 i = threadIdx.x; i < GX_SCHED_CTX / 8 * row; i += blockDim.x) s_hctx[i] = 0;
    const u64 t0 = steal_now_ns();
    ExecEnv open;
    u32 open_wcp = 0;
    bool is_open = false; /* block-uniform */
    u32 t[GX_STEAL_WORDS] = {0, 0, 0, 0};
    auto claim = [&](u32 s) -> u32 {
        __syncthreads();
        if (threadIdx.x == 0) s_word = atomicAdd(&H->next[s], 1u);
        __syncthreads();
        return s_word;
    };
    auto left = [&](u32 s, u32 size) -> u32 {
        __syncthreads();
        if (threadIdx.x == 0) {
            const u32 k = *(volatile const u32 *)&H->next[s];
            s_word = k < size ? size - k : 0u;
        }
        __syncthreads();
        return s_word;
    };
    /* block-parallel: each thread reads one share's counter per step, __syncthreads_or decides */
    auto find = [&](u32 after) -> u32 {
        __syncthreads();
        if (threadIdx.x == 0) s_word = shares;
        for (u32 o0 = after + 1; o0 < shares; o0 += blockDim.x) {
            const u32 o = o0 + threadIdx.x;
            bool has = false;
            if (o < shares) {
                const u32 v = share_after(self, o, shares);
                const u32 size = share_lo(v + 1, shares, n) - share_lo(v, shares, n);
                has = *(volatile const u32 *)&H->next[v] < size;
            }
            if (__syncthreads_or(has)) {
                if (has) atomicMin(&s_word, o);
                __syncthreads();
                return s_word;
            }
        }
        return shares;
    };
    auto ask = [&](u32 s, u32 l, u32 done) -> bool {
        __syncthreads();
        if (threadIdx.x < 32) {
            const u32 lane = threadIdx.x;
            if (lane == 0) {
                s_hctx[0 * row] = (u64)self | ((u64)steal_smid() << 32);
                s_hctx[1 * row] = (u64)done | ((u64)l << 32);
                s_hctx[2 * row] = steal_now_ns() - t0;
                s_hctx[3 * row] = H->budget_ns;
            }
            __syncwarp();
            const ExecEnv env = stage_env_at((uint8_t *)H->hook, 0, 0, 0);
            const u64 r0 = hook(env, s_hctx, lane == 0, (u64)self);
            if (lane == 0) s_word = r0 != 0 ? 1u : 0u;
        }
        __syncthreads();
        return s_word != 0;
    };
    auto run = [&](u32 c) {
        if (P.mode == 3 && threadIdx.x == 0) atomicAdd(&H->next[0], 1u);
        const gx_chunk ch = P.chunks[c];
        const u32 wcp = (ch.pad >> 63) ? (u32)(ch.pad >> 32) & 0x1FFu : P.wc_bits; /* the chunk's own choice */
        if (is_open && ((u32)ch.pad != open.slot || wcp != open_wcp)) {
            wc_flush(open);
            __syncthreads();
            is_open = false;
        }
        if (ch.image != s_image) {
            stage_image(smem, ch.image, ch.image_bytes);
            if (threadIdx.x == 0) s_image = ch.image;
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
    };
    if (P.mode != 3) {
        steal_walk(self, shares, n, claim, left, find, ask, run, t);
    } else {
        __syncthreads(); /* the barrier's initialisation */
        u32 phase = 0;
        auto cancel = [&]() -> u32 {
            __syncthreads();
            if (threadIdx.x == 0) {
                s_word = steal_cancel_one(resp, mbar, phase);
                if (s_word == GX_STEAL_STUCK) { /* the response never came: stop, and say so */
                    const ExecEnv he = stage_env_at((uint8_t *)H->hook, 0, 0, 0);
                    atomicAdd(&he.stats[GX_STAT_WAITS], 1ull);
                    set_status(he.stats, GX_E_TIMEOUT);
                    /* once more, bounded: the response is still owed to this block's shared memory */
                    steal_mbar_wait(mbar, phase);
                }
            }
            __syncthreads();
            phase ^= 1u;
            return s_word;
        };
        cancel_walk(
            self, n, [&]() -> u32 { return left(0, n); },
            [&](u32 l, u32 done) -> bool { return ask(0, l, done); }, cancel, run, t);
    }
    __syncthreads();
    if (is_open) wc_flush(open);
    if (threadIdx.x == 0)
        for (u32 k = 0; k < GX_STEAL_WORDS; k++) H->tally[self * GX_STEAL_WORDS + k] = t[k];
}

} // namespace gx
#endif /* __CUDACC__ */

#endif /* GX_STEAL_CUH */
