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

/* ExecParams.mode 2: ExecParams.cursor points at this header (the persistent header block) */
typedef struct gx_steal_hdr {
    uint32_t unused;        /* the claim cursor of mode 1 */
    uint32_t nchunks;       /* chunks in the table (where mode 1 keeps its count) */
    uint32_t shares;        /* one share per block of the launch */
    uint32_t hook_ctx_size; /* GX_SCHED_CTX */
    uint64_t budget_ns;     /* the context's budget field */
    const uint8_t *hook;    /* the scheduling program's device image */
    uint32_t *next;         /* per share: claims so far; zeroed before each launch */
    uint32_t *tally;        /* per block: GX_STEAL_WORDS counters; zeroed before each launch */
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

/*
 * One block's walk over the shares.  claim(s): the share's next offset (one atomic add);
 * left(s, size): chunks of share s not yet handed out (an advisory read, possibly stale);
 * ask(s, left, done): the hook's answer; run(c): run chunk c.  t[GX_STEAL_*] counts what
 * the block did.
 */
template <class Claim, class Left, class Ask, class Run>
GX_STEAL_FN void steal_walk(uint32_t self, uint32_t shares, uint32_t n, Claim claim, Left left, Ask ask, Run run,
                            uint32_t *t) {
    uint32_t lo = share_lo(self, shares, n), size = share_lo(self + 1, shares, n) - lo;
    for (;;) {
        const uint32_t k = claim(self);
        if (k >= size) break;
        run(lo + k);
        t[GX_STEAL_OWNED]++;
    }
    for (uint32_t i = 1; i < shares; i++) {
        const uint32_t v = self + i < shares ? self + i : self + i - shares;
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
 * The persistent skeleton of mode 2: exec_tiles' chunk handling (restaging on a program
 * change, the combining area kept open across a program's consecutive chunks) driven by
 * steal_walk.  Every callback's result is taken by thread 0 (the hook's by warp 0, with
 * lane 0 the only valid lane) and handed to the block through shared memory between two
 * barriers, so every thread takes the same path.  `hook(env, ctxw, valid, idx)` runs the
 * scheduling program's per-event code on a transposed one-record tile.
 */
template <typename RunChunk, typename Init, typename Flush, typename Hook>
__device__ __forceinline__ void exec_steal(const ExecParams &P, RunChunk run_chunk, Init wc_init, Flush wc_flush,
                                           Hook hook) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ u32 s_word;
    __shared__ const uint8_t *s_image;
    __shared__ u64 s_hctx[GX_SCHED_CTX / 8 * GX_CTX_ROW(GX_SCHED_CTX / 8)];
    const gx_steal_hdr *H = (const gx_steal_hdr *)P.cursor;
    const u32 n = H->nchunks, shares = H->shares, self = blockIdx.x;
    const u32 row = GX_CTX_ROW(GX_SCHED_CTX / 8);
    u64 *ctx_all = (u64 *)(smem + P.image_area);
    if (threadIdx.x == 0) s_image = nullptr;
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
    steal_walk(self, shares, n, claim, left, ask, run, t);
    __syncthreads();
    if (is_open) wc_flush(open);
    if (threadIdx.x == 0)
        for (u32 k = 0; k < GX_STEAL_WORDS; k++) H->tally[self * GX_STEAL_WORDS + k] = t[k];
}

} // namespace gx
#endif /* __CUDACC__ */

#endif /* GX_STEAL_CUH */
