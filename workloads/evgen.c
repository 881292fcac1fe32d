/*
 * Seeded synthetic event generator shared by the oracle tests and the engine tests.
 *
 * It writes 32-byte little-endian event records
 *     { u64 addr; u32 sm_id; u32 warp_id; u64 ts_ns; u32 kind; u32 size; }
 * standing in for the device hook contexts of the paper (memory-access and
 * page-fault contexts, Sec. 4.3.1 / Sec. 5.2; block enter/exit contexts,
 * Sec. 4.3.2).  It holds none of the engine's arithmetic: only random draws.
 *
 * Every draw is a pure function of (seed, event index, stream) so the output does
 * not depend on the thread count:
 *   - SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 *     generators", OOPSLA 2014), used as a counter-based generator;
 *   - Zipf ranks by rejection-inversion (Hoermann, Derflinger, "Rejection-inversion
 *     to generate variates from monotone discrete distributions", 1996);
 *   - standard normals by the Box-Muller transform.
 * Timestamps are prefix sums of per-event gaps, computed in two passes over
 * fixed chunks so they are identical for any thread count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint64_t addr;
    uint32_t sm_id;
    uint32_t warp_id;
    uint64_t ts_ns;
    uint32_t kind;
    uint32_t size;
} ev_rec;

_Static_assert(sizeof(ev_rec) == 32, "record layout");

#define GOLDEN 0x9E3779B97F4A7C15ULL
#define CHUNK 65536ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* draw k (0..63) of item i: the (i*64+k+1)-th output of a SplitMix64 stream */
static inline uint64_t draw(uint64_t seed, uint64_t i, uint32_t k) {
    return mix64(seed + (i * 64ULL + k + 1ULL) * GOLDEN);
}

static inline double unit(uint64_t x) { /* [0,1) with 53 bits */
    return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

static inline uint32_t below(uint64_t x, uint32_t n) { /* Lemire multiply-shift */
    return (uint32_t)(((x >> 32) * (uint64_t)n) >> 32);
}

/* exponential gap with mean `mean_ns`, at least 1 ns */
static inline uint64_t exp_gap(uint64_t x, double mean_ns) {
    double u = unit(x);
    return 1ULL + (uint64_t)floor(-mean_ns * log(1.0 - u));
}

/* ---------------- Zipf by rejection-inversion ---------------- */
typedef struct {
    double s, n;
    double h_x1, h_n, slack;
} zipf_t;

/* (e^x - 1)/x and log(1+x)/x, stable near 0 */
static double expm1_over(double x) { return fabs(x) > 1e-8 ? expm1(x) / x : 1.0 + x * 0.5 * (1.0 + x / 3.0); }
static double log1p_over(double x) { return fabs(x) > 1e-8 ? log1p(x) / x : 1.0 - x * (0.5 - x / 3.0); }

/* h(x) = x^-s ; H(x) = integral of h = (x^(1-s) - 1)/(1-s) ; Hinv its inverse */
static double zh(const zipf_t *z, double x) { return exp(-z->s * log(x)); }
static double zH(const zipf_t *z, double x) {
    double lx = log(x);
    return expm1_over((1.0 - z->s) * lx) * lx;
}
static double zHinv(const zipf_t *z, double y) {
    double t = y * (1.0 - z->s);
    if (t < -1.0) t = -1.0;
    return exp(log1p_over(t) * y);
}

static void zipf_init(zipf_t *z, double s, double n) {
    z->s = s;
    z->n = n;
    z->h_x1 = zH(z, 1.5) - 1.0;
    z->h_n = zH(z, n + 0.5);
    z->slack = 2.0 - zHinv(z, zH(z, 2.5) - zh(z, 2.0));
}

/* rank in [1, n]; draws 8..63 of item i feed the rejection loop */
static uint64_t zipf_rank(const zipf_t *z, uint64_t seed, uint64_t i) {
    for (uint32_t k = 8; k < 64; k++) {
        double u = z->h_n + unit(draw(seed, i, k)) * (z->h_x1 - z->h_n);
        double x = zHinv(z, u);
        double kk = floor(x + 0.5);
        if (kk < 1.0) kk = 1.0;
        if (kk > z->n) kk = z->n;
        if (kk - x <= z->slack || u >= zH(z, kk + 0.5) - zh(z, kk)) return (uint64_t)kk;
    }
    return 1; /* 56 rejections in a row: probability far below 1e-30 */
}

/* ---------------- generation jobs ---------------- */
enum { KIND_UNIFORM = 0, KIND_PAGEHEAT = 1, KIND_PAIRS = 2, KIND_WARPS = 3 };

typedef struct {
    int kind;
    uint64_t seed, n; /* n = records (uniform/pageheat) or pairs */
    ev_rec *out;
    double p0, p1; /* pageheat: zipf s ; pairs: mu, sigma ; warps: zipf s, coalesced fraction */
    uint32_t u0;   /* pageheat, warps: log2 pages ; pairs: kernel ids */
    uint32_t u1;   /* warps: lanes per warp */
    zipf_t zipf;
    uint64_t *chunk_sum; /* per-chunk timestamp totals */
    int nthreads;
} job_t;

typedef struct {
    job_t *job;
    int t;
    int pass;
} targ_t;

static const uint32_t SIZE_CHOICES[4] = {4, 8, 16, 32};

static inline uint64_t n_items(const job_t *j) { return j->n; }

/* gap (ts increment) of item i */
static inline uint64_t item_gap(const job_t *j, uint64_t i) { return exp_gap(draw(j->seed, i, 0), 1000.0); }

static void fill_item(const job_t *j, uint64_t i, uint64_t ts) {
    uint64_t d1 = draw(j->seed, i, 1), d2 = draw(j->seed, i, 2), d3 = draw(j->seed, i, 3);
    uint64_t d4 = draw(j->seed, i, 4);
    if (j->kind == KIND_UNIFORM) {
        ev_rec *r = &j->out[i];
        r->addr = d1 & 0xFFFFFFFFULL;
        r->sm_id = below(d2, 148);
        r->warp_id = below(d2 << 32 | d2 >> 32, 64);
        r->ts_ns = ts;
        r->kind = below(d3, 8);
        r->size = SIZE_CHOICES[below(d4, 4)];
    } else if (j->kind == KIND_PAGEHEAT) {
        ev_rec *r = &j->out[i];
        uint64_t pages_mask = (1ULL << j->u0) - 1ULL;
        uint64_t rank = zipf_rank(&j->zipf, j->seed, i);
        /* rank -> page: an odd multiplier is a bijection modulo 2^k */
        uint64_t page = ((rank - 1ULL) * 0x9E3779B1ULL + (j->seed & pages_mask)) & pages_mask;
        uint32_t size = SIZE_CHOICES[below(d4, 4)];
        uint64_t offset = (d1 & 4095ULL) & ~(uint64_t)(size - 1);
        r->addr = (page << 12) | offset;
        r->sm_id = below(d2, 148);
        r->warp_id = below(d2 << 32 | d2 >> 32, 64);
        r->ts_ns = ts;
        r->kind = below(d3, 8);
        r->size = size;
    } else if (j->kind == KIND_WARPS) { /* one warp: shared instruction fields, per-lane addresses */
        uint64_t pages_mask = (1ULL << j->u0) - 1ULL;
        uint32_t size = SIZE_CHOICES[below(d4, 4)];
        int coalesced = unit(draw(j->seed, i, 5)) < j->p1;
        uint64_t lane_seed = mix64(j->seed ^ 0xC0A1E5CEDULL); /* lanes draw from their own stream */
        uint64_t base = 0;
        if (coalesced) {
            uint64_t rank = zipf_rank(&j->zipf, j->seed, i);
            uint64_t page = ((rank - 1ULL) * 0x9E3779B1ULL + (j->seed & pages_mask)) & pages_mask;
            base = (page << 12) | ((d1 & 4095ULL) & ~(uint64_t)(size - 1));
        }
        for (uint32_t l = 0; l < j->u1; l++) {
            ev_rec *r = &j->out[i * j->u1 + l];
            if (coalesced) {
                r->addr = base + (uint64_t)l * size;
            } else {
                uint64_t li = i * j->u1 + l;
                uint64_t rank = zipf_rank(&j->zipf, lane_seed, li);
                uint64_t page = ((rank - 1ULL) * 0x9E3779B1ULL + (j->seed & pages_mask)) & pages_mask;
                r->addr = (page << 12) | ((draw(lane_seed, li, 1) & 4095ULL) & ~(uint64_t)(size - 1));
            }
            r->sm_id = below(d2, 148);
            r->warp_id = below(d2 << 32 | d2 >> 32, 64);
            r->ts_ns = ts;
            r->kind = below(d3, 8);
            r->size = size;
        }
    } else { /* entry/exit pair of one thread block */
        ev_rec *e = &j->out[2 * i], *x = &j->out[2 * i + 1];
        uint32_t kid = below(d1, j->u0);
        double u1 = unit(d2), u2 = unit(d3);
        double zn = sqrt(-2.0 * log(1.0 - u1)) * cos(6.283185307179586 * u2);
        double lat = exp(j->p0 + j->p1 * zn);
        uint64_t lat_ns = (uint64_t)llround(lat);
        e->addr = (uint64_t)kid | ((d4 >> 32) << 32);
        e->sm_id = below(d4, 148);
        e->warp_id = below(d3, 64);
        e->ts_ns = ts;
        e->kind = 0;
        e->size = 256;
        *x = *e;
        x->ts_ns = ts + lat_ns;
        x->kind = 1;
    }
}

static void *worker(void *p) {
    targ_t *a = (targ_t *)p;
    job_t *j = a->job;
    uint64_t n = n_items(j);
    uint64_t nch = (n + CHUNK - 1) / CHUNK;
    for (uint64_t c = (uint64_t)a->t; c < nch; c += (uint64_t)j->nthreads) {
        uint64_t b = c * CHUNK, e = b + CHUNK < n ? b + CHUNK : n;
        if (a->pass == 0) {
            uint64_t s = 0;
            for (uint64_t i = b; i < e; i++) s += item_gap(j, i);
            j->chunk_sum[c] = s;
        } else {
            uint64_t ts = j->chunk_sum[c]; /* exclusive prefix, filled between passes */
            for (uint64_t i = b; i < e; i++) {
                ts += item_gap(j, i);
                fill_item(j, i, ts);
            }
        }
    }
    return NULL;
}

static int run_job(job_t *j) {
    uint64_t n = n_items(j);
    if (n == 0) return 0;
    uint64_t nch = (n + CHUNK - 1) / CHUNK;
    j->chunk_sum = (uint64_t *)calloc(nch, sizeof(uint64_t));
    if (!j->chunk_sum) return -12;
    if (j->nthreads < 1) j->nthreads = 1;
    if (j->nthreads > 256) j->nthreads = 256;
    pthread_t th[256];
    targ_t args[256];
    for (int pass = 0; pass < 2; pass++) {
        for (int t = 0; t < j->nthreads; t++) {
            args[t].job = j;
            args[t].t = t;
            args[t].pass = pass;
            pthread_create(&th[t], NULL, worker, &args[t]);
        }
        for (int t = 0; t < j->nthreads; t++) pthread_join(th[t], NULL);
        if (pass == 0) { /* exclusive prefix sum of chunk totals, start at 1 ms */
            uint64_t acc = 1000000ULL;
            for (uint64_t c = 0; c < nch; c++) {
                uint64_t s = j->chunk_sum[c];
                j->chunk_sum[c] = acc;
                acc += s;
            }
        }
    }
    free(j->chunk_sum);
    return 0;
}

/* C1/C4-style records: addr uniform over [0, 2^32), kind 0..7, size in {4,8,16,32} */
int evgen_uniform(uint64_t seed, uint64_t n, void *out, int nthreads) {
    job_t j;
    memset(&j, 0, sizeof j);
    j.kind = KIND_UNIFORM;
    j.seed = seed;
    j.n = n;
    j.out = (ev_rec *)out;
    j.nthreads = nthreads;
    return run_job(&j);
}

/* C2-style records: 4 KiB pages drawn Zipf(s) over 2^log2_pages pages */
int evgen_pageheat(uint64_t seed, uint64_t n, double s, uint32_t log2_pages, void *out, int nthreads) {
    if (log2_pages < 1 || log2_pages > 40 || !(s > 0.0) || s == 1.0) return -22;
    job_t j;
    memset(&j, 0, sizeof j);
    j.kind = KIND_PAGEHEAT;
    j.seed = seed;
    j.n = n;
    j.out = (ev_rec *)out;
    j.u0 = log2_pages;
    zipf_init(&j.zipf, s, (double)(1ULL << log2_pages));
    j.nthreads = nthreads;
    return run_job(&j);
}

/*
 * Warp-context memory-access records: n_warps * lanes records, warp w in records
 * [w*lanes, (w+1)*lanes).  The lanes of a warp share sm_id, warp_id, ts_ns, kind and size
 * (one instruction of one warp); a fraction `coalesced` of the warps touch consecutive
 * size-strided addresses from one Zipf(s) page, the others one Zipf(s) page per lane.
 */
int evgen_warp_access(uint64_t seed, uint64_t n_warps, uint32_t lanes, double s, uint32_t log2_pages,
                      double coalesced, void *out, int nthreads) {
    if (lanes < 1 || lanes > 32 || log2_pages < 1 || log2_pages > 40 || !(s > 0.0) || s == 1.0 ||
        !(coalesced >= 0.0 && coalesced <= 1.0))
        return -22;
    job_t j;
    memset(&j, 0, sizeof j);
    j.kind = KIND_WARPS;
    j.seed = seed;
    j.n = n_warps;
    j.out = (ev_rec *)out;
    j.u0 = log2_pages;
    j.u1 = lanes;
    j.p0 = s;
    j.p1 = coalesced;
    zipf_init(&j.zipf, s, (double)(1ULL << log2_pages));
    j.nthreads = nthreads;
    return run_job(&j);
}

/* C3-style (entry, exit) record pairs: 2*n_pairs records, latency lognormal(mu, sigma) */
int evgen_latency_pairs(uint64_t seed, uint64_t n_pairs, double mu, double sigma, uint32_t n_kernels,
                        void *out, int nthreads) {
    if (n_kernels == 0) return -22;
    job_t j;
    memset(&j, 0, sizeof j);
    j.kind = KIND_PAIRS;
    j.seed = seed;
    j.n = n_pairs;
    j.out = (ev_rec *)out;
    j.p0 = mu;
    j.p1 = sigma;
    j.u0 = n_kernels;
    j.nthreads = nthreads;
    return run_job(&j);
}

/* raw draws, for tests of the generator itself */
uint64_t evgen_draw(uint64_t seed, uint64_t i, uint32_t k) { return draw(seed, i, k); }
