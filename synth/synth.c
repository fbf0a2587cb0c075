/*
 * Seeded synthetic temporal-graph generators.
 *
 * This module draws random inputs only; it contains none of the motif-mining
 * arithmetic.  Both the CPU oracle and the CUDA library consume the arrays it
 * writes.  Every value is a pure function of (seed, stream, index) through a
 * counter-based generator, so the output is identical for any thread count and
 * on any host (x86_64 or aarch64).
 *
 * Counter-based generator: SplitMix64 finaliser (Steele, Lea, Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014), applied to
 * seed, stream id and element index in turn.
 *
 * Workload shapes follow the paper's evaluation graphs (Section 6, Table 1:
 * power-law social / transaction graphs with second-resolution timestamps).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* one 64-bit draw for (seed, stream, index) */
static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t i) {
    return mix64(mix64(seed ^ mix64(stream)) + i);
}

/* uniform double in [0,1) with 53 bits */
static inline double unif(uint64_t seed, uint64_t stream, uint64_t i) {
    return (double)(draw(seed, stream, i) >> 11) * (1.0 / 9007199254740992.0);
}

/* uniform integer in [0, n) (multiply-shift; bias < n / 2^64) */
static inline uint64_t below(uint64_t seed, uint64_t stream, uint64_t i, uint64_t n) {
    return (uint64_t)(((__uint128_t)draw(seed, stream, i) * n) >> 64);
}

/* ---------------------------------------------------------------- threads */

typedef void (*range_fn)(void* ctx, int64_t lo, int64_t hi);
typedef struct { range_fn fn; void* ctx; int64_t lo, hi; } job_t;

static void* run_job(void* p) {
    job_t* j = (job_t*)p;
    j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}

static void parallel_for(int64_t n, int nthreads, range_fn fn, void* ctx) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (n < 65536 || nthreads == 1) { fn(ctx, 0, n); return; }
    pthread_t th[256];
    job_t jobs[256];
    for (int k = 0; k < nthreads; ++k) {
        jobs[k].fn = fn; jobs[k].ctx = ctx;
        jobs[k].lo = n * k / nthreads; jobs[k].hi = n * (k + 1) / nthreads;
        pthread_create(&th[k], NULL, run_job, &jobs[k]);
    }
    for (int k = 0; k < nthreads; ++k) pthread_join(th[k], NULL);
}

/* ------------------------------------------------------- uniform (tiny) */

typedef struct {
    uint64_t seed; int64_t n; int64_t tmax;
    int32_t *src, *dst; int64_t* t;
} uni_ctx;

static void uni_body(void* p, int64_t lo, int64_t hi) {
    uni_ctx* c = (uni_ctx*)p;
    for (int64_t e = lo; e < hi; ++e) {
        int64_t s = (int64_t)below(c->seed, 1, (uint64_t)e, (uint64_t)c->n);
        /* destination uniform over the other n-1 nodes: no self-loops */
        int64_t d = (int64_t)below(c->seed, 2, (uint64_t)e, (uint64_t)(c->n - 1));
        if (d >= s) d += 1;
        c->src[e] = (int32_t)s;
        c->dst[e] = (int32_t)d;
        c->t[e] = (int64_t)below(c->seed, 3, (uint64_t)e, (uint64_t)c->tmax);
    }
}

/* n >= 2 nodes, m edges, timestamps uniform in [0, tmax). */
int synth_uniform(uint64_t seed, int64_t n, int64_t m, int64_t tmax,
                  int32_t* src, int32_t* dst, int64_t* t, int nthreads) {
    if (n < 2 || m < 0 || tmax < 1) return 1;
    uni_ctx c = { seed, n, tmax, src, dst, t };
    parallel_for(m, nthreads, uni_body, &c);
    return 0;
}

/* ------------------------------------------------- power-law (bursty) */

/*
 * Node popularity follows a Chung-Lu weight w_i ~ (i+1)^-beta, beta = 1/(alpha-1),
 * which gives a degree distribution with tail exponent alpha.  A draw uses the
 * closed-form inverse CDF of the continuous weight density on [1, n+1), then a
 * fixed bijective hash maps rank -> node id so hubs are spread over the id space.
 */
typedef struct { double beta, a, b; int64_t n, r0; uint64_t perm_mul, perm_add; } zipf_t;

static uint64_t gcd_u64(uint64_t a, uint64_t b) { while (b) { uint64_t r = a % b; a = b; b = r; } return a; }

/* ranks r0..n-1 follow the weight density; r0 > 0 leaves ranks below r0 to the hubs */
static void zipf_init(zipf_t* z, int64_t n, double alpha, uint64_t seed, int64_t r0) {
    z->n = n;
    z->r0 = r0;
    z->beta = 1.0 / (alpha - 1.0);
    double om = 1.0 - z->beta;
    z->a = pow((double)r0 + 1.0, om);                /* (r0+1)^(1-beta) */
    z->b = pow((double)n + 1.0, om) - z->a;         /* (n+1)^(1-beta) - (r0+1)^(1-beta) */
    uint64_t mul = (draw(seed, 90, 0) % (uint64_t)n) | 1ULL;
    while (gcd_u64(mul, (uint64_t)n) != 1) mul += 2;
    z->perm_mul = mul % (uint64_t)n ? mul % (uint64_t)n : 1;
    z->perm_add = draw(seed, 91, 0) % (uint64_t)n;
}

static inline int64_t zipf_rank(const zipf_t* z, double u) {
    double om = 1.0 - z->beta;
    double x = pow(z->a + u * z->b, 1.0 / om) - 1.0;    /* in [r0, n) */
    int64_t r = (int64_t)x;
    if (r < z->r0) r = z->r0;
    if (r >= z->n) r = z->n - 1;
    return r;
}

static inline int64_t perm_node(const zipf_t* z, int64_t rank) {
    return (int64_t)(((__uint128_t)(uint64_t)rank * z->perm_mul + z->perm_add) % (uint64_t)z->n);
}

/* daily-modulated intensity: Lambda(t) = t + A (1 - cos(w t)), A = amp / w */
static double lambda_inv(double s, double w, double amp) {
    double A = amp / w;
    double t = s;                 /* Lambda(t) >= t - 0 and <= t + 2A */
    for (int it = 0; it < 40; ++it) {
        double f = t + A * (1.0 - cos(w * t)) - s;
        double fp = 1.0 + amp * sin(w * t);
        double nt = t - f / fp;
        if (nt < s - 2 * A) nt = s - 2 * A;
        if (nt > s) nt = s;
        if (fabs(nt - t) < 1e-7) { t = nt; break; }
        t = nt;
    }
    return t;
}

typedef struct {
    uint64_t seed;
    int64_t n, m_base, m_recip;
    double span, burst_frac, burst_mean, copy_p, amp;
    int64_t n_bursts;
    zipf_t zs;
    uint64_t rperm_mul, rperm_add;
    /* hub skew (0 => off): share of endpoints drawn from the top n_hubs ranks */
    double hub_share; int64_t n_hubs;
    int with_labels; int n_labels;
    int32_t *src, *dst; int64_t* t; uint8_t* elabel;
} pl_ctx;

static inline int64_t pl_endpoint(const pl_ctx* c, uint64_t stream, uint64_t e) {
    if (c->hub_share > 0.0 && unif(c->seed, stream + 100, e) < c->hub_share)
        return perm_node(&c->zs, (int64_t)below(c->seed, stream + 200, e, (uint64_t)c->n_hubs));
    return perm_node(&c->zs, zipf_rank(&c->zs, unif(c->seed, stream, e)));
}

static inline int64_t pl_src(const pl_ctx* c, int64_t e) { return pl_endpoint(c, 10, (uint64_t)e); }

/*
 * Destination by preferential attachment (copy model): with probability p the
 * edge copies the destination of a uniformly chosen earlier base edge, else the
 * destination is uniform over all nodes.  In-degree tail exponent 1 + 1/p.
 * Resolved by following the copy chain, so every edge is computed independently.
 */
static int64_t pl_dst_raw(const pl_ctx* c, int64_t e) {
    for (;;) {
        if (e == 0 || unif(c->seed, 20, (uint64_t)e) >= c->copy_p)
            return (int64_t)below(c->seed, 30, (uint64_t)e, (uint64_t)c->n);
        e = (int64_t)below(c->seed, 21, (uint64_t)e, (uint64_t)e);
    }
}

static inline int64_t pl_dst(const pl_ctx* c, int64_t e, int64_t s) {
    int64_t d = c->copy_p > 0.0 ? pl_dst_raw(c, e) : pl_endpoint(c, 30, (uint64_t)e);
    if (d == s) {                      /* no self-loops: uniform over the others */
        d = (int64_t)below(c->seed, 40, (uint64_t)e, (uint64_t)(c->n - 1));
        if (d >= s) d += 1;
    }
    return d;
}

static inline double pl_time(const pl_ctx* c, int64_t e) {
    double w = 2.0 * M_PI / 86400.0;
    double lam_total = c->span + (c->amp / w) * (1.0 - cos(w * c->span));
    if (c->n_bursts > 0 && unif(c->seed, 50, (uint64_t)e) < c->burst_frac) {
        int64_t b = (int64_t)below(c->seed, 51, (uint64_t)e, (uint64_t)c->n_bursts);
        double center = lambda_inv(unif(c->seed, 52, (uint64_t)b) * lam_total, w, c->amp);
        double off = -log(1.0 - unif(c->seed, 53, (uint64_t)e)) * c->burst_mean;
        double tt = center + off;
        if (tt >= c->span) tt = c->span - 1.0;
        return tt;
    }
    return lambda_inv(unif(c->seed, 54, (uint64_t)e) * lam_total, w, c->amp);
}

static void pl_body(void* p, int64_t lo, int64_t hi) {
    pl_ctx* c = (pl_ctx*)p;
    for (int64_t e = lo; e < hi; ++e) {
        if (e < c->m_base) {
            int64_t s = pl_src(c, e);
            int64_t d = pl_dst(c, e, s);
            double tt = pl_time(c, e);
            c->src[e] = (int32_t)s;
            c->dst[e] = (int32_t)d;
            c->t[e] = (int64_t)floor(tt);
            if (c->with_labels) c->elabel[e] = (uint8_t)below(c->seed, 60, (uint64_t)e, (uint64_t)c->n_labels);
        } else {
            /* reciprocal of a base edge j: (dst_j, src_j, t_j + U[1, 3600]) */
            int64_t r = e - c->m_base;
            int64_t j = (int64_t)(((__uint128_t)(uint64_t)r * c->rperm_mul + c->rperm_add) % (uint64_t)c->m_base);
            int64_t s = pl_src(c, j);
            int64_t d = pl_dst(c, j, s);
            int64_t tj = (int64_t)floor(pl_time(c, j));
            c->src[e] = (int32_t)d;
            c->dst[e] = (int32_t)s;
            c->t[e] = tj + 1 + (int64_t)below(c->seed, 70, (uint64_t)r, 3600);
            if (c->with_labels) c->elabel[e] = (uint8_t)below(c->seed, 60, (uint64_t)e, (uint64_t)c->n_labels);
        }
    }
}

/*
 * Power-law temporal graph.
 *   n, m        : nodes, total edges (base edges + reciprocals = m exactly)
 *   alpha       : degree tail exponent (out via Chung-Lu weights, in via copy model)
 *   span        : timestamps in [0, span) seconds, daily sinusoid amplitude amp
 *   recip_frac  : reciprocals per base edge (0.10 => 10% of base edges answered
 *                 within one hour)
 *   burst_frac  : share of base edges placed in bursts (exponential offsets of
 *                 mean burst_mean seconds around burst centres)
 *   hub_share, n_hubs : optional hub skew (share of endpoints on the top ranks)
 *   elabel      : optional (nullable) uint8 labels uniform in [0, n_labels)
 *   pa          : 1 = destinations by preferential attachment (copy model),
 *                 0 = destinations drawn like sources (hubs both send and receive)
 */
int synth_powerlaw(uint64_t seed, int64_t n, int64_t m, double alpha, double span,
                   double amp, double recip_frac, double burst_frac, double burst_mean,
                   double hub_share, int64_t n_hubs, int n_labels, int pa,
                   int32_t* src, int32_t* dst, int64_t* t, uint8_t* elabel, int nthreads) {
    if (n < 2 || m < 1 || alpha <= 1.0 || span < 1.0) return 1;
    pl_ctx c;
    memset(&c, 0, sizeof c);
    c.seed = seed; c.n = n; c.span = span; c.amp = amp;
    c.m_base = (int64_t)floor((double)m / (1.0 + recip_frac));
    if (c.m_base < 1) c.m_base = 1;
    if (c.m_base > m) c.m_base = m;
    c.m_recip = m - c.m_base;
    c.burst_frac = burst_frac; c.burst_mean = burst_mean;
    c.n_bursts = burst_frac > 0 ? (int64_t)(c.m_base * burst_frac / 50.0) + 1 : 0;
    /* pa != 0: destinations by preferential attachment (copy model);
       pa == 0: destinations drawn from the same popularity as sources */
    c.copy_p = pa ? 1.0 / (alpha - 1.0) : 0.0;
    if (c.copy_p > 0.98) c.copy_p = 0.98;
    c.hub_share = hub_share; c.n_hubs = n_hubs > 0 ? n_hubs : 1;
    zipf_init(&c.zs, n, alpha, seed, hub_share > 0.0 ? c.n_hubs : 0);
    uint64_t mul = (draw(seed, 92, 0) % (uint64_t)c.m_base) | 1ULL;
    while (gcd_u64(mul, (uint64_t)c.m_base) != 1) mul += 2;
    c.rperm_mul = mul; c.rperm_add = draw(seed, 93, 0) % (uint64_t)c.m_base;
    c.with_labels = elabel != NULL; c.n_labels = n_labels > 0 ? n_labels : 1;
    c.src = src; c.dst = dst; c.t = t; c.elabel = elabel;
    parallel_for(m, nthreads, pl_body, &c);
    return 0;
}

/* uint8 labels uniform in [0, n_labels) for n items (node or edge labels) */
typedef struct { uint64_t seed, stream; int n_labels; uint8_t* out; } lab_ctx;
static void lab_body(void* p, int64_t lo, int64_t hi) {
    lab_ctx* c = (lab_ctx*)p;
    for (int64_t i = lo; i < hi; ++i) c->out[i] = (uint8_t)below(c->seed, c->stream, (uint64_t)i, (uint64_t)c->n_labels);
}
int synth_labels(uint64_t seed, uint64_t stream, int64_t n, int n_labels, uint8_t* out, int nthreads) {
    if (n_labels < 1 || n_labels > 256) return 1;
    lab_ctx c = { seed, stream, n_labels, out };
    parallel_for(n, nthreads, lab_body, &c);
    return 0;
}

/* raw draws for Python-side recipes (query mixes, arrival traces) */
void synth_draws(uint64_t seed, uint64_t stream, int64_t n, uint64_t* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = draw(seed, stream, (uint64_t)i);
}
