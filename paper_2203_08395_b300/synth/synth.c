/*
 * synth.c -- seeded synthetic inputs for the task-graph executor and its oracle.
 *
 * This file holds none of the method's arithmetic: it never propagates arrivals and never
 * runs a payload. It only draws graph shapes (edge lists), edge delays, task picks, payload
 * sizes and payload data from seeded generators, so that the CUDA path and the CPU oracle
 * can be fed byte-identical inputs.
 *
 * Generators used (written from their published definitions):
 *   - splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
 *     OOPSLA 2014) to expand a 64-bit seed and as a counter-based hash for element data;
 *   - xoshiro256** (Blackman, Vigna, "Scrambled linear pseudorandom number generators",
 *     2018/2021) for sequential streams;
 *   - Box-Muller for normal deviates (lognormal delays).
 *
 * Memory returned in synth_dag is malloc'ed here and released by synth_dag_free.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct synth_dag {
    int32_t n;        /* tasks */
    int32_t levels;   /* construction levels (0 when not layered) */
    int64_t m;        /* edges */
    int32_t* src;     /* m predecessor ids */
    int32_t* dst;     /* m successor ids */
    float* delay;     /* m edge delays */
} synth_dag;

/* ---------------------------------------------------------------- generators */

static uint64_t sm64_next(uint64_t* x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } rng_t;

static void rng_init(rng_t* r, uint64_t seed, uint64_t stream) {
    uint64_t x = seed ^ sm64_mix(stream + 0x632BE59BD9B4E019ull);
    for (int i = 0; i < 4; ++i) r->s[i] = sm64_next(&x);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_u64(rng_t* r) {
    uint64_t* s = r->s;
    const uint64_t out = rotl64(s[1] * 5u, 7) * 9u;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

/* uniform double in [0,1) with 53 random bits */
static double rng_unit(rng_t* r) { return (double)(rng_u64(r) >> 11) * 0x1.0p-53; }

/* uniform integer in [0, n) for n >= 1 (multiply-shift; bias < n / 2^64, irrelevant here) */
static int64_t rng_below(rng_t* r, int64_t n) {
    unsigned __int128 p = (unsigned __int128)rng_u64(r) * (unsigned __int128)(uint64_t)n;
    return (int64_t)(p >> 64);
}

static double rng_normal(rng_t* r) {
    double u1 = rng_unit(r);
    double u2 = rng_unit(r);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}

/* ---------------------------------------------------------------- edge buffer */

typedef struct {
    int64_t m, cap;
    int32_t* src;
    int32_t* dst;
    float* delay;
} ebuf;

static int eb_push(ebuf* b, int32_t s, int32_t d, float w) {
    if (b->m == b->cap) {
        int64_t nc = b->cap ? b->cap * 2 : 1024;
        int32_t* ns = (int32_t*)realloc(b->src, (size_t)nc * sizeof(int32_t));
        if (!ns) return -1;
        b->src = ns;
        int32_t* nd = (int32_t*)realloc(b->dst, (size_t)nc * sizeof(int32_t));
        if (!nd) return -1;
        b->dst = nd;
        float* nw = (float*)realloc(b->delay, (size_t)nc * sizeof(float));
        if (!nw) return -1;
        b->delay = nw;
        b->cap = nc;
    }
    b->src[b->m] = s;
    b->dst[b->m] = d;
    b->delay[b->m] = w;
    b->m++;
    return 0;
}

static void eb_free(ebuf* b) {
    free(b->src);
    free(b->dst);
    free(b->delay);
    memset(b, 0, sizeof(*b));
}

static int eb_out(ebuf* b, int32_t n, int32_t levels, synth_dag* out) {
    out->n = n;
    out->levels = levels;
    out->m = b->m;
    out->src = b->src;
    out->dst = b->dst;
    out->delay = b->delay;
    return 0;
}

void synth_dag_free(synth_dag* d) {
    if (!d) return;
    free(d->src);
    free(d->dst);
    free(d->delay);
    memset(d, 0, sizeof(*d));
}

/* delay distributions: kind 0 = uniform [p0, p1), kind 1 = lognormal exp(p0 + p1 * z) */
static float draw_delay(rng_t* r, int kind, double p0, double p1) {
    if (kind == 1) return (float)exp(p0 + p1 * rng_normal(r));
    return (float)(p0 + (p1 - p0) * rng_unit(r));
}

static int contains(const int32_t* a, int k, int32_t x) {
    for (int i = 0; i < k; ++i)
        if (a[i] == x) return 1;
    return 0;
}

static inline int64_t level_start(int64_t l, int64_t n, int64_t levels) { return l * n / levels; }

/*
 * Layered DAG: n tasks spread evenly over `levels` construction levels, ids in level order.
 * Each task of level l >= 1 draws k ~ U{fin_lo..fin_hi} predecessors (at most the number of
 * earlier tasks): the first uniformly from level l-1 (so the depth is exactly `levels`), the
 * rest distinct and uniform over all earlier levels. Level-0 tasks are the sources.
 */
int synth_layered(uint64_t seed, int32_t n, int32_t levels, int32_t fin_lo, int32_t fin_hi,
                  int delay_kind, double p0, double p1, synth_dag* out) {
    if (!out || n <= 0 || levels <= 0 || levels > n || fin_lo < 1 || fin_hi < fin_lo || fin_hi > 64)
        return -1;
    rng_t r;
    rng_init(&r, seed, 1);
    ebuf b = {0};
    int32_t picked[64];
    for (int64_t l = 1; l < levels; ++l) {
        const int64_t s0 = level_start(l, n, levels), s1 = level_start(l + 1, n, levels);
        const int64_t p_lo = level_start(l - 1, n, levels);
        for (int64_t v = s0; v < s1; ++v) {
            int k = fin_lo + (int)rng_below(&r, fin_hi - fin_lo + 1);
            if (k > s0) k = (int)s0;
            int got = 0;
            picked[got++] = (int32_t)(p_lo + rng_below(&r, s0 - p_lo));
            while (got < k) {
                int32_t u = (int32_t)rng_below(&r, s0);
                if (!contains(picked, got, u)) picked[got++] = u;
            }
            for (int i = 0; i < got; ++i)
                if (eb_push(&b, picked[i], (int32_t)v, draw_delay(&r, delay_kind, p0, p1))) {
                    eb_free(&b);
                    return -2;
                }
        }
    }
    return eb_out(&b, n, levels, out);
}

/* binary search: first index i in [lo, hi) with cw[i] > x (cw non-decreasing) */
static int64_t upper_idx(const int64_t* cw, int64_t lo, int64_t hi, int64_t x) {
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (cw[mid] > x) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* draw an id in [a, b) with probability proportional to weight (cw = inclusive prefix sums) */
static int64_t draw_weighted(rng_t* r, const int64_t* cw, int64_t a, int64_t b) {
    const int64_t base = a > 0 ? cw[a - 1] : 0;
    const int64_t tot = cw[b - 1] - base;
    return upper_idx(cw, a, b, base + rng_below(r, tot));
}

/*
 * Circuit-like DAG: n tasks over `levels` construction levels (ids in level order).
 * Fan-in k ~ Geometric(p) on {1,2,...}, redrawn while k > fin_max. Every task gets an
 * attractiveness w ~ P(w) ∝ w^-alpha on {1..wmax}; predecessors are drawn ∝ w (first from
 * level l-1, the rest from all earlier levels), rejecting duplicates and tasks whose fan-out
 * already reached fout_max. Delays: lognormal exp(mu + sigma z).
 */
int synth_circuit(uint64_t seed, int32_t n, int32_t levels, double p_geom, int32_t fin_max,
                  double alpha, int32_t wmax, int32_t fout_max, double mu, double sigma,
                  synth_dag* out) {
    if (!out || n <= 0 || levels <= 0 || levels > n || fin_max < 1 || fin_max > 64 || wmax < 1 ||
        p_geom <= 0.0 || p_geom >= 1.0 || fout_max < 1)
        return -1;
    rng_t r;
    rng_init(&r, seed, 2);
    double* cdf = (double*)malloc((size_t)wmax * sizeof(double));
    int64_t* cw = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    int32_t* fout = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    if (!cdf || !cw || !fout) {
        free(cdf); free(cw); free(fout);
        return -2;
    }
    double acc = 0.0;
    for (int32_t w = 1; w <= wmax; ++w) {
        acc += pow((double)w, -alpha);
        cdf[w - 1] = acc;
    }
    int64_t run = 0;
    for (int64_t i = 0; i < n; ++i) {
        const double u = rng_unit(&r) * acc;
        int32_t lo = 0, hi = wmax - 1;
        while (lo < hi) {
            int32_t mid = (lo + hi) / 2;
            if (cdf[mid] > u) hi = mid; else lo = mid + 1;
        }
        run += lo + 1;
        cw[i] = run;
    }
    const double lq = log1p(-p_geom);
    ebuf b = {0};
    int32_t picked[64];
    int rc = 0;
    for (int64_t l = 1; l < levels && rc == 0; ++l) {
        const int64_t s0 = level_start(l, n, levels), s1 = level_start(l + 1, n, levels);
        const int64_t p_lo = level_start(l - 1, n, levels);
        for (int64_t v = s0; v < s1 && rc == 0; ++v) {
            int k;
            do {
                double u = rng_unit(&r);
                if (u < 1e-300) u = 1e-300;
                k = 1 + (int)floor(log(u) / lq);
            } while (k > fin_max);
            if (k > s0) k = (int)s0;
            int got = 0;
            for (int want = 0; want < k; ++want) {
                const int64_t a = want == 0 ? p_lo : 0;
                int32_t u = -1;
                for (int t = 0; t < 64 && u < 0; ++t) {
                    int32_t c = (int32_t)draw_weighted(&r, cw, a, s0);
                    if (fout[c] < fout_max && !contains(picked, got, c)) u = c;
                }
                for (int t = 0; t < 64 && u < 0; ++t) {
                    int32_t c = (int32_t)(a + rng_below(&r, s0 - a));
                    if (fout[c] < fout_max && !contains(picked, got, c)) u = c;
                }
                if (u < 0 && want == 0) u = (int32_t)(a + rng_below(&r, s0 - a));
                if (u < 0) continue;
                picked[got++] = u;
                fout[u]++;
            }
            for (int i = 0; i < got; ++i)
                if (eb_push(&b, picked[i], (int32_t)v, draw_delay(&r, 1, mu, sigma))) rc = -2;
        }
    }
    free(cdf);
    free(cw);
    free(fout);
    if (rc) {
        eb_free(&b);
        return rc;
    }
    return eb_out(&b, n, levels, out);
}

/*
 * Random DAG with ids in topological order: task 0 is the only source; task v >= 1 draws
 * k ~ U{fin_lo..fin_hi} distinct predecessors uniformly from [max(0, v - window), v)
 * (window <= 0: from [0, v)), capped at the size of that range.
 */
int synth_random(uint64_t seed, int32_t n, int32_t fin_lo, int32_t fin_hi, int32_t window,
                 double d0, double d1, synth_dag* out) {
    if (!out || n <= 0 || fin_lo < 1 || fin_hi < fin_lo || fin_hi > 64) return -1;
    rng_t r;
    rng_init(&r, seed, 3);
    ebuf b = {0};
    int32_t picked[64];
    for (int64_t v = 1; v < n; ++v) {
        const int64_t lo = (window > 0 && v > window) ? v - window : 0;
        const int64_t range = v - lo;
        int k = fin_lo + (int)rng_below(&r, fin_hi - fin_lo + 1);
        if (k > range) k = (int)range;
        int got = 0;
        while (got < k) {
            int32_t u = (int32_t)(lo + rng_below(&r, range));
            if (!contains(picked, got, u)) picked[got++] = u;
        }
        for (int i = 0; i < got; ++i)
            if (eb_push(&b, picked[i], (int32_t)v, draw_delay(&r, 0, d0, d1))) {
                eb_free(&b);
                return -2;
            }
    }
    return eb_out(&b, n, 0, out);
}

/* k distinct ids from [0, n), ascending (partial Fisher-Yates, then sort). */
static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

int synth_pick(uint64_t seed, uint64_t stream, int32_t n, int32_t k, int32_t* out) {
    if (n < 0 || k < 0 || k > n || (k > 0 && !out)) return -1;
    rng_t r;
    rng_init(&r, seed, 0x100000000ull + stream);
    int32_t* idx = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!idx) return -2;
    for (int32_t i = 0; i < n; ++i) idx[i] = i;
    for (int32_t i = 0; i < k; ++i) {
        int32_t j = i + (int32_t)rng_below(&r, n - i);
        int32_t t = idx[i];
        idx[i] = idx[j];
        idx[j] = t;
    }
    memcpy(out, idx, (size_t)k * sizeof(int32_t));
    free(idx);
    qsort(out, (size_t)k, sizeof(int32_t), cmp_i32);
    return 0;
}

/* k integers log-uniform on [lo, hi]: floor(exp(U(ln lo, ln(hi+1)))) clamped to [lo, hi] */
int synth_loguniform(uint64_t seed, uint64_t stream, int64_t k, int64_t lo, int64_t hi, int64_t* out) {
    if (k < 0 || lo < 1 || hi < lo || (k > 0 && !out)) return -1;
    rng_t r;
    rng_init(&r, seed, 0x200000000ull + stream);
    const double a = log((double)lo), b = log((double)hi + 1.0);
    for (int64_t i = 0; i < k; ++i) {
        int64_t v = (int64_t)floor(exp(a + (b - a) * rng_unit(&r)));
        if (v < lo) v = lo;
        if (v > hi) v = hi;
        out[i] = v;
    }
    return 0;
}

/* uniform draws in [lo, hi) from a sequential stream */
int synth_uniform_f32(uint64_t seed, uint64_t stream, int64_t k, double lo, double hi, float* out) {
    if (k < 0 || (k > 0 && !out)) return -1;
    rng_t r;
    rng_init(&r, seed, 0x300000000ull + stream);
    for (int64_t i = 0; i < k; ++i) out[i] = (float)(lo + (hi - lo) * rng_unit(&r));
    return 0;
}

/* Counter-based element data: value(seed, stream, i) depends only on its arguments, so any
 * element of a large buffer can be regenerated on its own. */
static inline uint64_t elem_hash(uint64_t seed, uint64_t stream, uint64_t i) {
    return sm64_mix(sm64_mix(seed ^ 0x5851F42D4C957F2Dull) ^ sm64_mix(stream * 0x9E3779B97F4A7C15ull + 1) ^
                    (i * 0xD1B54A32D192ED03ull));
}

float synth_value_f32(uint64_t seed, uint64_t stream, int64_t i, double lo, double hi) {
    const double u = (double)(elem_hash(seed, stream, (uint64_t)i) >> 40) * 0x1.0p-24;
    return (float)(lo + (hi - lo) * u);
}

int32_t synth_value_i32(uint64_t seed, uint64_t stream, int64_t i, int32_t lo, int32_t hi) {
    const uint64_t span = (uint64_t)((int64_t)hi - (int64_t)lo) + 1u;
    return (int32_t)((int64_t)lo + (int64_t)((elem_hash(seed, stream, (uint64_t)i) >> 16) % span));
}

int synth_fill_f32(uint64_t seed, uint64_t stream, int64_t first, int64_t n, double lo, double hi, float* out) {
    if (n < 0 || (n > 0 && !out)) return -1;
#pragma omp parallel for schedule(static) if (n > (1 << 20))
    for (int64_t i = 0; i < n; ++i) out[i] = synth_value_f32(seed, stream, first + i, lo, hi);
    return 0;
}

int synth_fill_i32(uint64_t seed, uint64_t stream, int64_t first, int64_t n, int32_t lo, int32_t hi, int32_t* out) {
    if (n < 0 || hi < lo || (n > 0 && !out)) return -1;
#pragma omp parallel for schedule(static) if (n > (1 << 20))
    for (int64_t i = 0; i < n; ++i) out[i] = synth_value_i32(seed, stream, first + i, lo, hi);
    return 0;
}

/* Many counter-based buffers at once: buffer j (stream streams[j], counts[j] elements) is
 * written at out + offsets[j]; same values as synth_fill_f32 / synth_fill_i32 per buffer. */
int synth_fill_multi_f32(uint64_t seed, int64_t k, const uint64_t* streams, const int64_t* counts,
                         const int64_t* offsets, double lo, double hi, float* out) {
    if (k < 0 || (k > 0 && (!streams || !counts || !offsets || !out))) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < k; ++j) {
        float* o = out + offsets[j];
        for (int64_t i = 0; i < counts[j]; ++i) o[i] = synth_value_f32(seed, streams[j], i, lo, hi);
    }
    return 0;
}

int synth_fill_multi_i32(uint64_t seed, int64_t k, const uint64_t* streams, const int64_t* counts,
                         const int64_t* offsets, int32_t lo, int32_t hi, int32_t* out) {
    if (k < 0 || hi < lo || (k > 0 && (!streams || !counts || !offsets || !out))) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < k; ++j) {
        int32_t* o = out + offsets[j];
        for (int64_t i = 0; i < counts[j]; ++i) o[i] = synth_value_i32(seed, streams[j], i, lo, hi);
    }
    return 0;
}
