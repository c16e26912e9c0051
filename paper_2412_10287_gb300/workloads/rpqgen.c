/*
 * Seeded synthetic-input generators for single-source 2-RPQ workloads.
 *
 * This file holds random-number generation and graph/query sampling only:
 * no part of the query method (no traversal, no automaton) lives here.  Both
 * the CPU oracle and the GPU library consume its outputs.
 *
 * Determinism: every output is a pure function of (parameters, seed) and is
 * bit-identical on x86-64 and aarch64.  Floating point is limited to IEEE
 * basic operations (+ - * /, frexp/ldexp/floor, all exactly specified), the
 * file must be compiled with -ffp-contract=off so that no fused multiply-add
 * changes a rounding, and logarithm/exponential are computed by the series
 * below rather than by the platform libm (whose last-bit results differ
 * between libraries).
 *
 * PRNG: xoshiro256** (Blackman & Vigna, "Scrambled linear pseudorandom number
 * generators", 2018) seeded through splitmix64 (Steele, Lea & Flood 2014).
 * Discrete distributions are sampled with Vose's alias method (Vose 1991).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define EXPORT __attribute__((visibility("default")))

/* ----------------------------------------------------------------- PRNG -- */

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t result = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* One independent stream per (seed, stream id). */
static void rng_seed(rng_t *r, uint64_t seed, uint64_t stream) {
    uint64_t x = seed ^ (0xD1B54A32D192ED03ULL * (stream + 1));
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64_next(&x);
}

/* uniform integer in [0, k) by 64x64->128 multiply (Lemire 2019). */
static inline uint64_t rng_below(rng_t *r, uint64_t k) {
    return (uint64_t)(((unsigned __int128)rng_next(r) * k) >> 64);
}

/* uniform double in [0, 1) with 53 random bits. */
static inline double rng_unit(rng_t *r) {
    return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------- deterministic log / exp ------ */

static const double LN2 = 0.69314718055994530942;

/* natural log for x > 0: x = m 2^e with m in [sqrt(1/2), sqrt(2)), then
 * ln m = 2 atanh(t), t = (m-1)/(m+1), |t| < 0.172, by its odd power series. */
static double det_log(double x) {
    int e;
    double m = frexp(x, &e); /* m in [0.5, 1) */
    if (m < 0.70710678118654752440) { m *= 2.0; e -= 1; }
    double t = (m - 1.0) / (m + 1.0);
    double t2 = t * t, term = t, sum = 0.0;
    for (int k = 1; k <= 41; k += 2) { sum += term / (double)k; term *= t2; }
    return 2.0 * sum + (double)e * LN2;
}

/* exp(y): y = k ln2 + r, |r| <= ln2/2, Taylor series for exp(r). */
static double det_exp(double y) {
    double k = floor(y / LN2 + 0.5);
    double r = y - k * LN2;
    double term = 1.0, sum = 1.0;
    for (int i = 1; i <= 27; i++) { term = term * r / (double)i; sum += term; }
    return ldexp(sum, (int)k);
}

static double det_pow(double x, double y) { return det_exp(y * det_log(x)); }

/* ------------------------------------------------------- alias tables ---- */

typedef struct { int64_t n; double *prob; int64_t *alias; } alias_t;

static int alias_build(alias_t *a, const double *w, int64_t n) {
    a->n = n;
    a->prob = (double *)malloc(sizeof(double) * (size_t)n);
    a->alias = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *small = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *large = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    if (!a->prob || !a->alias || !small || !large || !p) {
        free(a->prob); free(a->alias); free(small); free(large); free(p);
        return -1;
    }
    double total = 0.0;
    for (int64_t i = 0; i < n; i++) total += w[i];
    int64_t ns = 0, nl = 0;
    for (int64_t i = 0; i < n; i++) {
        p[i] = w[i] * (double)n / total;
        if (p[i] < 1.0) small[ns++] = i; else large[nl++] = i;
    }
    while (ns > 0 && nl > 0) {
        int64_t s = small[--ns], l = large[--nl];
        a->prob[s] = p[s];
        a->alias[s] = l;
        p[l] = (p[l] + p[s]) - 1.0;
        if (p[l] < 1.0) small[ns++] = l; else large[nl++] = l;
    }
    while (nl > 0) { int64_t l = large[--nl]; a->prob[l] = 1.0; a->alias[l] = l; }
    while (ns > 0) { int64_t s = small[--ns]; a->prob[s] = 1.0; a->alias[s] = s; }
    free(small); free(large); free(p);
    return 0;
}

static void alias_free(alias_t *a) { free(a->prob); free(a->alias); }

static inline int64_t alias_draw(const alias_t *a, rng_t *r) {
    int64_t i = (int64_t)rng_below(r, (uint64_t)a->n);
    double u = rng_unit(r);
    return u < a->prob[i] ? i : a->alias[i];
}

/* Zipf(s) weights over ranks 1..k (rank 1 = label 0, the most frequent). */
static double *zipf_weights(int64_t k, double s) {
    double *w = (double *)malloc(sizeof(double) * (size_t)k);
    if (!w) return NULL;
    for (int64_t i = 0; i < k; i++) w[i] = 1.0 / det_pow((double)(i + 1), s);
    return w;
}

static void shuffle_i32(int32_t *v, int64_t n, rng_t *r) {
    for (int64_t i = n - 1; i > 0; i--) {
        int64_t j = (int64_t)rng_below(r, (uint64_t)(i + 1));
        int32_t t = v[i]; v[i] = v[j]; v[j] = t;
    }
}

/* ----------------------------------------------------------- exports ----- */

EXPORT int rpqgen_version(void) { return 1; }

/* Raw PRNG draws of stream `stream` under `seed`. */
EXPORT int rpqgen_draw_u64(uint64_t seed, uint64_t stream, int64_t count, uint64_t *out) {
    rng_t r; rng_seed(&r, seed, stream);
    for (int64_t i = 0; i < count; i++) out[i] = rng_next(&r);
    return 0;
}

/* Uniform integers in [0, bound). */
EXPORT int rpqgen_below(uint64_t seed, uint64_t stream, int64_t count, uint64_t bound, int64_t *out) {
    if (bound == 0) return -1;
    rng_t r; rng_seed(&r, seed, stream);
    for (int64_t i = 0; i < count; i++) out[i] = (int64_t)rng_below(&r, bound);
    return 0;
}

/* Zipf(s) ranks in [0, k). */
EXPORT int rpqgen_zipf(int64_t k, double s, uint64_t seed, uint64_t stream, int64_t count, int32_t *out) {
    if (k <= 0) return -1;
    double *w = zipf_weights(k, s);
    if (!w) return -2;
    alias_t a;
    if (alias_build(&a, w, k)) { free(w); return -2; }
    rng_t r; rng_seed(&r, seed, stream);
    for (int64_t i = 0; i < count; i++) out[i] = (int32_t)alias_draw(&a, &r);
    alias_free(&a); free(w);
    return 0;
}

/* Exponential variates with the given rate (Poisson inter-arrival gaps). */
EXPORT int rpqgen_exponential(double rate, uint64_t seed, uint64_t stream, int64_t count, double *out) {
    if (!(rate > 0.0)) return -1;
    rng_t r; rng_seed(&r, seed, stream);
    for (int64_t i = 0; i < count; i++) {
        double u = 1.0 - rng_unit(&r); /* (0, 1] */
        out[i] = -det_log(u) / rate;
    }
    return 0;
}

EXPORT double rpqgen_det_pow(double x, double y) { return det_pow(x, y); }
EXPORT double rpqgen_det_log(double x) { return det_log(x); }
EXPORT double rpqgen_det_exp(double x) { return det_exp(x); }

/*
 * Directed Erdos-Renyi G(n, M): M distinct ordered pairs (u, v), u != v,
 * uniform; labels uniform over [0, L).  n <= 16384 (pair bitmap).
 */
EXPORT int rpqgen_er(int64_t n, int64_t m, int32_t L, uint64_t seed,
                     int32_t *src, int32_t *dst, int32_t *lab) {
    if (n < 2 || n > 16384 || m < 0 || m > n * (n - 1) || L <= 0) return -1;
    uint64_t nbits = (uint64_t)n * (uint64_t)n;
    uint64_t *seen = (uint64_t *)calloc((nbits + 63) / 64, sizeof(uint64_t));
    if (!seen) return -2;
    rng_t r; rng_seed(&r, seed, 0);
    rng_t rl; rng_seed(&rl, seed, 1);
    int64_t k = 0;
    while (k < m) {
        int64_t u = (int64_t)rng_below(&r, (uint64_t)n);
        int64_t v = (int64_t)rng_below(&r, (uint64_t)n);
        if (u == v) continue;
        uint64_t b = (uint64_t)u * (uint64_t)n + (uint64_t)v;
        if (seen[b >> 6] & (1ULL << (b & 63))) continue;
        seen[b >> 6] |= 1ULL << (b & 63);
        src[k] = (int32_t)u; dst[k] = (int32_t)v;
        lab[k] = (int32_t)rng_below(&rl, (uint64_t)L);
        k++;
    }
    free(seen);
    return 0;
}

/*
 * R-MAT (Chakrabarti, Zhan & Faloutsos 2004): `samples` edges on 2^scale
 * vertices, quadrant probabilities (a, b, c, 1-a-b-c) at every level, vertex
 * ids then relabelled by a seeded random permutation.  Labels Zipf(zipf_s)
 * over [0, L).  Duplicates and self-loops are kept (the consumer decides).
 */
EXPORT int rpqgen_rmat(int32_t scale, int64_t samples, double a, double b, double c,
                       int32_t L, double zipf_s, uint64_t seed,
                       int32_t *src, int32_t *dst, int32_t *lab) {
    if (scale < 1 || scale > 30 || samples < 0 || L <= 0) return -1;
    const double two32 = 4294967296.0;
    uint64_t ta = (uint64_t)floor(a * two32);
    uint64_t tb = ta + (uint64_t)floor(b * two32);
    uint64_t tc = tb + (uint64_t)floor(c * two32);
    int64_t n = (int64_t)1 << scale;
    rng_t r; rng_seed(&r, seed, 0);
    for (int64_t i = 0; i < samples; i++) {
        uint64_t u = 0, v = 0, x = 0;
        for (int lv = 0; lv < scale; lv++) {
            uint64_t q;
            if ((lv & 1) == 0) { x = rng_next(&r); q = x >> 32; } else { q = x & 0xFFFFFFFFULL; }
            uint64_t bu, bv;
            if (q < ta) { bu = 0; bv = 0; }
            else if (q < tb) { bu = 0; bv = 1; }
            else if (q < tc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu; v = (v << 1) | bv;
        }
        src[i] = (int32_t)u; dst[i] = (int32_t)v;
    }
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!perm) return -2;
    for (int64_t i = 0; i < n; i++) perm[i] = (int32_t)i;
    rng_t rp; rng_seed(&rp, seed, 1);
    shuffle_i32(perm, n, &rp);
    for (int64_t i = 0; i < samples; i++) { src[i] = perm[src[i]]; dst[i] = perm[dst[i]]; }
    free(perm);
    int rc = rpqgen_zipf(L, zipf_s, seed, 2, samples, lab);
    return rc;
}

/*
 * Chung-Lu style power-law graph: `m` edges on `n` vertices; the source of
 * each edge is drawn with weight (i+1)^(-1/(gamma-1)) (out-degree tail
 * exponent gamma), the destination with the same weights under an
 * independent random permutation of the ids.  Labels Zipf(zipf_s) over
 * [0, L).  Duplicates and self-loops are kept.
 */
EXPORT int rpqgen_chung_lu(int64_t n, int64_t m, double gamma, int32_t L, double zipf_s,
                           uint64_t seed, int32_t *src, int32_t *dst, int32_t *lab) {
    if (n < 1 || n > 2147483647LL || m < 0 || L <= 0 || !(gamma > 1.0)) return -1;
    double expo = 1.0 / (gamma - 1.0);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    if (!w) return -2;
    for (int64_t i = 0; i < n; i++) w[i] = 1.0 / det_pow((double)(i + 1), expo);
    alias_t al;
    if (alias_build(&al, w, n)) { free(w); return -2; }
    free(w);
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!perm) { alias_free(&al); return -2; }
    for (int64_t i = 0; i < n; i++) perm[i] = (int32_t)i;
    rng_t rp; rng_seed(&rp, seed, 3);
    shuffle_i32(perm, n, &rp);
    rng_t rs; rng_seed(&rs, seed, 0);
    rng_t rd; rng_seed(&rd, seed, 1);
    for (int64_t i = 0; i < m; i++) {
        src[i] = (int32_t)alias_draw(&al, &rs);
        dst[i] = perm[alias_draw(&al, &rd)];
    }
    free(perm);
    alias_free(&al);
    return rpqgen_zipf(L, zipf_s, seed, 2, m, lab);
}
