/*
 * Seeded synthetic inputs for the sorter's tests and benchmarks.
 *
 * This module only draws records; it holds none of the sorting arithmetic.  Both the
 * CPU oracle and the GPU sorter receive the bytes it writes, so the two sides always
 * see identical inputs.
 *
 * Every value is counter based: record i of a stream depends only on (seed, stream, i).
 * So any slice of a workload can be generated alone (first_index), in any thread split,
 * and gives the same bytes.
 *
 * Generator: SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014).  Output i of a SplitMix64 stream with state k is
 * mix(k + (i + 1) * gamma), gamma = 0x9e3779b97f4a7c15, where mix is the 64-bit finaliser
 * published with it.  Stream s of seed x uses state k = mix(x + (s + 1) * gamma).
 *
 * Record layout written here: rec_size bytes = 8-byte little-endian words.  The key is
 * the first key_size bytes (read as a little-endian unsigned integer).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <string.h>

#define GAMMA 0x9e3779b97f4a7c15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Output i of stream `stream` for seed `seed`. */
uint64_t wl_u64(uint64_t seed, uint64_t stream, uint64_t i) {
    uint64_t k = mix64(seed + (stream + 1) * GAMMA);
    return mix64(k + (i + 1) * GAMMA);
}

/* Uniform double in [0, 1) from the top 53 bits. */
static inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

/* Streams used by the record fillers. */
enum { ST_KEY = 0, ST_PAYLOAD = 64, ST_ZIPF = 200, ST_KMER_PICK = 300, ST_KMER_TABLE = 301,
       ST_BIJ_A = 400, ST_BIJ_B = 401 };

/* ---------------------------------------------------------------- threading */
typedef struct {
    void (*fn)(void *ctx, uint64_t lo, uint64_t hi);
    void *ctx;
    uint64_t lo, hi;
} job_t;

static void *run_job(void *p) {
    job_t *j = (job_t *)p;
    j->fn(j->ctx, j->lo, j->hi);
    return 0;
}

static void parallel_for(uint64_t n, int threads, void (*fn)(void *, uint64_t, uint64_t), void *ctx) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if (n < 65536 || threads == 1) { fn(ctx, 0, n); return; }
    pthread_t th[256];
    int ok[256];
    job_t jobs[256];
    uint64_t per = (n + threads - 1) / threads;
    int used = 0;
    for (int t = 0; t < threads; t++) {
        uint64_t lo = (uint64_t)t * per, hi = lo + per;
        if (lo >= n) break;
        if (hi > n) hi = n;
        jobs[t].fn = fn; jobs[t].ctx = ctx; jobs[t].lo = lo; jobs[t].hi = hi;
        ok[t] = pthread_create(&th[t], 0, run_job, &jobs[t]) == 0;
        if (!ok[t]) fn(ctx, lo, hi);     /* no thread: do the slice here */
        used = t + 1;
    }
    for (int t = 0; t < used; t++) if (ok[t]) pthread_join(th[t], 0);
}

/* ------------------------------------------------------------ record fillers */
typedef struct {
    uint8_t *buf;
    uint32_t rec_words, key_words;
    uint64_t seed, first;
    int kind;          /* 0 uniform, 1 zipf, 2 kmer */
    double zipf_s;
    uint64_t zipf_n;
    uint64_t bij_a, bij_b;
    const uint64_t *kmer_table;
    uint32_t kmer_prefixes;
} fill_t;

/* --- Zipf by rejection-inversion (W. Hormann, G. Derflinger, "Rejection-inversion to
 * generate variates from monotone discrete distributions", ACM TOMACS 6(3), 1996).
 * The weight of rank k is h(k) = k^-s on k = 1..N.  H is an antiderivative of h; a draw
 * inverts H at a uniform point between H(N + 1/2) and H(3/2) - h(1), rounds to the
 * nearest rank k, and accepts when the point lies under the step h(k) on [k-1/2, k+1/2]
 * (or when k is close enough to the continuous inverse that no test is needed). */
static double zipf_expm1_over(double t) { return fabs(t) > 1e-8 ? expm1(t) / t : 1.0 + t * 0.5 * (1.0 + t / 3.0); }
static double zipf_log1p_over(double t) { return fabs(t) > 1e-8 ? log1p(t) / t : 1.0 - t * (0.5 - t / 3.0); }
static double zipf_h(double x, double s) { return exp(-s * log(x)); }
static double zipf_H(double x, double s) { double lx = log(x); return zipf_expm1_over((1.0 - s) * lx) * lx; }
static double zipf_Hinv(double y, double s) { double t = y * (1.0 - s); if (t < -1.0) t = -1.0; return exp(zipf_log1p_over(t) * y); }

uint64_t wl_zipf_rank(uint64_t seed, uint64_t i, double s, uint64_t n_ranks) {
    double hx1 = zipf_H(1.5, s) - 1.0;
    double hn = zipf_H((double)n_ranks + 0.5, s);
    double sc = 2.0 - zipf_Hinv(zipf_H(2.5, s) - zipf_h(2.0, s), s);
    for (uint64_t attempt = 0;; attempt++) {
        double u = hn + u01(wl_u64(seed, ST_ZIPF + attempt % 64, i + (attempt / 64) * 0x100000000ULL)) * (hx1 - hn);
        double x = zipf_Hinv(u, s);
        double kf = floor(x + 0.5);
        if (kf < 1.0) kf = 1.0;
        if (kf > (double)n_ranks) kf = (double)n_ranks;
        if (kf - x <= sc || u >= zipf_H(kf + 0.5, s) - zipf_h(kf, s)) return (uint64_t)kf;
    }
}

/* A seeded bijection of the 64-bit integers: xor, SplitMix64 finaliser (xor-shifts and
 * odd multiplies, each invertible), xor. */
static inline uint64_t bijection(uint64_t x, uint64_t a, uint64_t b) { return mix64(x ^ a) ^ b; }

static void fill_range(void *vctx, uint64_t lo, uint64_t hi) {
    fill_t *c = (fill_t *)vctx;
    uint64_t *w = (uint64_t *)c->buf;
    for (uint64_t r = lo; r < hi; r++) {
        uint64_t i = c->first + r;
        uint64_t *rec = w + r * c->rec_words;
        uint32_t next = 0;
        if (c->kind == 0) {
            for (uint32_t k = 0; k < c->key_words; k++) rec[k] = wl_u64(c->seed, ST_KEY + k, i);
            next = c->key_words;
        } else if (c->kind == 1) {
            uint64_t rank = wl_zipf_rank(c->seed, i, c->zipf_s, c->zipf_n);
            rec[0] = bijection(rank, c->bij_a, c->bij_b);
            next = 1;
        } else {
            uint64_t pick = wl_u64(c->seed, ST_KMER_PICK, i) % c->kmer_prefixes;
            rec[0] = wl_u64(c->seed, ST_KEY, i);          /* bases 32..63: least significant word */
            rec[1] = c->kmer_table[pick];                  /* bases 0..31: most significant word */
            next = 2;
        }
        if (next < c->rec_words) rec[next++] = i;          /* payload: the record's original index */
        for (uint32_t k = next; k < c->rec_words; k++) rec[k] = wl_u64(c->seed, ST_PAYLOAD + k, i);
    }
}

/* Uniform keys: the first ceil(key_size/8) words are i.i.d. uniform, then the index, then
 * uniform payload words.  rec_size must be a multiple of 8. */
int wl_fill_uniform(uint8_t *buf, uint64_t n, uint32_t rec_size, uint32_t key_size, uint64_t seed,
                    uint64_t first_index, int threads) {
    if (rec_size == 0 || rec_size % 8 || key_size == 0 || key_size > rec_size) return -1;
    fill_t c; memset(&c, 0, sizeof c);
    c.buf = buf; c.rec_words = rec_size / 8; c.key_words = (key_size + 7) / 8;
    c.seed = seed; c.first = first_index; c.kind = 0;
    parallel_for(n, threads, fill_range, &c);
    return 0;
}

/* Zipf(s) ranks over 1..n_ranks mapped through a seeded bijection to an 8-byte key,
 * then the index, then uniform payload words. */
int wl_fill_zipf(uint8_t *buf, uint64_t n, uint32_t rec_size, uint64_t seed, double s, uint64_t n_ranks,
                 uint64_t first_index, int threads) {
    if (rec_size == 0 || rec_size % 8 || s <= 0.0 || n_ranks == 0) return -1;
    fill_t c; memset(&c, 0, sizeof c);
    c.buf = buf; c.rec_words = rec_size / 8; c.key_words = 1;
    c.seed = seed; c.first = first_index; c.kind = 1; c.zipf_s = s; c.zipf_n = n_ranks;
    c.bij_a = wl_u64(seed, ST_BIJ_A, 0); c.bij_b = wl_u64(seed, ST_BIJ_B, 0);
    parallel_for(n, threads, fill_range, &c);
    return 0;
}

uint64_t wl_zipf_key_of_rank(uint64_t seed, uint64_t rank) {
    return bijection(rank, wl_u64(seed, ST_BIJ_A, 0), wl_u64(seed, ST_BIJ_B, 0));
}

/* The i-th of the distinct 32-mers used as most significant key words (A,C,G,T = 0..3,
 * 2 bits per base, base 0 in the top bits): a uniform 64-bit value, made distinct from the
 * earlier ones by re-drawing on a clash. */
static uint64_t kmer_prefix(uint64_t seed, uint32_t j, const uint64_t *earlier) {
    for (uint64_t attempt = 0;; attempt++) {
        uint64_t v = wl_u64(seed, ST_KMER_TABLE, (uint64_t)j + attempt * 0x100000000ULL);
        int clash = 0;
        for (uint32_t q = 0; q < j; q++) if (earlier[q] == v) { clash = 1; break; }
        if (!clash) return v;
    }
}

int wl_kmer_table(uint64_t seed, uint32_t prefixes, uint64_t *out) {
    for (uint32_t j = 0; j < prefixes; j++) out[j] = kmer_prefix(seed, j, out);
    return 0;
}

/* 64-mer keys of 16 bytes: the most significant word (bytes 8..15) is one of `prefixes`
 * distinct random 32-mers picked uniformly; the least significant word (bytes 0..7) is a
 * uniform random 32-mer; then the index; then uniform payload words. */
int wl_fill_kmer(uint8_t *buf, uint64_t n, uint32_t rec_size, uint64_t seed, uint32_t prefixes,
                 uint64_t first_index, int threads, uint64_t *table_scratch) {
    if (rec_size < 16 || rec_size % 8 || prefixes == 0) return -1;
    wl_kmer_table(seed, prefixes, table_scratch);
    fill_t c; memset(&c, 0, sizeof c);
    c.buf = buf; c.rec_words = rec_size / 8; c.key_words = 2;
    c.seed = seed; c.first = first_index; c.kind = 2;
    c.kmer_table = table_scratch; c.kmer_prefixes = prefixes;
    parallel_for(n, threads, fill_range, &c);
    return 0;
}

/* Log-uniform integers in [lo, hi]: floor(exp(ln lo + U (ln(hi+1) - ln lo))), clamped. */
int wl_log_uniform(uint64_t *out, uint64_t m, uint64_t lo, uint64_t hi, uint64_t seed) {
    if (lo == 0 || hi < lo) return -1;
    double a = log((double)lo), b = log((double)hi + 1.0);
    for (uint64_t i = 0; i < m; i++) {
        double v = floor(exp(a + u01(wl_u64(seed, 0, i)) * (b - a)));
        if (v < (double)lo) v = (double)lo;
        if (v > (double)hi) v = (double)hi;
        out[i] = (uint64_t)v;
    }
    return 0;
}

/* Exponential inter-arrival gaps with the given rate (events per unit time). */
int wl_exponential(double *out, uint64_t m, double rate, uint64_t seed) {
    if (rate <= 0) return -1;
    for (uint64_t i = 0; i < m; i++) out[i] = -log1p(-u01(wl_u64(seed, 1, i))) / rate;
    return 0;
}

/* Uniform integers in [0, bound) (bound > 0), by multiply-high of a 64-bit draw. */
int wl_uniform_below(uint64_t *out, uint64_t m, uint64_t bound, uint64_t seed, uint64_t stream) {
    if (bound == 0) return -1;
    for (uint64_t i = 0; i < m; i++) {
        unsigned __int128 p = (unsigned __int128)wl_u64(seed, stream, i) * bound;
        out[i] = (uint64_t)(p >> 64);
    }
    return 0;
}
