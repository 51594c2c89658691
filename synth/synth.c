/*
 * Seeded synthetic protein inputs: residue codes and sequence lengths.
 *
 * This module holds only random-number generation and table lookups. It
 * contains none of the Smith-Waterman arithmetic; both the CPU oracle and the
 * GPU library are fed from it. Every function is integer-only so that x86-64
 * and aarch64 produce identical bytes for the same seed.
 *
 * Generators, written from their published definitions:
 *   - splitmix64 (Steele, Lea, Flood 2014) for seeding and counter hashing;
 *   - xoshiro256** (Blackman, Vigna 2018) for per-sequence residue streams.
 */
#include <stdint.h>
#include <stddef.h>
#include <pthread.h>

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

/* splitmix64: advance the state by the golden-ratio increment, then mix. */
static inline uint64_t splitmix64_next(uint64_t* state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Counter-based draw: one splitmix64 output keyed by (seed, stream, index). */
static inline uint64_t keyed_draw(uint64_t seed, uint64_t stream, uint64_t index) {
    uint64_t s = seed ^ (stream * 0xD1B54A32D192ED03ULL);
    (void)splitmix64_next(&s);
    s ^= index * 0xA0761D6478BD642FULL;
    return splitmix64_next(&s);
}

typedef struct { uint64_t s[4]; } xoshiro_t;

static inline void xoshiro_seed(xoshiro_t* g, uint64_t key) {
    uint64_t sm = key;
    for (int i = 0; i < 4; ++i) g->s[i] = splitmix64_next(&sm);
}

/* xoshiro256**: scrambled output rotl(s1*5, 7)*9, then the linear update. */
static inline uint64_t xoshiro_next(xoshiro_t* g) {
    uint64_t* s = g->s;
    const uint64_t out = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

/* Draw a code from integer weights: cdf[c] = sum of weights 0..c, total = cdf[A-1]. */
static inline uint8_t draw_code(xoshiro_t* g, const uint32_t* cdf, uint32_t A) {
    const uint32_t total = cdf[A - 1];
    const uint32_t u = (uint32_t)(((xoshiro_next(g) >> 32) * (uint64_t)total) >> 32);
    uint32_t c = 0;
    while (c + 1 < A && cdf[c] <= u) ++c;
    return (uint8_t)c;
}

/* out[i] = qtable[top 16 bits of keyed_draw(seed, stream, i)], i < n. */
void synth_lengths(uint64_t seed, uint64_t stream, uint64_t n, const uint32_t* qtable,
                   uint32_t* out) {
    for (uint64_t i = 0; i < n; ++i) out[i] = qtable[keyed_draw(seed, stream, i) >> 48];
}

typedef struct {
    uint64_t seed, stream;
    const uint64_t* offsets;
    uint64_t first, last;
    const uint32_t* cdf;
    uint32_t A;
    uint8_t* out;
} residue_job;

static void* residue_worker(void* arg) {
    residue_job* j = (residue_job*)arg;
    for (uint64_t s = j->first; s < j->last; ++s) {
        xoshiro_t g;
        xoshiro_seed(&g, keyed_draw(j->seed, j->stream, s));
        for (uint64_t p = j->offsets[s]; p < j->offsets[s + 1]; ++p)
            j->out[p] = draw_code(&g, j->cdf, j->A);
    }
    return NULL;
}

/*
 * Fill out[offsets[s] .. offsets[s+1]) for every sequence s < n_seqs with
 * i.i.d. codes drawn by weight. Sequence s uses its own xoshiro stream keyed by
 * (seed, stream, s), so the bytes do not depend on the thread count.
 */
int synth_residues(uint64_t seed, uint64_t stream, const uint64_t* offsets, uint64_t n_seqs,
                   const uint32_t* cdf, uint32_t A, uint8_t* out, int nthreads) {
    if (A == 0 || A > 256) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 64) nthreads = 64;
    pthread_t th[64];
    residue_job jobs[64];
    const uint64_t total = offsets[n_seqs] - offsets[0];
    int threaded[64] = {0};
    uint64_t s = 0;
    for (int t = 0; t < nthreads; ++t) {
        /* split by residue count so threads get equal work */
        const uint64_t target = offsets[0] + total * (uint64_t)(t + 1) / (uint64_t)nthreads;
        uint64_t e = s;
        while (e < n_seqs && offsets[e] < target) ++e;
        if (t == nthreads - 1) e = n_seqs;
        jobs[t] = (residue_job){seed, stream, offsets, s, e, cdf, A, out};
        if (pthread_create(&th[t], NULL, residue_worker, &jobs[t]) == 0)
            threaded[t] = 1;
        else
            residue_worker(&jobs[t]);
        s = e;
    }
    for (int t = 0; t < nthreads; ++t)
        if (threaded[t]) pthread_join(th[t], NULL);
    return 0;
}

/*
 * Near-duplicate of src: each position is replaced, with probability
 * rate_per_10000 / 10000, by a different code drawn by weight.
 */
void synth_mutate(uint64_t seed, uint64_t stream, uint64_t index, const uint8_t* src, uint64_t len,
                  const uint32_t* cdf, uint32_t A, uint32_t rate_per_10000, uint8_t* out) {
    xoshiro_t g;
    xoshiro_seed(&g, keyed_draw(seed, stream, index));
    for (uint64_t p = 0; p < len; ++p) {
        const uint32_t u = (uint32_t)(((xoshiro_next(&g) >> 32) * 10000ULL) >> 32);
        uint8_t c = src[p];
        if (u < rate_per_10000 && A > 1) {
            uint8_t r;
            do { r = draw_code(&g, cdf, A); } while (r == c);
            c = r;
        }
        out[p] = c;
    }
}

/* Uniform integers in [lo, hi]: out[i] = lo + floor(draw * (hi-lo+1) / 2^32). */
void synth_uniform_u32(uint64_t seed, uint64_t stream, uint64_t n, uint32_t lo, uint32_t hi,
                       uint32_t* out) {
    const uint64_t span = (uint64_t)hi - lo + 1;
    for (uint64_t i = 0; i < n; ++i)
        out[i] = lo + (uint32_t)(((keyed_draw(seed, stream, i) >> 32) * span) >> 32);
}

/* Raw 64-bit keyed draws, for positions, arrival times and other host-side choices. */
void synth_draws(uint64_t seed, uint64_t stream, uint64_t n, uint64_t* out) {
    for (uint64_t i = 0; i < n; ++i) out[i] = keyed_draw(seed, stream, i);
}
