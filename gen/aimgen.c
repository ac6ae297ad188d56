/*
 * Seeded synthetic read/target pairs, shared by the tests, the benchmark and
 * the oracle timing.  This file holds no alignment arithmetic: it only draws
 * random DNA and applies random edits, so both the CUDA path and the oracle
 * can be fed the same inputs.
 *
 * Workload shapes follow the paper's datasets (Section 3.1, Table 2): reads of
 * a fixed length or of a length drawn log-uniformly from a range, targets made
 * from the read by a given fraction of edits (substitution, insertion or
 * deletion, equally likely), optionally a fraction of unrelated targets.
 *
 * Random numbers: xoshiro256** (Blackman and Vigna, 2018) seeded through
 * splitmix64.  Pair i uses its own stream seeded with seed ^ (i * 0x9E3779B97F4A7C15),
 * so any pair can be regenerated from its index alone.
 *
 * Build: gcc -O2 -fPIC -shared -fopenmp aimgen.c -o libaimgen.so
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct {
    uint64_t seed;
    uint32_t len_min, len_max;   /* equal: fixed length; else log-uniform over [len_min, len_max] */
    double rate_min, rate_max;   /* equal: fixed edit rate; else uniform over [rate_min, rate_max] */
    double unrelated_frac;       /* probability that a pair's target is an independent random sequence */
} aimgen_spec;

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t next_u64(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t result = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return result;
}

static void rng_init(rng_t *r, uint64_t seed, uint64_t pair) {
    uint64_t x = seed ^ (pair * 0x9E3779B97F4A7C15ULL);
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

/* uniform double in [0, 1) from the top 53 bits */
static double next_unit(rng_t *r) { return (double)(next_u64(r) >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0, bound) by multiply-shift on the top 32 bits */
static uint32_t next_below(rng_t *r, uint32_t bound) {
    return (uint32_t)(((next_u64(r) >> 32) * (uint64_t)bound) >> 32);
}

static const char BASES[4] = {'A', 'C', 'G', 'T'};

typedef struct {
    uint32_t n;          /* read length */
    uint32_t unrelated;  /* 1: independent target */
    uint32_t edits;      /* number of edits applied (0 for unrelated) */
    double rate;
} pair_params;

static pair_params draw_params(const aimgen_spec *sp, rng_t *r) {
    pair_params p;
    if (sp->len_min == sp->len_max) {
        p.n = sp->len_min;
    } else {
        double la = log((double)sp->len_min), lb = log((double)sp->len_max);
        double v = floor(exp(la + (lb - la) * next_unit(r)));
        if (v < sp->len_min) v = sp->len_min;
        if (v > sp->len_max) v = sp->len_max;
        p.n = (uint32_t)v;
    }
    p.rate = (sp->rate_min == sp->rate_max) ? sp->rate_min
                                            : sp->rate_min + (sp->rate_max - sp->rate_min) * next_unit(r);
    p.unrelated = (sp->unrelated_frac > 0.0 && next_unit(r) < sp->unrelated_frac) ? 1u : 0u;
    double e = floor(p.rate * (double)p.n + 0.5);
    if (e > p.n) e = p.n;
    p.edits = p.unrelated ? 0u : (uint32_t)e;
    return p;
}

/*
 * Generate one pair into caller buffers.  read must hold n bytes, target n + edits bytes.
 * pos_scratch must hold n uint32.  Returns the target length.
 */
static uint32_t gen_one(const aimgen_spec *sp, uint64_t idx, char *read, char *target, uint32_t *pos_scratch,
                        pair_params *out_p, uint32_t *n_sub, uint32_t *n_ins, uint32_t *n_del) {
    rng_t r;
    rng_init(&r, sp->seed, idx);
    pair_params p = draw_params(sp, &r);
    *out_p = p;
    *n_sub = *n_ins = *n_del = 0;
    for (uint32_t j = 0; j < p.n; ++j) read[j] = BASES[next_u64(&r) >> 62];
    if (p.unrelated) {
        for (uint32_t j = 0; j < p.n; ++j) target[j] = BASES[next_u64(&r) >> 62];
        return p.n;
    }
    /* edit positions without replacement: partial Fisher-Yates over [0, n) */
    for (uint32_t j = 0; j < p.n; ++j) pos_scratch[j] = j;
    for (uint32_t j = 0; j < p.edits; ++j) {
        uint32_t k = j + next_below(&r, p.n - j);
        uint32_t t = pos_scratch[j]; pos_scratch[j] = pos_scratch[k]; pos_scratch[k] = t;
    }
    /* sort the chosen positions descending (insertion sort: edits are few) */
    for (uint32_t a = 1; a < p.edits; ++a) {
        uint32_t v = pos_scratch[a]; int32_t b = (int32_t)a - 1;
        while (b >= 0 && pos_scratch[b] < v) { pos_scratch[b + 1] = pos_scratch[b]; --b; }
        pos_scratch[b + 1] = v;
    }
    memcpy(target, read, p.n);
    uint32_t m = p.n;
    for (uint32_t j = 0; j < p.edits; ++j) {
        uint32_t pos = pos_scratch[j];
        uint32_t kind = next_below(&r, 3);
        if (kind == 0) {            /* substitution: one of the three other bases */
            uint32_t code = 0;
            while (BASES[code] != target[pos]) ++code;
            target[pos] = BASES[(code + 1 + next_below(&r, 3)) & 3];
            ++*n_sub;
        } else if (kind == 1) {     /* insertion of a uniform base before pos */
            memmove(target + pos + 1, target + pos, m - pos);
            target[pos] = BASES[next_u64(&r) >> 62];
            ++m; ++*n_ins;
        } else {                    /* deletion of the base at pos */
            memmove(target + pos, target + pos + 1, m - pos - 1);
            --m; ++*n_del;
        }
    }
    return m;
}

/*
 * Pass 1: per-pair read length, target length and edit counts for pairs
 * [first, first + count).  Any output pointer may be NULL.
 */
int aimgen_sizes(const aimgen_spec *sp, uint64_t first, uint64_t count, uint32_t *read_len, uint32_t *target_len,
                 uint32_t *n_sub, uint32_t *n_ins, uint32_t *n_del, uint8_t *unrelated) {
    int err = 0;
#pragma omp parallel
    {
        uint32_t cap = sp->len_max + 1;
        char *rb = (char *)malloc(cap), *tb = (char *)malloc(2 * (size_t)cap + 1);
        uint32_t *ps = (uint32_t *)malloc(sizeof(uint32_t) * cap);
        if (!rb || !tb || !ps) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 256)
            for (uint64_t i = 0; i < count; ++i) {
                pair_params p; uint32_t s, a, d;
                uint32_t m = gen_one(sp, first + i, rb, tb, ps, &p, &s, &a, &d);
                if (read_len) read_len[i] = p.n;
                if (target_len) target_len[i] = m;
                if (n_sub) n_sub[i] = s;
                if (n_ins) n_ins[i] = a;
                if (n_del) n_del[i] = d;
                if (unrelated) unrelated[i] = (uint8_t)p.unrelated;
            }
        }
        free(rb); free(tb); free(ps);
    }
    return err ? -1 : 0;
}

/*
 * Pass 2: write the ASCII bytes of pairs [first, first + count) at the given
 * byte offsets (relative to the buffers).  Lengths must come from aimgen_sizes.
 */
int aimgen_fill(const aimgen_spec *sp, uint64_t first, uint64_t count, char *reads, const uint64_t *read_off,
                char *targets, const uint64_t *target_off) {
    int err = 0;
#pragma omp parallel
    {
        uint32_t cap = sp->len_max + 1;
        char *rb = (char *)malloc(cap), *tb = (char *)malloc(2 * (size_t)cap + 1);
        uint32_t *ps = (uint32_t *)malloc(sizeof(uint32_t) * cap);
        if (!rb || !tb || !ps) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 256)
            for (uint64_t i = 0; i < count; ++i) {
                pair_params p; uint32_t s, a, d;
                uint32_t m = gen_one(sp, first + i, rb, tb, ps, &p, &s, &a, &d);
                memcpy(reads + read_off[i], rb, p.n);
                memcpy(targets + target_off[i], tb, m);
            }
        }
        free(rb); free(tb); free(ps);
    }
    return err ? -1 : 0;
}

/* Log-uniform request sizes and exponential inter-arrival gaps for an open-loop arrival process. */
int aimgen_arrivals(uint64_t seed, uint64_t count, double rate_per_s, uint32_t size_min, uint32_t size_max,
                    double *arrival_s, uint32_t *size) {
    rng_t r;
    rng_init(&r, seed, 0xA11A11ULL);
    double t = 0.0, la = log((double)size_min), lb = log((double)size_max);
    for (uint64_t i = 0; i < count; ++i) {
        double u = next_unit(&r);
        t += -log(1.0 - u) / rate_per_s;
        arrival_s[i] = t;
        double v = floor(exp(la + (lb - la) * next_unit(&r)));
        if (v < size_min) v = size_min;
        if (v > size_max) v = size_max;
        size[i] = (uint32_t)v;
    }
    return 0;
}
