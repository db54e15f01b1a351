/*
 * Seeded synthetic read libraries shaped like the paper's benchmark data
 * (Table 2: genomes of 10^8..10^9 bp, short reads, substitution errors, N calls).
 *
 * This file holds input generation only: genomes, reads, errors and N calls.
 * It contains none of the k-mer counting arithmetic. Both the CPU oracle and
 * the GPU path receive the bytes produced here.
 *
 * Randomness: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014), used counter-style: every (seed, purpose,
 * index) triple names an independent stream, so any genome block or read can be
 * produced on its own, in any order, by any thread, with identical results.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ull

static inline uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static inline uint64_t sm_next(uint64_t *s) {
    *s += GOLDEN;
    return sm_mix(*s);
}
/* uniform double in (0, 1] */
static inline double u01(uint64_t *s) { return ((sm_next(s) >> 11) + 1) * (1.0 / 9007199254740992.0); }
/* uniform integer in [0, range) (Lemire's multiply-shift reduction) */
static inline uint64_t below(uint64_t *s, uint64_t range) {
    return (uint64_t)(((unsigned __int128)sm_next(s) * range) >> 64);
}
static uint64_t stream(uint64_t seed, uint64_t purpose, uint64_t index) {
    return sm_mix(sm_mix(seed + purpose * 0xD1B54A32D192ED03ull) ^ (index * GOLDEN + 0x632BE59BD9B4E019ull));
}
/* number of Bernoulli(p) failures before the next success: geometric gap sampling */
static inline uint64_t gap(uint64_t *s, double log1mp) {
    double g = floor(log(u01(s)) / log1mp);
    return g > 1e18 ? (uint64_t)1e18 : (uint64_t)g;
}

static const char BASE[4] = {'A', 'C', 'G', 'T'};
static inline int code_of(char c) {
    switch (c) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    case 'T': return 3;
    default: return -1;
    }
}
static inline char comp(char c) {
    switch (c) {
    case 'A': return 'T';
    case 'C': return 'G';
    case 'G': return 'C';
    case 'T': return 'A';
    default: return c;
    }
}

/* ---------------------------------------------------------------- threads */
typedef void (*range_fn)(void *ctx, uint64_t lo, uint64_t hi);
typedef struct { range_fn fn; void *ctx; uint64_t lo, hi; } job_t;
static void *run_job(void *a) { job_t *j = (job_t *)a; j->fn(j->ctx, j->lo, j->hi); return NULL; }
static void parallel_for(uint64_t n, int threads, range_fn fn, void *ctx) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if ((uint64_t)threads > n) threads = n ? (int)n : 1;
    pthread_t tid[256];
    job_t jobs[256];
    for (int t = 0; t < threads; t++) {
        jobs[t].fn = fn; jobs[t].ctx = ctx;
        jobs[t].lo = n * t / threads; jobs[t].hi = n * (t + 1) / threads;
    }
    for (int t = 1; t < threads; t++) pthread_create(&tid[t], NULL, run_job, &jobs[t]);
    run_job(&jobs[0]);
    for (int t = 1; t < threads; t++) pthread_join(tid[t], NULL);
}

/* ---------------------------------------------------------------- genome */
#define GBLOCK 65536ull
typedef struct { uint64_t seed, len; char *out; } genome_ctx;
static void genome_range(void *c, uint64_t lo, uint64_t hi) {
    genome_ctx *g = (genome_ctx *)c;
    for (uint64_t b = lo; b < hi; b++) {
        uint64_t s = stream(g->seed, 1, b);
        uint64_t p0 = b * GBLOCK, p1 = p0 + GBLOCK < g->len ? p0 + GBLOCK : g->len;
        uint64_t word = 0;
        for (uint64_t p = p0; p < p1; p++) {
            if (((p - p0) & 31) == 0) word = sm_next(&s);
            g->out[p] = BASE[word & 3];
            word >>= 2;
        }
    }
}
/* iid uniform A/C/G/T genome of `len` bases */
void synth_genome_iid(uint64_t seed, uint64_t len, char *out, int threads) {
    genome_ctx g = {seed, len, out};
    parallel_for((len + GBLOCK - 1) / GBLOCK, threads, genome_range, &g);
}

typedef struct { uint64_t pos, src, len, copy_seed, order; } insert_t;
static int insert_cmp(const void *a, const void *b) {
    const insert_t *x = (const insert_t *)a, *y = (const insert_t *)b;
    if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
    return x->order < y->order ? -1 : (x->order > y->order);
}
/* Upper bound on the length synth_genome_repeats can produce. */
uint64_t synth_genome_repeats_cap(uint64_t base_len, double repeat_frac, int seg_max, int copy_max) {
    return base_len + (uint64_t)(repeat_frac * (double)base_len) + (uint64_t)seg_max * (uint64_t)copy_max + 16;
}
/*
 * iid genome of base_len bases plus repeat families: each family is a segment
 * of U[seg_min, seg_max] bases copied U[copy_min, copy_max] times, each copy with
 * iid substitutions at rate `divergence`, inserted at uniform positions, until
 * the inserted bases reach repeat_frac * base_len. Returns the final length.
 */
uint64_t synth_genome_repeats(uint64_t seed, uint64_t base_len, double repeat_frac, int seg_min, int seg_max,
                              int copy_min, int copy_max, double divergence, char *out, uint64_t out_cap,
                              int threads) {
    char *base = (char *)malloc(base_len ? base_len : 1);
    if (!base) return 0;
    synth_genome_iid(seed, base_len, base, threads);
    uint64_t s = stream(seed, 2, 0);
    uint64_t target = (uint64_t)(repeat_frac * (double)base_len), inserted = 0, n_ins = 0, cap_ins = 1024;
    insert_t *ins = (insert_t *)malloc(cap_ins * sizeof(insert_t));
    while (inserted < target && base_len >= (uint64_t)seg_max) {
        uint64_t L = seg_min + below(&s, (uint64_t)(seg_max - seg_min + 1));
        uint64_t c = copy_min + below(&s, (uint64_t)(copy_max - copy_min + 1));
        uint64_t src = below(&s, base_len - L + 1);
        for (uint64_t j = 0; j < c; j++) {
            if (n_ins == cap_ins) { cap_ins *= 2; ins = (insert_t *)realloc(ins, cap_ins * sizeof(insert_t)); }
            ins[n_ins].pos = below(&s, base_len + 1);
            ins[n_ins].src = src;
            ins[n_ins].len = L;
            ins[n_ins].copy_seed = sm_next(&s);
            ins[n_ins].order = n_ins;
            n_ins++;
            inserted += L;
        }
    }
    qsort(ins, n_ins, sizeof(insert_t), insert_cmp);
    uint64_t o = 0, cur = 0;
    double l1mp = log1p(-divergence);
    for (uint64_t i = 0; i < n_ins && o < out_cap; i++) {
        uint64_t take = ins[i].pos - cur;
        if (o + take > out_cap) take = out_cap - o;
        memcpy(out + o, base + cur, take);
        o += take; cur = ins[i].pos;
        uint64_t L = ins[i].len;
        if (o + L > out_cap) L = out_cap - o;
        memcpy(out + o, base + ins[i].src, L);
        if (divergence > 0) {
            uint64_t cs = ins[i].copy_seed;
            for (uint64_t p = gap(&cs, l1mp); p < L; p += 1 + gap(&cs, l1mp)) {
                int c0 = code_of(out[o + p]);
                out[o + p] = BASE[(c0 + 1 + (int)below(&cs, 3)) & 3];
            }
        }
        o += L;
    }
    uint64_t rest = base_len - cur;
    if (o + rest > out_cap) rest = out_cap - o;
    memcpy(out + o, base + cur, rest);
    o += rest;
    free(ins);
    free(base);
    return o;
}

/* ---------------------------------------------------------------- reads */
typedef struct {
    const char *genome; uint64_t G; uint64_t seed; int R; double err, nrate;
    char *bases; uint64_t *offsets; uint64_t first;   /* global index of the first read produced */
    const uint64_t *region_prefix; uint64_t n_regions, region_len; /* NULL: uniform starts */
} reads_ctx;

static uint64_t region_of(const uint64_t *prefix, uint64_t n_regions, uint64_t read) {
    uint64_t lo = 0, hi = n_regions; /* prefix[lo] <= read < prefix[hi] */
    while (hi - lo > 1) {
        uint64_t mid = (lo + hi) / 2;
        if (prefix[mid] <= read) lo = mid; else hi = mid;
    }
    return lo;
}

static void reads_range(void *c, uint64_t lo, uint64_t hi) {
    reads_ctx *r = (reads_ctx *)c;
    const int R = r->R;
    double le = r->err > 0 ? log1p(-r->err) : 0, ln = r->nrate > 0 ? log1p(-r->nrate) : 0;
    for (uint64_t i = lo; i < hi; i++) {
        uint64_t gi = r->first + i;
        uint64_t s = stream(r->seed, 3, gi);
        uint64_t start;
        if (r->region_prefix) {
            uint64_t reg = region_of(r->region_prefix, r->n_regions, gi);
            start = reg * r->region_len + below(&s, r->region_len);
        } else {
            start = below(&s, r->G - (uint64_t)R + 1);
        }
        if (start > r->G - (uint64_t)R) start = r->G - (uint64_t)R;
        int minus = (int)(sm_next(&s) & 1);
        char *dst = r->bases + i * (uint64_t)R;
        const char *src = r->genome + start;
        if (!minus) memcpy(dst, src, (size_t)R);
        else for (int j = 0; j < R; j++) dst[j] = comp(src[R - 1 - j]);
        if (r->err > 0)
            for (uint64_t p = gap(&s, le); p < (uint64_t)R; p += 1 + gap(&s, le)) {
                int c0 = code_of(dst[p]);
                dst[p] = BASE[(c0 + 1 + (int)below(&s, 3)) & 3];
            }
        if (r->nrate > 0)
            for (uint64_t p = gap(&s, ln); p < (uint64_t)R; p += 1 + gap(&s, ln)) dst[p] = 'N';
        r->offsets[i] = i * (uint64_t)R;
    }
}

/*
 * n_reads reads of R bases, starts uniform on [0, G-R], strand 50/50 (minus =
 * reverse complement), iid substitutions at rate err (uniform over the other 3
 * bases), then iid N calls at rate nrate. Reads first..first+n_reads-1 of the
 * stream named by seed are produced; offsets[0..n_reads] are local to `bases`.
 */
void synth_reads_uniform(const char *genome, uint64_t G, uint64_t seed, uint64_t first, uint64_t n_reads, int R,
                         double err, double nrate, char *bases, uint64_t *offsets, int threads) {
    reads_ctx c = {genome, G, seed, R, err, nrate, bases, offsets, first, NULL, 0, 0};
    parallel_for(n_reads, threads, reads_range, &c);
    offsets[n_reads] = n_reads * (uint64_t)R;
}

/*
 * Coverage plan for amplification-skewed libraries: region r of region_len
 * bases gets coverage median * exp(sigma * z_r), z_r standard normal
 * (Box-Muller), i.e. a log-normal with the given median; its read count is that
 * coverage * region_len / R, randomly rounded. Writes prefix[0..n_regions]
 * (prefix[r] = first read of region r) and returns the total read count.
 */
uint64_t synth_region_plan(uint64_t seed, uint64_t G, uint64_t region_len, double median, double sigma, int R,
                           uint64_t *prefix) {
    uint64_t n_regions = (G + region_len - 1) / region_len, total = 0;
    for (uint64_t r = 0; r < n_regions; r++) {
        uint64_t s = stream(seed, 4, r);
        double u1 = u01(&s), u2 = u01(&s);
        double z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
        double cov = median * exp(sigma * z);
        double expect = cov * (double)region_len / (double)R;
        uint64_t n = (uint64_t)floor(expect + u01(&s) - 1e-300);
        prefix[r] = total;
        total += n;
    }
    prefix[n_regions] = total;
    return total;
}

/* Reads first..first+n_reads-1 of a region plan (see synth_region_plan). */
void synth_reads_regions(const char *genome, uint64_t G, uint64_t seed, const uint64_t *prefix, uint64_t n_regions,
                         uint64_t region_len, uint64_t first, uint64_t n_reads, int R, double err, double nrate,
                         char *bases, uint64_t *offsets, int threads) {
    reads_ctx c = {genome, G, seed, R, err, nrate, bases, offsets, first, prefix, n_regions, region_len};
    parallel_for(n_reads, threads, reads_range, &c);
    offsets[n_reads] = n_reads * (uint64_t)R;
}
