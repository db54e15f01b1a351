/*
 * CPU oracle for the Turtle frequent k-mer method (Roy, Bhattacharya & Schliep,
 * arXiv:1305.1861). TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * benchmark's CPU-baseline leg may call it; the library never does.
 *
 * Plain, slow, obviously correct. It shares nothing with the CUDA path.
 *
 * What the method computes (Sec. 2.1.1 Outline, Sec. 2.1.2, Sec. 2.1.4, Alg. 1):
 * the frequency of every k-mer in a read library, where a k-mer and its reverse
 * complement are one object (Sec. 2.1.1), represented by the numerically smaller
 * of the two 2-bit encodings (Sec. 2.1.2); reads are split at ambiguous calls so
 * that every k-mer holds only A, C, G, T (Sec. 2.1.2); k-mers whose frequency
 * reaches the cutoff are reported with their counts (Sec. 2.1.1, Alg. 1). The Bloom
 * filter and the sort-and-compact array only make this faster; the exact result
 * is the plain definition written out below.
 *
 * Readings where the paper is silent:
 *  - code A=0, C=1, G=2, T=3 and complement x -> 3-x (numeric order then equals
 *    lexicographic order of the strings);
 *  - the first base of a window is the most significant 2-bit digit;
 *  - any byte other than A/C/G/T (either case) is an ambiguous call;
 *  - "frequency greater than the chosen cutoff" is read as count >= min_count;
 *  - keys are 64-bit for k <= 32 and 128-bit for 33 <= k <= 64 (Sec. 3).
 *
 * The pattern-blocked Bloom filter (Sec. 2.1.3, after Putze et al.) is also
 * written out sequentially here so that its false-positive behaviour can be
 * pinned against the blocked-Bloom formula and the GPU filter compared with it.
 */
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <thread>
#include <utility>
#include <vector>

typedef unsigned __int128 u128;

extern "C" {
typedef struct {
    uint64_t n;         /* reported (key, count) pairs */
    int words;          /* 1 (k <= 32) or 2 (k > 32, stored hi then lo) */
    uint64_t *keys;     /* n * words */
    uint64_t *counts;   /* n */
    uint64_t n_windows; /* number of valid windows seen */
} oracle_result;
}

/* Sec. 2.1.2: two bits per nucleotide; anything else splits the read. */
static inline int code_of(uint8_t c) {
    switch (c) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return -1;
    }
}

/*
 * Canonical key of the window read[p .. p+k), or false if the window holds an
 * ambiguous call. fwd puts base 0 in the most significant digit; rc is the
 * encoding of the reverse complement (its first base is the complement of the
 * window's last base). Sec. 2.1.2: keep the numerically smaller.
 */
template <class K>
static inline bool canonical_at(const uint8_t *read, int k, K *out) {
    K fwd = 0, rc = 0;
    for (int j = 0; j < k; j++) {
        int c = code_of(read[j]);
        if (c < 0) return false;
        fwd = (K)((fwd << 2) | (K)c);
        rc |= (K)(3 - c) << (2 * j);
    }
    *out = fwd < rc ? fwd : rc;
    return true;
}

template <class K>
static void windows_of_reads(const uint8_t *bases, const uint64_t *off, uint64_t r0, uint64_t r1, int k,
                             std::vector<K> &keys) {
    for (uint64_t r = r0; r < r1; r++) {
        uint64_t len = off[r + 1] - off[r];
        if (len < (uint64_t)k) continue;
        const uint8_t *read = bases + off[r];
        for (uint64_t p = 0; p + k <= len; p++) {
            K key;
            if (canonical_at<K>(read + p, k, &key)) keys.push_back(key);
        }
    }
}

/* Sort-and-compact (Sec. 2.1.4): sort, then replace each run of equal keys by one (key, run length). */
template <class K>
static void sort_and_compact(std::vector<K> &keys, std::vector<std::pair<K, uint64_t>> &out) {
    std::sort(keys.begin(), keys.end());
    for (size_t i = 0; i < keys.size();) {
        size_t j = i;
        while (j < keys.size() && keys[j] == keys[i]) j++;
        out.push_back(std::make_pair(keys[i], (uint64_t)(j - i)));
        i = j;
    }
}

template <class K> static void put_key(uint64_t *dst, K key, int words);
template <> void put_key<uint64_t>(uint64_t *dst, uint64_t key, int) { dst[0] = key; }
template <> void put_key<u128>(uint64_t *dst, u128 key, int) {
    dst[0] = (uint64_t)(key >> 64);
    dst[1] = (uint64_t)key;
}

template <class K>
static int count_impl(const uint8_t *bases, const uint64_t *off, uint64_t n_reads, int k, uint64_t min_count,
                      int threads, oracle_result *res) {
    if (threads < 1) threads = 1;
    if ((uint64_t)threads > n_reads) threads = n_reads ? (int)n_reads : 1;
    std::vector<std::vector<std::pair<K, uint64_t>>> part(threads);
    std::vector<uint64_t> nw(threads, 0);
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; t++)
        pool.emplace_back([&, t]() {
            std::vector<K> keys;
            windows_of_reads<K>(bases, off, n_reads * t / threads, n_reads * (t + 1) / threads, k, keys);
            nw[t] = keys.size();
            sort_and_compact<K>(keys, part[t]);
        });
    for (auto &th : pool) th.join();
    /* merge the per-thread compacted arrays: concatenate, sort by key, add up equal keys */
    std::vector<std::pair<K, uint64_t>> all;
    uint64_t n_windows = 0;
    for (int t = 0; t < threads; t++) {
        all.insert(all.end(), part[t].begin(), part[t].end());
        n_windows += nw[t];
        std::vector<std::pair<K, uint64_t>>().swap(part[t]);
    }
    std::sort(all.begin(), all.end(),
              [](const std::pair<K, uint64_t> &a, const std::pair<K, uint64_t> &b) { return a.first < b.first; });
    std::vector<std::pair<K, uint64_t>> merged;
    for (size_t i = 0; i < all.size();) {
        size_t j = i;
        uint64_t c = 0;
        while (j < all.size() && all[j].first == all[i].first) c += all[j++].second;
        if (c >= min_count) merged.push_back(std::make_pair(all[i].first, c));
        i = j;
    }
    int words = sizeof(K) / 8;
    res->n = merged.size();
    res->words = words;
    res->n_windows = n_windows;
    res->keys = (uint64_t *)malloc((merged.size() * words + 1) * 8);
    res->counts = (uint64_t *)malloc((merged.size() + 1) * 8);
    if (!res->keys || !res->counts) return -2;
    for (size_t i = 0; i < merged.size(); i++) {
        put_key<K>(res->keys + i * words, merged[i].first, words);
        res->counts[i] = merged[i].second;
    }
    return 0;
}

template <class K>
static int count_map_impl(const uint8_t *bases, const uint64_t *off, uint64_t n_reads, int k, uint64_t min_count,
                          oracle_result *res) {
    std::map<K, uint64_t> m;
    uint64_t n_windows = 0;
    for (uint64_t r = 0; r < n_reads; r++) {
        uint64_t len = off[r + 1] - off[r];
        for (uint64_t p = 0; p + k <= len; p++) {
            K key;
            if (canonical_at<K>(bases + off[r] + p, k, &key)) {
                m[key]++;
                n_windows++;
            }
        }
    }
    int words = sizeof(K) / 8;
    uint64_t n = 0;
    for (auto &kv : m) n += kv.second >= min_count;
    res->n = n;
    res->words = words;
    res->n_windows = n_windows;
    res->keys = (uint64_t *)malloc((n * words + 1) * 8);
    res->counts = (uint64_t *)malloc((n + 1) * 8);
    if (!res->keys || !res->counts) return -2;
    uint64_t i = 0;
    for (auto &kv : m)
        if (kv.second >= min_count) {
            put_key<K>(res->keys + i * words, kv.first, words);
            res->counts[i++] = kv.second;
        }
    return 0;
}

static int check_args(const uint64_t *off, uint64_t n_reads, int k) {
    if (k < 1 || k > 64 || !off) return -1;
    for (uint64_t r = 0; r < n_reads; r++)
        if (off[r + 1] < off[r]) return -1;
    return 0;
}

/* ---------------------------------------------------------------- MurmurHash3 / SplitMix64
 * Block selection hashes with the 64-bit finaliser of MurmurHash3 (Appleby,
 * public domain); 128-bit keys hash as fmix64(lo ^ fmix64(hi)). The pattern
 * table is drawn with SplitMix64 (Steele, Lea & Flood 2014). */
static inline uint64_t fmix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}
static inline uint64_t splitmix64_next(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" {

int oracle_count(const uint8_t *bases, const uint64_t *offsets, uint64_t n_reads, int k, uint64_t min_count,
                 int threads, oracle_result *res) {
    memset(res, 0, sizeof(*res));
    if (check_args(offsets, n_reads, k)) return -1;
    if (k <= 32) return count_impl<uint64_t>(bases, offsets, n_reads, k, min_count, threads, res);
    return count_impl<u128>(bases, offsets, n_reads, k, min_count, threads, res);
}

/* The same definition counted in a std::map (for small inputs). */
int oracle_count_map(const uint8_t *bases, const uint64_t *offsets, uint64_t n_reads, int k, uint64_t min_count,
                     oracle_result *res) {
    memset(res, 0, sizeof(*res));
    if (check_args(offsets, n_reads, k)) return -1;
    if (k <= 32) return count_map_impl<uint64_t>(bases, offsets, n_reads, k, min_count, res);
    return count_map_impl<u128>(bases, offsets, n_reads, k, min_count, res);
}

void oracle_result_free(oracle_result *res) {
    if (!res) return;
    free(res->keys);
    free(res->counts);
    memset(res, 0, sizeof(*res));
}

/*
 * Every valid window in read order: pos[i] = offset of its first base within
 * `bases`, keys[i*words ..] its canonical key (hi word first for k > 32).
 * Returns the number of windows (writes at most cap).
 */
uint64_t oracle_windows(const uint8_t *bases, const uint64_t *off, uint64_t n_reads, int k, uint64_t *pos,
                        uint64_t *keys, uint64_t cap) {
    uint64_t n = 0;
    int words = k <= 32 ? 1 : 2;
    for (uint64_t r = 0; r < n_reads; r++) {
        uint64_t len = off[r + 1] - off[r];
        for (uint64_t p = 0; p + k <= len; p++) {
            const uint8_t *w = bases + off[r] + p;
            bool ok;
            if (k <= 32) {
                uint64_t key;
                ok = canonical_at<uint64_t>(w, k, &key);
                if (ok && n < cap) keys[n] = key;
            } else {
                u128 key;
                ok = canonical_at<u128>(w, k, &key);
                if (ok && n < cap) put_key<u128>(keys + n * 2, key, 2);
            }
            if (ok) {
                if (n < cap) pos[n] = off[r] + p;
                n++;
            }
        }
    }
    (void)words;
    return n;
}

/* Sort-and-compact of an arbitrary key array (Sec. 2.1.4): unique keys ascending with run lengths. */
int oracle_sort_compact(const uint64_t *keys, uint64_t n, int words, oracle_result *res) {
    memset(res, 0, sizeof(*res));
    if (words == 1) {
        std::vector<uint64_t> v(keys, keys + n);
        std::vector<std::pair<uint64_t, uint64_t>> out;
        sort_and_compact<uint64_t>(v, out);
        res->n = out.size();
        res->words = 1;
        res->keys = (uint64_t *)malloc((out.size() + 1) * 8);
        res->counts = (uint64_t *)malloc((out.size() + 1) * 8);
        for (size_t i = 0; i < out.size(); i++) {
            res->keys[i] = out[i].first;
            res->counts[i] = out[i].second;
        }
    } else {
        std::vector<u128> v(n);
        for (uint64_t i = 0; i < n; i++) v[i] = ((u128)keys[2 * i] << 64) | keys[2 * i + 1];
        std::vector<std::pair<u128, uint64_t>> out;
        sort_and_compact<u128>(v, out);
        res->n = out.size();
        res->words = 2;
        res->keys = (uint64_t *)malloc((out.size() * 2 + 1) * 8);
        res->counts = (uint64_t *)malloc((out.size() + 1) * 8);
        for (size_t i = 0; i < out.size(); i++) {
            put_key<u128>(res->keys + 2 * i, out[i].first, 2);
            res->counts[i] = out[i].second;
        }
    }
    res->n_windows = n;
    return 0;
}

/*
 * Exact count of each query key (sorted ascending, unique; hi word first for
 * k > 32) over the whole library, by enumerating every window. Used to check
 * sampled outputs of libraries too large for a full oracle run.
 */
int oracle_count_queries(const uint8_t *bases, const uint64_t *off, uint64_t n_reads, int k, const uint64_t *queries,
                         uint64_t nq, int threads, uint64_t *counts) {
    if (check_args(off, n_reads, k)) return -1;
    if (threads < 1) threads = 1;
    std::vector<std::vector<uint64_t>> part(threads, std::vector<uint64_t>(nq, 0));
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; t++)
        pool.emplace_back([&, t]() {
            uint64_t r0 = n_reads * t / threads, r1 = n_reads * (t + 1) / threads;
            if (k <= 32) {
                std::vector<uint64_t> q(queries, queries + nq);
                for (uint64_t r = r0; r < r1; r++) {
                    uint64_t len = off[r + 1] - off[r];
                    for (uint64_t p = 0; p + k <= len; p++) {
                        uint64_t key;
                        if (!canonical_at<uint64_t>(bases + off[r] + p, k, &key)) continue;
                        auto it = std::lower_bound(q.begin(), q.end(), key);
                        if (it != q.end() && *it == key) part[t][it - q.begin()]++;
                    }
                }
            } else {
                std::vector<u128> q(nq);
                for (uint64_t i = 0; i < nq; i++) q[i] = ((u128)queries[2 * i] << 64) | queries[2 * i + 1];
                for (uint64_t r = r0; r < r1; r++) {
                    uint64_t len = off[r + 1] - off[r];
                    for (uint64_t p = 0; p + k <= len; p++) {
                        u128 key;
                        if (!canonical_at<u128>(bases + off[r] + p, k, &key)) continue;
                        auto it = std::lower_bound(q.begin(), q.end(), key);
                        if (it != q.end() && *it == key) part[t][it - q.begin()]++;
                    }
                }
            }
        });
    for (auto &th : pool) th.join();
    for (uint64_t i = 0; i < nq; i++) {
        uint64_t c = 0;
        for (int t = 0; t < threads; t++) c += part[t][i];
        counts[i] = c;
    }
    return 0;
}

/* ---------------------------------------------------------------- pattern-blocked Bloom filter
 * Sec. 2.1.3: a bit array initialised to zero; a hash of the item selects a
 * block, and a precomputed pattern of bit positions inside that block is tested
 * and then set. "Seen before" means every pattern bit was already one.
 *
 * Block geometry (a reading; the paper leaves b and the hash open): the block is
 * one 32-byte sector (four 64-bit words) selected by the top bits of the hash;
 * the pattern is a set of `pattern_bits` distinct positions inside one 64-bit
 * word of that sector. Hash fields: sector = h >> (64 - log2 n_sectors),
 * pattern index = h & (n_patterns - 1), word = (h >> 16) & 3.
 * Pattern j of the table: SplitMix64 seeded with `seed`, draws taken in order,
 * bit position = draw >> 58, repeated positions skipped, until the word has
 * pattern_bits distinct bits.
 */
typedef struct {
    uint64_t n_sectors;
    int sector_bits;
    int n_patterns;
    int pattern_bits;
    uint64_t *words;    /* 4 * n_sectors */
    uint64_t *patterns; /* n_patterns masks */
} oracle_pbbf;

oracle_pbbf *oracle_pbbf_new(uint64_t n_sectors, int pattern_bits, int n_patterns, uint64_t seed) {
    if (n_sectors == 0 || (n_sectors & (n_sectors - 1)) || n_patterns <= 0 || (n_patterns & (n_patterns - 1)) ||
        n_patterns > 65536 || pattern_bits < 1 || pattern_bits > 64)
        return NULL;
    oracle_pbbf *f = (oracle_pbbf *)calloc(1, sizeof(oracle_pbbf));
    f->n_sectors = n_sectors;
    f->sector_bits = 0;
    while ((1ull << f->sector_bits) < n_sectors) f->sector_bits++;
    f->n_patterns = n_patterns;
    f->pattern_bits = pattern_bits;
    f->words = (uint64_t *)calloc(n_sectors * 4, 8);
    f->patterns = (uint64_t *)calloc(n_patterns, 8);
    uint64_t state = seed;
    for (int j = 0; j < n_patterns; j++) {
        uint64_t m = 0;
        int have = 0;
        while (have < pattern_bits) {
            uint64_t bit = 1ull << (splitmix64_next(&state) >> 58);
            if (!(m & bit)) {
                m |= bit;
                have++;
            }
        }
        f->patterns[j] = m;
    }
    return f;
}

void oracle_pbbf_free(oracle_pbbf *f) {
    if (!f) return;
    free(f->words);
    free(f->patterns);
    free(f);
}

static inline uint64_t pbbf_hash(const uint64_t *key, int words) {
    return words == 1 ? fmix64(key[0]) : fmix64(key[1] ^ fmix64(key[0]));
}

/* Test-and-set of n keys in order; seen[i] = 1 iff every pattern bit of key i was already set. */
void oracle_pbbf_test_and_set(oracle_pbbf *f, const uint64_t *keys, uint64_t n, int words, uint8_t *seen) {
    for (uint64_t i = 0; i < n; i++) {
        uint64_t h = pbbf_hash(keys + i * words, words);
        uint64_t sector = f->sector_bits ? h >> (64 - f->sector_bits) : 0;
        uint64_t mask = f->patterns[h & (uint64_t)(f->n_patterns - 1)];
        uint64_t *w = &f->words[sector * 4 + ((h >> 16) & 3)];
        int all = 1;
        for (int b = 0; b < 64; b++)
            if (((mask >> b) & 1) && !((*w >> b) & 1)) all = 0;
        if (seen) seen[i] = (uint8_t)all;
        *w |= mask;
    }
}

/* Membership test only (nothing is set): seen[i] = 1 iff every pattern bit of key i is set. */
void oracle_pbbf_test(const oracle_pbbf *f, const uint64_t *keys, uint64_t n, int words, uint8_t *seen) {
    for (uint64_t i = 0; i < n; i++) {
        uint64_t h = pbbf_hash(keys + i * words, words);
        uint64_t sector = f->sector_bits ? h >> (64 - f->sector_bits) : 0;
        uint64_t mask = f->patterns[h & (uint64_t)(f->n_patterns - 1)];
        uint64_t w = f->words[sector * 4 + ((h >> 16) & 3)];
        seen[i] = (uint8_t)((w & mask) == mask);
    }
}

const uint64_t *oracle_pbbf_words(const oracle_pbbf *f) { return f->words; }
const uint64_t *oracle_pbbf_patterns(const oracle_pbbf *f) { return f->patterns; }


/* ---------------------------------------------------------------- cTurtle (Sec. 2.2)
 * A counting pattern-blocked Bloom filter in two stages, over the windows in read order.
 * Stage 1 is the filter above: the key's pattern in its block. A window whose stage-1
 * pattern was not complete sets it (a first sighting) and is done. Otherwise the key has
 * been seen: stage 2 looks at a second pattern in the adjacent block (the paper's
 * [h(x)+b, h(x)+2b]): if that pattern was not complete, it is set and the key is reported
 * as frequent; if it was, the key was reported before (or its stage-2 bits were all set by
 * other keys: a false negative). A singleton whose stage-1 bits were all set by other keys
 * is reported too (a false positive). No counts are kept.
 *
 * Stage-2 geometry (a reading): block = sector (s + 1) mod n_sectors after the stage-1
 * sector s; word = (h >> 18) & 3; pattern index = (h >> 20) & (n_patterns - 1), from the
 * same table.
 */
} /* extern "C" */

static inline void cturtle_addr(const oracle_pbbf *f, uint64_t h, uint64_t *w1, uint64_t *m1, uint64_t *w2,
                                uint64_t *m2) {
    const uint64_t pm = (uint64_t)(f->n_patterns - 1);
    const uint64_t s1 = f->sector_bits ? h >> (64 - f->sector_bits) : 0;
    const uint64_t s2 = (s1 + 1) & (f->n_sectors - 1);
    *w1 = s1 * 4 + ((h >> 16) & 3);
    *m1 = f->patterns[h & pm];
    *w2 = s2 * 4 + ((h >> 18) & 3);
    *m2 = f->patterns[(h >> 20) & pm];
}

template <class K>
static int cturtle_impl(const uint8_t *bases, const uint64_t *off, uint64_t n_reads, int k, oracle_pbbf *f,
                        oracle_result *res) {
    std::vector<K> keys;
    windows_of_reads<K>(bases, off, 0, n_reads, k, keys);
    const int words = sizeof(K) == 8 ? 1 : 2;
    std::vector<K> reported;
    for (size_t i = 0; i < keys.size(); i++) {
        uint64_t kw[2];
        put_key<K>(kw, keys[i], words);
        const uint64_t h = pbbf_hash(kw, words);
        uint64_t w1, m1, w2, m2;
        cturtle_addr(f, h, &w1, &m1, &w2, &m2);
        if ((f->words[w1] & m1) != m1) {  // first sighting
            f->words[w1] |= m1;
            continue;
        }
        if ((f->words[w2] & m2) != m2) {  // second sighting: report once
            f->words[w2] |= m2;
            reported.push_back(keys[i]);
        }
    }
    res->words = words;
    res->n = reported.size();
    res->n_windows = keys.size();
    res->keys = (uint64_t *)calloc(res->n * words + 1, 8);
    res->counts = (uint64_t *)calloc(res->n + 1, 8);
    for (size_t i = 0; i < reported.size(); i++) put_key<K>(res->keys + i * words, reported[i], words);
    return 0;
}

extern "C" {

/* Keys reported by the sequential two-stage filter, in report order (counts are left 0). */
int oracle_cturtle(const uint8_t *bases, const uint64_t *off, uint64_t n_reads, int k, uint64_t n_sectors,
                   int pattern_bits, int n_patterns, uint64_t seed, oracle_result *res) {
    memset(res, 0, sizeof(*res));
    if (check_args(off, n_reads, k)) return -1;
    oracle_pbbf *f = oracle_pbbf_new(n_sectors, pattern_bits, n_patterns, seed);
    if (!f) return -1;
    const int rc = k <= 32 ? cturtle_impl<uint64_t>(bases, off, n_reads, k, f, res)
                           : cturtle_impl<u128>(bases, off, n_reads, k, f, res);
    oracle_pbbf_free(f);
    return rc;
}

/*
 * For n distinct keys: free_out[i] = 1 iff key i's outcome cannot depend on the order of
 * the windows: its stage-1 pattern has a bit that no other key's stage-1 or stage-2
 * pattern sets, and its stage-2 pattern has a bit that no other key's patterns (nor its
 * own stage-1 pattern) set. Such a key is reported exactly when it occurs at least twice,
 * under any interleaving of test-and-set operations that are each atomic on one word.
 */
void oracle_cturtle_collision_free(const uint64_t *keys, uint64_t n, int words, uint64_t n_sectors, int pattern_bits,
                                   int n_patterns, uint64_t seed, uint8_t *free_out) {
    oracle_pbbf *f = oracle_pbbf_new(n_sectors, pattern_bits, n_patterns, seed);
    if (!f) return;
    std::vector<uint64_t> w1(n), m1(n), w2(n), m2(n);
    std::map<uint64_t, std::vector<std::pair<uint64_t, uint64_t>>> by_word;  // word -> (key index, mask)
    for (uint64_t i = 0; i < n; i++) {
        cturtle_addr(f, pbbf_hash(keys + i * words, words), &w1[i], &m1[i], &w2[i], &m2[i]);
        by_word[w1[i]].push_back(std::make_pair(i, m1[i]));
        by_word[w2[i]].push_back(std::make_pair(i, m2[i]));
    }
    for (uint64_t i = 0; i < n; i++) {
        uint64_t other1 = 0, other2 = 0;
        for (auto &e : by_word[w1[i]])
            if (e.first != i) other1 |= e.second;
        for (auto &e : by_word[w2[i]])
            if (e.first != i) other2 |= e.second;
        if (w2[i] == w1[i]) other2 |= m1[i];
        free_out[i] = (uint8_t)((m1[i] & ~other1) != 0 && (m2[i] & ~other2) != 0);
    }
    oracle_pbbf_free(f);
}

} /* extern "C" */
