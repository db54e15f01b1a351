// libturtle C ABI: contexts, device memory, stage orchestration, host <-> device copies.
//
// One call of turtle_count_device runs steps a1..a6 on one stream:
//   pack + valid -> W (window count)              [sync: sizes the filter and the key buffers]
//   pass 1 -> candidates + first sightings, with the bucket-index digit histograms
//                                                 [sync: their numbers]
//   bucketed form (default): two radix passes on the bucket index for each stream, bucket
//     bounds, the per-bucket kernel (merge, recount, threshold, sort), an output scan
//                                                 [sync: the output size] -> gather
//   global form: radix sort of the candidates, run-length compaction [sync], recount table,
//     first sightings (or pass 2), threshold -> result in key order
// Inputs larger than the device's budget run once per key range (super-partitions). Host
// calls copy the reads in chunks alongside pass 1 (run_count_overlapped), or stream them
// through staging buffers when they exceed a quarter of the free memory. Scratch comes from
// a per-context CUDA memory pool whose memory is retained between calls, so repeated calls do
// not return to the driver.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <initializer_list>
#include <chrono>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "turtle.h"
#include "turtle_testing.h"
#include "common.cuh"
#include "host.h"
#include "kernels.h"

using namespace turtle;

namespace {

constexpr uint64_t SPLITMIX_GAMMA = 0x9E3779B97F4A7C15ull;

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) drives the pattern table of Sec. 2.1.3:
// pattern j = `bits` distinct positions of a 64-bit word, position = draw >> 58,
// repeats skipped, draws taken in order from one stream seeded with `seed`.
void make_patterns(uint64_t seed, uint32_t bits, uint32_t n, std::vector<uint64_t> &out) {
    out.assign(n, 0);
    uint64_t x = seed;
    for (uint32_t j = 0; j < n; j++) {
        uint64_t m = 0;
        uint32_t have = 0;
        while (have < bits) {
            x += SPLITMIX_GAMMA;
            uint64_t z = x;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            const uint64_t bit = 1ull << (z >> 58);
            if (!(m & bit)) {
                m |= bit;
                have++;
            }
        }
        out[j] = m;
    }
}

uint64_t pow2_at_least(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}
int log2_exact(uint64_t p) {
    int b = 0;
    while ((1ull << b) < p) b++;
    return b;
}

// Device counters read back at the sync points.
enum { C_WINDOWS = 0, C_CAND, C_UNIQUE, C_OUT, C_FIRST, C_N };

}  // namespace

struct turtle_ctx {
    int device = 0;
    int sms = 1;
    cudaMemPool_t pool = nullptr;
    uint32_t *d_err = nullptr;
    unsigned long long *d_ctr = nullptr;  // C_N counters
    unsigned long long *h_ctr = nullptr;  // pinned mirror
    uint32_t *h_err = nullptr;
    uint64_t *h_hist = nullptr;  // pinned copy of the sort histograms (16 passes x 256 bins)
    // pattern table cache
    uint64_t *d_patterns = nullptr;
    uint64_t pat_seed = 0;
    uint32_t pat_bits = 0, pat_n = 0;
    // buffers of the current call (freed at its end) and of the last result (freed at the next call)
    std::vector<void *> scratch, result;
    cudaStream_t last_stream = nullptr;
    cudaEvent_t ev[2 * TURTLE_STAGE_COUNT] = {};
    turtle_stats stats{};
    uint64_t scratch_bytes = 0;
    // streamed input: a copy stream and the events that order it with the packing stream
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_h2d[2] = {}, ev_packed[2] = {};
    cudaEvent_t ev_in[2] = {};  // host-memory calls: first byte of the reads queued, last byte landed
    // host transfers, measured once per context: GB/s of a pageable copy, of page-locking (registering)
    // host memory, and of a copy from registered memory (0 = not measured yet)
    double gbs_pageable = 0, gbs_register = 0, gbs_registered = 0;
};

namespace {

struct Fail {
    int code;
};

// Failure injection (turtle_testing.h): armed by turtle_test_inject, each fires once.
struct Injection {
    std::atomic<int64_t> device_alloc{-1};  // allocations to let through before one fails (-1: off)
    std::atomic<int64_t> host_alloc{-1};
    std::atomic<uint32_t> lookback_spins{0};  // > 0: the next merge skips tile 0, waits run out after this many
    std::atomic<uint64_t> cand_cap{0};        // > 0: pass 1's candidate capacity for the next call
};
Injection g_inject;

// True when an armed countdown reaches its allocation (and disarms it).
bool inject_fires(std::atomic<int64_t> &left) {
    int64_t v = left.load();
    while (v >= 0) {
        if (left.compare_exchange_weak(v, v - 1)) return v == 0;
    }
    return false;
}

void ck(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) throw Fail{TURTLE_E_NOMEM};
    if (e != cudaSuccess) throw Fail{TURTLE_E_CUDA};
}

void *ctx_alloc(turtle_ctx *c, size_t bytes, cudaStream_t s, bool is_result = false) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (inject_fires(g_inject.device_alloc)) throw Fail{TURTLE_E_NOMEM};
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, c->pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Fail{TURTLE_E_NOMEM};
    }
    (is_result ? c->result : c->scratch).push_back(p);
    c->scratch_bytes += bytes;
    return p;
}

void free_list(std::vector<void *> &v, cudaStream_t s) {
    for (void *p : v) cudaFreeAsync(p, s);
    v.clear();
}

void ctx_begin(turtle_ctx *c, cudaStream_t s) {
    ck(cudaSetDevice(c->device));
    if (!c->result.empty()) free_list(c->result, c->last_stream ? c->last_stream : s);
    if (c->last_stream && c->last_stream != s) ck(cudaStreamSynchronize(c->last_stream));
    c->last_stream = s;
    c->scratch_bytes = 0;
    ck(cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), s));
    ck(cudaMemsetAsync(c->d_ctr, 0, sizeof(unsigned long long) * C_N, s));
}

// Free this call's scratch. The pool keeps freed memory for the next call: re-growing a pool maps
// physical memory again, which cost a large input hundreds of milliseconds per call when the pool
// was trimmed at the end of each call. The context's budget counts the pool's idle memory as free;
// turtle_ctx_trim (or turtle_ctx_destroy) gives it back to the device.
void ctx_end(turtle_ctx *c, cudaStream_t s) {
    free_list(c->scratch, s);
    cudaGetLastError();
}

// Copy the counters and the error word to the host (synchronises s).
void read_back(turtle_ctx *c, cudaStream_t s) {
    ck(cudaMemcpyAsync(c->h_ctr, c->d_ctr, sizeof(unsigned long long) * C_N, cudaMemcpyDeviceToHost, s));
    ck(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    const uint32_t e = *c->h_err;
    if (e & ERR_BAD_OFFSETS) throw Fail{TURTLE_E_ARG};
    if (e & ERR_COUNT_OVERFLOW) throw Fail{TURTLE_E_OVERFLOW};
    if (e & ERR_CAND_OVERFLOW) throw Fail{TURTLE_E_CAPACITY};  // an output larger than the room given to it
    if (e & ERR_PART_MISMATCH) throw Fail{TURTLE_E_DEVICE};    // a key-range test disagreed with the key
    if (e) throw Fail{TURTLE_E_DEVICE};
}

const uint64_t *ctx_patterns(turtle_ctx *c, const turtle_params &p, cudaStream_t s) {
    if (c->d_patterns && c->pat_seed == p.pattern_seed && c->pat_bits == p.pattern_bits && c->pat_n == p.n_patterns)
        return c->d_patterns;
    std::vector<uint64_t> h;
    make_patterns(p.pattern_seed, p.pattern_bits, p.n_patterns, h);
    if (c->d_patterns) {
        ck(cudaStreamSynchronize(s));
        cudaFree(c->d_patterns);
        c->d_patterns = nullptr;
    }
    ck(cudaMalloc(&c->d_patterns, sizeof(uint64_t) * p.n_patterns));
    ck(cudaMemcpyAsync(c->d_patterns, h.data(), sizeof(uint64_t) * p.n_patterns, cudaMemcpyHostToDevice, s));
    ck(cudaStreamSynchronize(s));
    c->pat_seed = p.pattern_seed;
    c->pat_bits = p.pattern_bits;
    c->pat_n = p.n_patterns;
    return c->d_patterns;
}

// Caller buffers that kernels read or write as 8- or 16-byte words must be aligned to that width: a
// 128-bit key is accessed as one 16-byte word, a 64-bit key or word as 8 bytes, a count as 4. A NULL
// pointer passes (the entry points check NULL separately).
bool aligned(const void *p, size_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

// params.sort_tile -> onesweep variant (keys per thread and CTAs per SM; 3 = persistent with bulk-copied
// tiles). Default: variant 0 for the global sort; for the bucket sort variant 1 with 64-bit keys (16 per
// thread, 4 CTAs/SM) and variant 0 with 128-bit keys (16 per thread, 2 CTAs/SM), both 4,096-key tiles:
// measured on long-k, 128-bit bucket sorts took 348 ms with it against 433 ms with 8 keys per thread.
int sort_variant(const turtle_params &p, bool bucket, int key_words) {
    switch (p.sort_tile) {
    case 0: return bucket && key_words == 1 ? 1 : 0;
    case 3: return 0;
    case 4: return 3;
    default: return (int)p.sort_tile;
    }
}

bool params_ok(const turtle_params &p) {
    return (p.l2_fetch_bytes == 0 || (p.l2_fetch_bytes >= 32 && p.l2_fetch_bytes <= 128)) && p.pattern_bits >= 1 &&
           p.pattern_bits <= 64 && p.n_patterns >= 1 && p.n_patterns <= 4096 &&
           (p.n_patterns & (p.n_patterns - 1)) == 0 && p.filter_bits_per_window > 0.f &&
           p.filter_bits_per_window <= 1024.f && p.sort_tile <= 4 && p.compact <= 3 && p.hash_slots_log2 <= 40 &&
           (p.bucket_slots == 0 || p.bucket_slots == 4096 || p.bucket_slots == 8192) &&
           p.shard_count <= TURTLE_PARTS && p.shard_index < (p.shard_count ? p.shard_count : 1) &&
           !(p.shard_count > 1 && p.compact == 3) && p.probe_order <= 1 &&
           (p.bucket_windows == 0 || (p.bucket_windows >= 1024 && p.bucket_windows <= (1u << 20))) &&
           p.host_transfer <= 2 && p.batch_mixed <= 2;
}

// Shard s of n takes the key-range parts [bounds[s], bounds[s+1]): bounds[s] is the first part at which
// the windows of the parts below it reach s/n of all windows.
void shard_bounds(const uint64_t *w, uint32_t n_parts, uint32_t n_shards, uint32_t *bounds) {
    unsigned __int128 total = 0;
    for (uint32_t p = 0; p < n_parts; p++) total += w[p];
    uint32_t p = 0;
    unsigned __int128 below = 0;  // windows of parts [0, p)
    bounds[0] = 0;
    for (uint32_t sh = 1; sh < n_shards; sh++) {
        while (p < n_parts && below * n_shards < total * sh) below += w[p++];
        bounds[sh] = p;
    }
    bounds[n_shards] = n_parts;
}

turtle_params resolve(const turtle_params *p) {
    turtle_params d;
    turtle_params_default(&d);
    if (!p) return d;
    turtle_params r = *p;
    if (r.struct_size != sizeof(turtle_params)) return d;
    return r;
}

struct Timer {
    turtle_ctx *c;
    cudaStream_t s;
    bool on;
    void start(int st) {
        if (on) ck(cudaEventRecord(c->ev[2 * st], s));
    }
    void stop(int st) {
        if (on) ck(cudaEventRecord(c->ev[2 * st + 1], s));
    }
};

// Reads already packed on the device (streamed input): P, B and S filled, S marked.
struct PrePacked {
    uint64_t *P, *B, *S;
};

// Batched form: positions [lib_starts[l], lib_starts[l+1]) are library l; keys carry l above their 2k bits.
// A mixed batch (libraries of different k, 128-bit keys) carries each library's k and puts the tag in the
// key's top bits; its libraries start on 128-position boundaries, so no pass-1 tile or validity word
// spans two libraries.
struct BatchTag {
    const uint64_t *lib_starts;  // device, n_libs + 1
    int n_libs;
    int tag_bits;
    unsigned long long *lib_windows;  // device, n_libs counters (zeroed by run_count)
    const int *lib_k = nullptr;       // mixed batch: device, each library's k
    int tag_shift = 0;                // mixed batch: bit of the tag (128 - tag_bits); else 2k
    const uint64_t *host_starts = nullptr;  // mixed batch: lib_starts on the host
    const int *host_k = nullptr;            // mixed batch: each library's k on the host
};

struct DeviceOut {
    void *keys = nullptr;
    uint32_t *counts = nullptr;
    uint64_t n = 0, n_windows = 0;
};

struct PartOut {
    void *keys;
    uint32_t *counts;
    uint64_t n;
};

// Bucketed sort-and-compact: stable radix sort of the candidates and of the first sightings by
// bucket index, bucket bounds, then per bucket merge + first-sighting recount + threshold + sort,
// then a dense gather (bucketed_part below).
constexpr uint64_t BUCKET_WINDOWS = 16384;  // candidates + first sightings per bucket, about (default)

uint64_t bucket_windows_of(const turtle_params &p) { return p.bucket_windows ? p.bucket_windows : BUCKET_WINDOWS; }

// Bucket-index bits actually used, given the bits wanted: 8 per sort pass, and up to three bits
// beyond a multiple of 8 are dropped rather than paid for with a whole extra pass (buckets up to
// eight times fuller; measured on the long-k library: 6.07 vs 5.64G k-mers/s).
int bucket_bits_for(int want) {
    if (want > 8 && want % 8 >= 1 && want % 8 <= 3) return want - want % 8;
    return want < 24 ? want : 24;
}

// Buckets for n_all windows of the key range [part_lo, part_hi) of 2^part_bits parts; *bits = index bits.
BucketGeom bucket_geom(uint64_t n_all, uint32_t part_lo, uint32_t part_hi, int part_bits, int k, int *bits,
                       uint64_t per_bucket = BUCKET_WINDOWS) {
    int b = 0;
    while (b < 24 && (n_all >> b) > per_bucket) b++;
    b = bucket_bits_for(b);
    BucketGeom bg{};
    bg.k = k;
    bg.f_lo = (uint64_t)part_lo << (62 - part_bits);
    const uint64_t span = (uint64_t)(part_hi - part_lo) << (62 - part_bits);
    bg.shift = 0;
    while (bg.shift < 62 && (span >> bg.shift) > ((uint64_t)1 << b)) bg.shift++;
    bg.n_buckets = (uint32_t)(((span - 1) >> bg.shift) + 1);  // <= 2^b
    *bits = b;
    return bg;
}

// Batch: library l gets 2^b[l] buckets for its lib_w[l] windows; the total is capped the same way
// (the largest libraries give up bits first). Returns the index bits of the total.
int batch_bucket_bits(const std::vector<unsigned long long> &lib_w, std::vector<int> &b,
                      uint64_t per_bucket = BUCKET_WINDOWS) {
    const size_t n = lib_w.size();
    b.assign(n, 0);
    uint64_t total = 0;
    for (size_t l = 0; l < n; l++) {
        while (b[l] < 20 && (lib_w[l] >> b[l]) > per_bucket) b[l]++;
        total += (uint64_t)1 << b[l];
    }
    int want = 0;
    while (((uint64_t)1 << want) < total) want++;
    const int bits = bucket_bits_for(want);
    while (total > ((uint64_t)1 << bits)) {
        size_t big = 0;
        for (size_t l = 1; l < n; l++)
            if (b[l] > b[big]) big = l;
        if (b[big] == 0) break;  // cannot happen: n libraries <= 2^bits
        total -= (uint64_t)1 << (b[big] - 1);
        b[big]--;
    }
    return bits;
}

// One key range: candidates cand[0, n_cand) and first sightings first_keys[0, n_first) (which may
// sit in the top of the same buffer), bucket geometry bg with `bits` index bits and pass 1's digit
// histograms in hist. Returns the range's output, ascending.
template <class K>
PartOut bucketed_part(turtle_ctx *c, const LaunchCfg &lc, Timer &tm, turtle_stats &st, uint32_t min_count,
                      K *cand, uint64_t n_cand, K *first_keys, uint64_t n_first, const BucketGeom &bg, int bits,
                      uint64_t *hist, bool result_buffers, int variant, bool large_table, cudaStream_t s,
                      K *alt_pre = nullptr) {
    constexpr int KW = sizeof(K) / 8;
    uint32_t *err = c->d_err;
    unsigned long long *ctr = c->d_ctr;
    const uint64_t n_all = n_cand + n_first;
    const uint32_t B = bg.n_buckets;
    unsigned long long *off_c = (unsigned long long *)ctx_alloc(c, 8 * ((uint64_t)B + 1), s);
    unsigned long long *off_f = (unsigned long long *)ctx_alloc(c, 8 * ((uint64_t)B + 1), s);
    unsigned long long *nrep = (unsigned long long *)ctx_alloc(c, 8 * (uint64_t)B, s);
    unsigned long long *out_off = (unsigned long long *)ctx_alloc(c, 8 * ((uint64_t)B + 1), s);
    uint32_t *ticket = (uint32_t *)ctx_alloc(c, 16, s);
    K *alt = alt_pre ? alt_pre : (K *)ctx_alloc(c, sizeof(K) * (n_all ? n_all : 1), s);  // room for n_all keys
    uint32_t *tmp_counts = (uint32_t *)ctx_alloc(c, 4 * (n_cand ? n_cand : 1), s);
    const int passes_all = (bits + 7) / 8;
    SortScratch ss{};
    ss.lookback_words = sort_lookback_words(n_cand > n_first ? n_cand : n_first, KW);
    ss.lookback = (uint64_t *)ctx_alloc(c, 8 * ss.lookback_words, s);
    ss.tile_ctr = (uint32_t *)ctx_alloc(c, 4 * 32, s);
    tm.start(TURTLE_STAGE_SORT);
    int passes = 0;
    ss.alt = alt;
    ss.hist = hist;  // digit histograms from pass 1: candidates, then first sightings
    K *sc = launch_bucket_sort<K>(lc, cand, n_cand, bg, bits, ss, err, &passes, true, variant);
    ss.alt = alt + n_cand;
    ss.hist = hist + 256 * passes_all;
    K *sf = n_first ? launch_bucket_sort<K>(lc, first_keys, n_first, bg, bits, ss, err, nullptr, true, variant)
                    : nullptr;
    launch_bucket_bounds<K>(lc, sc, n_cand, bg, off_c);
    if (sf) launch_bucket_bounds<K>(lc, sf, n_first, bg, off_f);
    tm.stop(TURTLE_STAGE_SORT);
    // per-bucket results go to whichever buffer holds neither sorted array
    K *tmp = sc == cand ? alt : cand;
    tm.start(TURTLE_STAGE_RLE);
    ck(cudaMemsetAsync(ticket, 0, 16, s));
    // each bucket's results land in tmp at the bucket's candidate offset (room for all its candidates)
    launch_bucket_count<K>(lc, sc, off_c, sf, off_f, B, min_count, tmp, tmp_counts, nrep, ticket, ctr + C_UNIQUE,
                           err, large_table ? 1 : 0);
    launch_scan_u64(lc, nrep, B, out_off);
    tm.stop(TURTLE_STAGE_RLE);
    ck(cudaMemcpyAsync(ctr + C_OUT, out_off + B, 8, cudaMemcpyDeviceToDevice, s));
    const int sorts = (n_cand > 1 && passes ? 1 : 0) + (n_first > 1 && passes ? 1 : 0);
    st.stage_launches[TURTLE_STAGE_SORT] += sorts * (passes + 1) + (sf ? 2 : 1);
    st.stage_launches[TURTLE_STAGE_RLE] += 2;
    st.sort_passes = (uint32_t)passes;
    read_back(c, s);
    const uint64_t n_out = c->h_ctr[C_OUT];
    st.n_unique += c->h_ctr[C_UNIQUE];
    K *okeys = (K *)ctx_alloc(c, sizeof(K) * (n_out ? n_out : 1), s, result_buffers);
    uint32_t *ocounts = (uint32_t *)ctx_alloc(c, 4 * (n_out ? n_out : 1), s, result_buffers);
    tm.start(TURTLE_STAGE_THRESHOLD);
    launch_bucket_gather<K>(lc, tmp, tmp_counts, off_c, out_off, B, okeys, ocounts);
    tm.stop(TURTLE_STAGE_THRESHOLD);
    st.stage_launches[TURTLE_STAGE_THRESHOLD] += 1;
    return PartOut{okeys, ocounts, n_out};
}

// HyperLogLog estimate of the number of distinct keys from 2^bits registers (Flajolet, Fusy,
// Gandouet & Meunier 2007), with linear counting when the raw estimate is small.
double hll_estimate(const uint32_t *regs, int bits) {
    const double m = (double)(1u << bits);
    double sum = 0.0;
    int zeros = 0;
    for (uint32_t j = 0; j < (1u << bits); j++) {
        sum += std::ldexp(1.0, -(int)regs[j]);
        zeros += regs[j] == 0;
    }
    const double e = 0.7213 / (1.0 + 1.079 / m) * m * m / sum;
    return (e <= 2.5 * m && zeros) ? m * std::log(m / zeros) : e;
}

void ctx_free(turtle_ctx *c, void *p, cudaStream_t s) {
    for (auto it = c->scratch.begin(); it != c->scratch.end(); ++it)
        if (*it == p) {
            c->scratch.erase(it);
            cudaFreeAsync(p, s);
            return;
        }
}

// Hash-table form of one key range (params.compact = 2): count the candidates in an
// open-addressing table, add the first sightings, extract the keys that reach min_count and sort
// them, then look their counts up. Returns the range's output, ascending.
template <class K>
PartOut hashed_part(turtle_ctx *c, const LaunchCfg &lc, Timer &tm, turtle_stats &st, uint32_t min_count,
                    const K *cand, uint64_t n_cand, const K *first_keys, uint64_t n_first, int key_bits,
                    bool check_overflow, bool result_buffers, const turtle_params &prm, cudaStream_t s) {
    constexpr int KW = sizeof(K) / 8;
    uint32_t *err = c->d_err;
    unsigned long long *ctr = c->d_ctr;
    const int S = hash_slots_per_line(KW);
    const int rbits = hash_sketch_bits();
    uint32_t *regs = (uint32_t *)ctx_alloc(c, 4u << rbits, s);
    uint32_t *full = (uint32_t *)ctx_alloc(c, 16, s);
    uint32_t *h_words = reinterpret_cast<uint32_t *>(c->h_hist);  // pinned, 32 KB
    tm.start(TURTLE_STAGE_TABLE);
    uint64_t lines = 1;
    if (prm.hash_slots_log2) {
        lines = std::max<uint64_t>(1, (1ull << prm.hash_slots_log2) / S);
    } else {
        ck(cudaMemsetAsync(regs, 0, 4u << rbits, s));
        launch_hash_sketch<K>(lc, cand, n_cand, regs);
        st.stage_launches[TURTLE_STAGE_TABLE] += n_cand ? 1 : 0;
        ck(cudaMemcpyAsync(h_words, regs, 4u << rbits, cudaMemcpyDeviceToHost, s));
        read_back(c, s);
        const double distinct = n_cand ? hll_estimate(h_words, rbits) : 0.0;
        // 10% above the estimate (eight standard errors of 2^12 registers), load at most 1/2
        lines = pow2_at_least((uint64_t)(1.1 * distinct / (0.5 * S)) + 1);
    }
    void *table = nullptr;
    for (;;) {
        table = ctx_alloc(c, 128 * lines, s);
        ck(cudaMemsetAsync(full, 0, 4, s));
        ck(cudaMemsetAsync(ctr + C_UNIQUE, 0, 8, s));
        launch_hash_clear<K>(lc, table, lines);
        launch_hash_insert<K>(lc, cand, n_cand, table, lines, check_overflow, ctr + C_UNIQUE, full, err);
        st.stage_launches[TURTLE_STAGE_TABLE] += n_cand ? 2 : 1;
        ck(cudaMemcpyAsync(h_words, full, 4, cudaMemcpyDeviceToHost, s));
        read_back(c, s);
        if (!h_words[0]) break;
        ctx_free(c, table, s);  // a key found no room: count again in a table twice as large
        lines *= 2;
    }
    tm.stop(TURTLE_STAGE_TABLE);
    st.table_bytes = std::max<uint64_t>(st.table_bytes, 128 * lines);
    const uint64_t nu = c->h_ctr[C_UNIQUE];
    st.n_unique += nu;
    tm.start(TURTLE_STAGE_RECOUNT);
    if (first_keys) launch_hash_firsts<K>(lc, first_keys, n_first, table, lines, check_overflow, err);
    tm.stop(TURTLE_STAGE_RECOUNT);
    st.stage_launches[TURTLE_STAGE_RECOUNT] += first_keys && n_first ? 1 : 0;
    K *kept = (K *)ctx_alloc(c, sizeof(K) * (nu ? nu : 1), s);
    K *alt = (K *)ctx_alloc(c, sizeof(K) * (nu ? nu : 1), s);
    ck(cudaMemsetAsync(ctr + C_OUT, 0, 8, s));
    tm.start(TURTLE_STAGE_THRESHOLD);
    launch_hash_extract<K>(lc, table, lines, min_count, kept, nu, ctr + C_OUT, err);
    tm.stop(TURTLE_STAGE_THRESHOLD);
    st.stage_launches[TURTLE_STAGE_THRESHOLD] += 1;
    read_back(c, s);
    const uint64_t n_out = c->h_ctr[C_OUT];
    SortScratch ss{};
    ss.alt = alt;
    ss.hist = (uint64_t *)ctx_alloc(c, 8 * 256 * 16, s);
    ss.lookback_words = sort_lookback_words(n_out, KW);
    ss.lookback = (uint64_t *)ctx_alloc(c, 8 * ss.lookback_words, s);
    ss.tile_ctr = (uint32_t *)ctx_alloc(c, 4 * 32, s);
    uint32_t *ocounts = (uint32_t *)ctx_alloc(c, 4 * (n_out ? n_out : 1), s, result_buffers);
    tm.start(TURTLE_STAGE_SORT);
    int passes = 0;
    K *sorted = launch_radix_sort<K>(lc, kept, n_out, key_bits, ss, err, false, 0, &passes,
                                     sort_variant(prm, false, (int)(sizeof(K) / 8)));
    launch_hash_lookup<K>(lc, sorted, n_out, table, lines, ocounts, err);
    tm.stop(TURTLE_STAGE_SORT);
    st.sort_passes = (uint32_t)passes;
    st.stage_launches[TURTLE_STAGE_SORT] += (n_out > 1 && passes ? passes + 2 : 0) + (n_out ? 1 : 0);
    if (result_buffers) {  // the sorted keys are part of the result
        for (auto it = c->scratch.begin(); it != c->scratch.end(); ++it)
            if (*it == (void *)sorted) {
                c->result.push_back(*it);
                c->scratch.erase(it);
                break;
            }
    }
    return PartOut{sorted, ocounts, n_out};
}

// Batch: one filter region per library, each sized for that library's windows (lib_w); the
// device table gives each library's first sector and hash shift. Returns the total sectors.
uint64_t lib_filter_regions(turtle_ctx *c, const std::vector<unsigned long long> &lib_w, float bits_per_window,
                            uint64_t **d_table, cudaStream_t s) {
    std::vector<uint64_t> lf(2 * lib_w.size());
    uint64_t at = 0;
    for (size_t l = 0; l < lib_w.size(); l++) {
        const uint64_t sec = pow2_at_least((uint64_t)(lib_w[l] * bits_per_window / 256.0) + 1);
        lf[2 * l] = at;
        lf[2 * l + 1] = (uint64_t)(64 - log2_exact(sec));
        at += sec;
    }
    *d_table = (uint64_t *)ctx_alloc(c, 8 * lf.size(), s);
    ck(cudaMemcpyAsync(*d_table, lf.data(), 8 * lf.size(), cudaMemcpyHostToDevice, s));
    return at;
}

// Batch: each library its own range of buckets, sized by its windows (lib_w); *bits = index bits.
BucketGeom lib_buckets(turtle_ctx *c, const std::vector<unsigned long long> &lib_w, int k, int *bits,
                       cudaStream_t s, uint64_t per_bucket = BUCKET_WINDOWS, const BatchTag *tag = nullptr) {
    std::vector<int> lb;
    *bits = batch_bucket_bits(lib_w, lb, per_bucket);
    std::vector<uint4> lg(lib_w.size());
    uint32_t at = 0;
    const bool mixed = tag && tag->lib_k;
    for (size_t l = 0; l < lib_w.size(); l++) {
        lg[l] = make_uint4(at, 1u << lb[l], (uint32_t)(62 - lb[l]), mixed ? (uint32_t)tag->host_k[l] : 0u);
        at += 1u << lb[l];
    }
    uint4 *d_lg = (uint4 *)ctx_alloc(c, sizeof(uint4) * lg.size(), s);
    ck(cudaMemcpyAsync(d_lg, lg.data(), sizeof(uint4) * lg.size(), cudaMemcpyHostToDevice, s));
    BucketGeom bg{};
    bg.k = k;
    bg.n_buckets = at;
    bg.tag_shift = mixed ? tag->tag_shift : 2 * k;
    bg.lib = d_lg;
    return bg;
}

// cTurtle (Sec. 2.2) on packed reads with W valid windows: the two-stage counting filter reports
// the keys seen (probably) at least twice, then they are sorted ascending. No counts.
constexpr uint32_t CTURTLE_BITS_DEFAULT = 8;
template <class K>
void run_cturtle(turtle_ctx *c, const LaunchCfg &lc, Timer &tm, turtle_stats &st, const PackLayout &L, int k,
                 const uint64_t *P, const uint64_t *V, uint64_t W, const turtle_params &prm, cudaStream_t s,
                 DeviceOut &out) {
    uint32_t *err = c->d_err;
    unsigned long long *ctr = c->d_ctr;
    const double bits = prm.cturtle_bits_per_window ? prm.cturtle_bits_per_window : CTURTLE_BITS_DEFAULT;
    FilterGeom fg{};
    fg.n_sectors = pow2_at_least((uint64_t)((double)W * bits / 256.0) + 1);
    if (fg.n_sectors < 2) fg.n_sectors = 2;
    fg.sector_shift = 64 - log2_exact(fg.n_sectors);
    fg.words = (uint64_t *)ctx_alloc(c, 32 * fg.n_sectors, s);
    ck(cudaMemsetAsync(fg.words, 0, 32 * fg.n_sectors, s));
    fg.patterns = ctx_patterns(c, prm, s);
    fg.pat_mask = prm.n_patterns - 1;
    st.filter_bytes = 32 * fg.n_sectors;
    // reported keys <= distinct keys <= W; room for all of them unless that exceeds 40% of free memory
    size_t free_b = 0, total_b = 0;
    ck(cudaMemGetInfo(&free_b, &total_b));
    uint64_t cap = W;
    if ((double)cap * sizeof(K) > 0.4 * (double)free_b) cap = (uint64_t)(0.4 * (double)free_b / sizeof(K));
    K *emit = (K *)ctx_alloc(c, sizeof(K) * (cap ? cap : 1), s);
    ck(cudaMemsetAsync(ctr + C_CAND, 0, 8, s));
    tm.start(TURTLE_STAGE_FILTER);
    launch_cturtle<K>(lc, L, k, P, V, fg, fg.n_sectors - 1, emit, ctr + C_CAND, cap, err);
    tm.stop(TURTLE_STAGE_FILTER);
    read_back(c, s);
    const uint64_t n = c->h_ctr[C_CAND];
    SortScratch ss{};
    ss.alt = ctx_alloc(c, sizeof(K) * (n ? n : 1), s);
    ss.hist = (uint64_t *)ctx_alloc(c, 8 * 256 * 16, s);
    ss.lookback_words = sort_lookback_words(n, sizeof(K) / 8);
    ss.lookback = (uint64_t *)ctx_alloc(c, 8 * ss.lookback_words, s);
    ss.tile_ctr = (uint32_t *)ctx_alloc(c, 4 * 32, s);
    int passes = 0;
    tm.start(TURTLE_STAGE_SORT);
    K *sorted = launch_radix_sort<K>(lc, emit, n, 2 * k, ss, err, false, 0, &passes, 0);
    tm.stop(TURTLE_STAGE_SORT);
    K *okeys = (K *)ctx_alloc(c, sizeof(K) * (n ? n : 1), s, true);
    if (n) ck(cudaMemcpyAsync(okeys, sorted, sizeof(K) * n, cudaMemcpyDeviceToDevice, s));
    read_back(c, s);
    st.stage_launches[TURTLE_STAGE_FILTER] = 1;
    st.stage_launches[TURTLE_STAGE_SORT] = n > 1 ? passes + 2 : 0;
    st.sort_passes = (uint32_t)passes;
    st.n_candidates = n;
    st.n_out = n;
    st.super_partitions = 1;
    out.keys = okeys;
    out.counts = nullptr;
    out.n = n;
    if (prm.timing) ck(cudaStreamSynchronize(s));  // the last stage's events may still be pending
    if (prm.timing)
        for (int i : {(int)TURTLE_STAGE_PACK, (int)TURTLE_STAGE_VALID, (int)TURTLE_STAGE_FILTER, (int)TURTLE_STAGE_SORT}) {
            float ms = 0.f;
            if ((i != TURTLE_STAGE_PACK || st.stage_launches[i]) &&
                cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]) == cudaSuccess)
                st.stage_ms[i] = ms;
            else cudaGetLastError();
        }
    for (int i = 0; i < TURTLE_STAGE_COUNT; i++) st.launches += st.stage_launches[i];
    st.scratch_bytes = c->scratch_bytes;
    c->stats = st;
}

// Free the context's scratch allocated after position `mark` of its list, except the buffers in `keep`.
void scratch_trim(turtle_ctx *c, size_t mark, std::initializer_list<const void *> keep, cudaStream_t s) {
    std::vector<void *> kept;
    for (size_t i = mark; i < c->scratch.size(); i++) {
        void *p = c->scratch[i];
        if (std::find(keep.begin(), keep.end(), (const void *)p) != keep.end()) kept.push_back(p);
        else cudaFreeAsync(p, s);
    }
    c->scratch.resize(mark);
    c->scratch.insert(c->scratch.end(), kept.begin(), kept.end());
}

// Free memory on the device for this call: cudaMemGetInfo plus what this context's pool holds unused.
double device_room(turtle_ctx *c) {
    size_t free_b = 0, total_b = 0;
    ck(cudaMemGetInfo(&free_b, &total_b));
    uint64_t pool_reserved = 0, pool_used = 0;
    if (cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrReservedMemCurrent, &pool_reserved) == cudaSuccess &&
        cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrUsedMemCurrent, &pool_used) == cudaSuccess &&
        pool_reserved > pool_used)
        free_b += pool_reserved - pool_used;
    cudaGetLastError();
    return (double)free_b;
}

// Lazy sort-and-compact phases (params.compact = 3; Sec. 2.1.4 and Alg. 1), the memory-capped form.
// The windows are taken in chunks of pass-1 tiles, in read order, through one filter shared by all
// chunks. A chunk's candidates are sorted and compacted on their own (bucketed form, every key kept
// with its run length) and merged in one linear pass into the running sorted array of distinct
// candidates: the compacted prefix is never sorted again. A key seen twice has at least one
// candidate (the filter has no false negatives), so the running array holds every key that can
// reach min_count >= 2; the exact count of each is then taken by the second pass, which re-extracts
// every window and counts it in a table of the running array's keys (the exact recount); the keys are
// kept in the array's order when count >= min_count. With min_count = 1 every window is a
// candidate and the merged run lengths are the counts.
template <class K>
void run_lazy(turtle_ctx *c, const LaunchCfg &lc, Timer &tm, turtle_stats &st, const PackLayout &L, int k,
              uint32_t min_count, const uint64_t *P, const uint64_t *V, uint64_t W, const turtle_params &prm,
              cudaStream_t s, DeviceOut &out) {
    constexpr int KW = sizeof(K) / 8;
    constexpr int PART_BITS = 6;
    uint32_t *err = c->d_err;
    unsigned long long *ctr = c->d_ctr;
    const bool use_filter = min_count >= 2;
    FilterGeom fg{};
    if (use_filter) {
        fg.n_sectors = pow2_at_least((uint64_t)((double)W * prm.filter_bits_per_window / 256.0) + 1);
        fg.sector_shift = 64 - log2_exact(fg.n_sectors);
        fg.words = (uint64_t *)ctx_alloc(c, 32 * fg.n_sectors, s);
        ck(cudaMemsetAsync(fg.words, 0, 32 * fg.n_sectors, s));
        fg.patterns = ctx_patterns(c, prm, s);
        fg.pat_mask = prm.n_patterns - 1;
        st.filter_bytes = 32 * fg.n_sectors;
    }
    // Chunk size: 60% of the budget for one chunk's working set (candidates, the bucket sort's second
    // buffer, per-candidate counts, the compacted chunk and its share of the merged array), the rest for
    // the running array (held twice during a merge).
    const double budget = prm.budget_mib ? (double)prm.budget_mib * (1 << 20) : 0.8 * device_room(c);
    const double per_pos = 4.0 * sizeof(K) + 12.0;
    const uint64_t all_tiles = (L.n_bases + 127) / 128;
    uint64_t tiles = (uint64_t)(0.6 * budget / per_pos / 128.0);
    if (tiles < 1) tiles = 1;
    if (tiles > all_tiles) tiles = all_tiles;
    const uint64_t cap = tiles * 128;  // windows of a chunk <= its positions
    K *cand = (K *)ctx_alloc(c, sizeof(K) * cap, s);
    uint64_t *hist = (uint64_t *)ctx_alloc(c, 8 * 256 * 16, s);
    K *R = nullptr;
    uint32_t *Rc = nullptr;
    uint64_t nR = 0;
    const int variant = sort_variant(prm, true, (int)(sizeof(K) / 8));
    for (uint64_t t0 = 0; t0 < all_tiles; t0 += tiles) {
        const uint64_t t1 = std::min(all_tiles, t0 + tiles);
        ck(cudaMemsetAsync(ctr + C_CAND, 0, 8 * (C_N - C_CAND), s));
        ck(cudaMemsetAsync(hist, 0, 8 * 256 * 16, s));
        int bits = 0;
        const BucketGeom bg = bucket_geom((t1 - t0) * 128, 0u, 1u << PART_BITS, PART_BITS, k, &bits,
                                          bucket_windows_of(prm));
        tm.start(TURTLE_STAGE_FILTER);
        launch_pass1<K>(lc, L, k, P, V, use_filter, fg, cand, ctr + C_CAND, cap, nullptr, ctr + C_FIRST, 0, hist,
                        (bits + 7) / 8, 0, 0u, 1u << PART_BITS, nullptr, 0, nullptr, err, &bg, t0, t1);
        tm.stop(TURTLE_STAGE_FILTER);
        st.stage_launches[TURTLE_STAGE_FILTER] += 1;
        read_back(c, s);
        const uint64_t n_cand = c->h_ctr[C_CAND];
        st.n_candidates += n_cand;
        st.chunks += 1;
        const size_t mark = c->scratch.size();
        const PartOut po = bucketed_part<K>(c, lc, tm, st, 1, cand, n_cand, nullptr, 0, bg, bits, hist, false,
                                            variant, prm.bucket_slots != 4096, s);
        if (!R) {  // the first chunk's compacted keys start the running array
            scratch_trim(c, mark, {po.keys, po.counts}, s);
            R = (K *)po.keys;
            Rc = po.counts;
            nR = po.n;
        } else if (po.n) {
            const uint64_t n = nR + po.n, mt = merge_tiles(n);
            K *Rn = (K *)ctx_alloc(c, sizeof(K) * n, s);
            uint32_t *Rnc = (uint32_t *)ctx_alloc(c, 4 * n, s);
            uint64_t *split = (uint64_t *)ctx_alloc(c, 8 * (mt + 1), s);
            uint64_t *lb = (uint64_t *)ctx_alloc(c, 8 * mt, s);
            uint32_t *tc = (uint32_t *)ctx_alloc(c, 16, s);
            tm.start(TURTLE_STAGE_MERGE);
            const uint32_t inj = g_inject.lookback_spins.exchange(0);
            launch_merge_counts<K>(lc, R, Rc, nR, (const K *)po.keys, po.counts, po.n, Rn, Rnc, ctr + C_UNIQUE, split,
                                   lb, tc, err, inj > 0, inj);
            tm.stop(TURTLE_STAGE_MERGE);
            st.stage_launches[TURTLE_STAGE_MERGE] += 2;
            read_back(c, s);
            scratch_trim(c, mark, {Rn, Rnc}, s);
            ctx_free(c, R, s);
            ctx_free(c, Rc, s);
            R = Rn;
            Rc = Rnc;
            nR = c->h_ctr[C_UNIQUE];
        } else {
            scratch_trim(c, mark, {}, s);
        }
        if (prm.timing) {  // accumulate this chunk's stage times (the events are reused per chunk)
            ck(cudaStreamSynchronize(s));
            for (int i = TURTLE_STAGE_FILTER; i < TURTLE_STAGE_COUNT; i++) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]) == cudaSuccess) st.stage_ms[i] += ms;
                else cudaGetLastError();
                ck(cudaEventRecord(c->ev[2 * i], s));
                ck(cudaEventRecord(c->ev[2 * i + 1], s));
            }
        }
    }
    ctx_free(c, cand, s);
    ctx_free(c, hist, s);
    if (use_filter) ctx_free(c, fg.words, s);
    st.n_unique = nR;
    K *okeys = (K *)ctx_alloc(c, sizeof(K) * (nR ? nR : 1), s, true);
    uint32_t *ocounts = (uint32_t *)ctx_alloc(c, 4 * (nR ? nR : 1), s, true);
    uint64_t n_out = 0;
    if (!use_filter) {  // every window was a candidate: the merged run lengths are the counts
        if (nR) {
            ck(cudaMemcpyAsync(okeys, R, sizeof(K) * nR, cudaMemcpyDeviceToDevice, s));
            ck(cudaMemcpyAsync(ocounts, Rc, 4 * nR, cudaMemcpyDeviceToDevice, s));
        }
        n_out = nR;
    } else if (nR) {
        ctx_free(c, Rc, s);  // candidate run lengths: the second pass counts every window itself
        Rc = nullptr;
        const uint64_t lines = pow2_at_least((uint64_t)(nR / (0.4 * slots_per_line(KW))) + 1);
        const TableGeom tg{lines - 1, nullptr, 0, 0};
        void *table = ctx_alloc(c, 128 * lines, s);
        st.table_bytes = 128 * lines;
        c->h_ctr[C_N - 1] = nR;  // the insert kernel reads the key count from device memory
        ck(cudaMemcpyAsync(ctr + C_UNIQUE, &c->h_ctr[C_N - 1], 8, cudaMemcpyHostToDevice, s));
        tm.start(TURTLE_STAGE_TABLE);
        launch_table_clear<K>(lc, table, lines);
        launch_table_insert<K>(lc, R, nullptr, ctr + C_UNIQUE, nR, table, tg, nullptr, 0, err);
        tm.stop(TURTLE_STAGE_TABLE);
        tm.start(TURTLE_STAGE_RECOUNT);
        launch_pass2<K>(lc, L, k, P, V, table, tg, W >= 0xfffffffeull, err);
        tm.stop(TURTLE_STAGE_RECOUNT);
        const uint64_t lw = sort_lookback_words(nR, KW);
        uint64_t *lookback = (uint64_t *)ctx_alloc(c, 8 * lw, s);
        uint32_t *tc = (uint32_t *)ctx_alloc(c, 16, s);
        tm.start(TURTLE_STAGE_THRESHOLD);
        launch_threshold<K>(lc, R, nR, table, tg, min_count, okeys, ocounts, ctr + C_OUT, lookback, tc, err);
        tm.stop(TURTLE_STAGE_THRESHOLD);
        st.stage_launches[TURTLE_STAGE_TABLE] += 1;
        st.stage_launches[TURTLE_STAGE_RECOUNT] += 1;
        st.stage_launches[TURTLE_STAGE_THRESHOLD] += 1;
        read_back(c, s);
        n_out = c->h_ctr[C_OUT];
        if (prm.timing) {
            ck(cudaStreamSynchronize(s));
            for (int i : {(int)TURTLE_STAGE_TABLE, (int)TURTLE_STAGE_RECOUNT, (int)TURTLE_STAGE_THRESHOLD}) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]) == cudaSuccess) st.stage_ms[i] += ms;
                else cudaGetLastError();
            }
        }
    }
    read_back(c, s);
    out.keys = okeys;
    out.counts = ocounts;
    out.n = n_out;
    st.n_out = n_out;
    st.super_partitions = 1;
    if (prm.timing)
        for (int i = 0; i < TURTLE_STAGE_FILTER; i++) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]) == cudaSuccess) st.stage_ms[i] = ms;
            else cudaGetLastError();
        }
    for (int i = 0; i < TURTLE_STAGE_COUNT; i++) st.launches += st.stage_launches[i];
    st.scratch_bytes = c->scratch_bytes;
    c->stats = st;
}

template <class K>
void run_count(turtle_ctx *c, const uint8_t *bases, uint64_t n_bases, const uint64_t *offsets, uint64_t n_reads,
               int k, uint32_t min_count, const turtle_params &prm, cudaStream_t s, DeviceOut &out,
               const PrePacked *pre = nullptr, const BatchTag *tag = nullptr, bool cturtle = false) {
    constexpr int KW = sizeof(K) / 8;
    const LaunchCfg lc{c->sms, s};
    turtle_stats st{};
    Timer tm{c, s, prm.timing != 0};
    uint32_t *err = c->d_err;
    unsigned long long *ctr = c->d_ctr;

    const PackLayout L = PackLayout::of(n_bases);
    uint64_t *P, *B, *S;
    if (pre) {
        P = pre->P;
        B = pre->B;
        S = pre->S;
    } else {
        P = (uint64_t *)ctx_alloc(c, 8 * L.p_words, s);
        B = (uint64_t *)ctx_alloc(c, 8 * L.b_words, s);
        S = (uint64_t *)ctx_alloc(c, 8 * L.b_words, s);
        ck(cudaMemsetAsync(S, 0, 8 * L.b_words, s));
    }
    uint64_t *V = (uint64_t *)ctx_alloc(c, 8 * L.v_words, s);
    ck(cudaMemsetAsync(V + (L.v_words - 2), 0, 16, s));

    if (!pre) {
        tm.start(TURTLE_STAGE_PACK);
        launch_pack(lc, bases, offsets, n_reads, L, P, B, S, err);
        tm.stop(TURTLE_STAGE_PACK);
        st.stage_launches[TURTLE_STAGE_PACK] = 2;
    }
    tm.start(TURTLE_STAGE_VALID);
    if (tag && tag->lib_k) {  // mixed batch: each library's windows with its own k, over its own words
        for (int l = 0; l < tag->n_libs; l++)
            launch_valid(lc, L, tag->host_k[l], B, S, V, ctr + C_WINDOWS, tag->host_starts[l] / 64,
                         (tag->host_starts[l + 1] + 63) / 64);
        st.stage_launches[TURTLE_STAGE_VALID] = (uint32_t)tag->n_libs;
    } else {
        launch_valid(lc, L, k, B, S, V, ctr + C_WINDOWS);
        st.stage_launches[TURTLE_STAGE_VALID] = 1;
    }
    tm.stop(TURTLE_STAGE_VALID);
    std::vector<unsigned long long> lib_w;
    if (tag) {
        ck(cudaMemsetAsync(tag->lib_windows, 0, 8 * tag->n_libs, s));
        launch_lib_windows(lc, L, V, tag->lib_starts, tag->n_libs, tag->lib_windows);
        lib_w.resize(tag->n_libs);
        ck(cudaMemcpyAsync(lib_w.data(), tag->lib_windows, 8 * tag->n_libs, cudaMemcpyDeviceToHost, s));
    }
    read_back(c, s);
    const uint64_t W = c->h_ctr[C_WINDOWS];
    st.n_windows = W;
    out.n_windows = W;
    if (W == 0) {
        out.keys = ctx_alloc(c, 16, s, true);
        out.counts = (uint32_t *)ctx_alloc(c, 16, s, true);
        out.n = 0;
        c->stats = st;
        return;
    }

    // the ambiguous-call and read-start bitmaps are only needed for the validity bitmap: give their
    // memory back before the key-range budget is taken
    ctx_free(c, B, s);
    ctx_free(c, S, s);
    if (cturtle) {
        run_cturtle<K>(c, lc, tm, st, L, k, P, V, W, prm, s, out);
        return;
    }
    if (prm.compact == 3 && !tag) {  // lazy sort-and-compact phases
        run_lazy<K>(c, lc, tm, st, L, k, min_count, P, V, W, prm, s, out);
        return;
    }
    const bool use_filter = min_count >= 2;
    const bool hashed = prm.compact == 2;
    // batches and the hash-table form recount from first sightings
    const bool firsts_mode = use_filter && (!prm.recount_windows || tag || hashed);
    const int key_bits = tag && tag->lib_k ? 128 : 2 * k + (tag ? tag->tag_bits : 0);
    const int passes = sort_passes_for(key_bits);
    const uint64_t *patterns = use_filter ? ctx_patterns(c, prm, s) : nullptr;

    // Super-partitions (key routing, Sec. 2.1.5): when the post-filter working set of all windows does
    // not fit in free device memory, split the key space into consecutive key ranges and run the rest
    // of the path once per range; outputs are appended in key order.
    // Working set per window of a range. Bucketed: candidates + first sightings share one buffer, the
    // bucket sort's second buffer, per-candidate result counts, filter, a share of the output.
    // Global: the same two buffers, run starts and lengths, recount table, filter.
    // the bucketed form of sort-and-compact; the window-recount mode uses the global form
    const bool bucketed = prm.compact == 0 && (firsts_mode || !use_filter);
    const double filter_bpw = use_filter ? prm.filter_bits_per_window / 8.0 : 0.0;
    // Hash table: the candidate buffer, a table of at most two slots per distinct key (taken as up to
    // half the windows) and the kept keys with their sort buffer.
    const double bytes_per_window = bucketed ? 2.0 * sizeof(K) + 8.0 + filter_bpw
                                    : hashed ? 2.0 * sizeof(K) + 2.0 * sizeof(K) + filter_bpw
                                             : 2.0 * sizeof(K) + 20.0 + filter_bpw;
    // free device memory, plus what this context's pool holds unused from earlier calls
    size_t free_b = 0, total_b = 0;
    ck(cudaMemGetInfo(&free_b, &total_b));
    uint64_t pool_reserved = 0, pool_used = 0;
    if (cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrReservedMemCurrent, &pool_reserved) == cudaSuccess &&
        cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrUsedMemCurrent, &pool_used) == cudaSuccess &&
        pool_reserved > pool_used)
        free_b += pool_reserved - pool_used;
    cudaGetLastError();
    const double budget = prm.budget_mib ? (double)prm.budget_mib * (1 << 20) : 0.8 * (double)free_b;
    constexpr int PART_BITS = 6;
    static_assert((1 << PART_BITS) == TURTLE_PARTS, "key-range parts");
    std::vector<std::pair<uint32_t, uint32_t>> groups;  // [part_lo, part_hi) of each super-partition
    std::vector<uint64_t> group_w;
    const bool sharded = !tag && prm.shard_count > 1;
    // this call's key range: the whole key space, or its shard's consecutive parts
    uint32_t range_lo = 0, range_hi = 1u << PART_BITS;
    uint64_t W_range = W;
    if (tag || (!sharded && (double)W * bytes_per_window <= budget)) {  // batches are sized by the caller
        groups.push_back({0u, 1u << PART_BITS});
        group_w.push_back(W);
    } else {
        unsigned long long *pc = (unsigned long long *)ctx_alloc(c, 8 << PART_BITS, s);
        ck(cudaMemsetAsync(pc, 0, 8 << PART_BITS, s));
        launch_part_count<K>(lc, L, k, P, V, PART_BITS, pc);
        st.stage_launches[TURTLE_STAGE_VALID] += 1;
        std::vector<unsigned long long> cnt(1 << PART_BITS);
        ck(cudaMemcpyAsync(cnt.data(), pc, 8 << PART_BITS, cudaMemcpyDeviceToHost, s));
        read_back(c, s);
        if (sharded) {  // every shard sees the same part counts, so all agree on the bounds
            std::vector<uint32_t> bounds(prm.shard_count + 1);
            std::vector<uint64_t> w64(cnt.begin(), cnt.end());
            shard_bounds(w64.data(), 1u << PART_BITS, prm.shard_count, bounds.data());
            range_lo = bounds[prm.shard_index];
            range_hi = bounds[prm.shard_index + 1];
            W_range = 0;
            for (uint32_t p = range_lo; p < range_hi; p++) W_range += cnt[p];
        }
        // balanced groups within the range: as many as the budget needs, each near the average size
        const double n_groups = std::max(1.0, std::ceil((double)W_range * bytes_per_window / budget));
        const double target = (double)W_range / n_groups;
        uint32_t lo = range_lo;
        uint64_t acc = 0;
        for (uint32_t p = range_lo; p < range_hi; p++) {
            const double next = (double)(acc + cnt[p]);
            if (p > lo && (next * bytes_per_window > budget || next > 1.02 * target)) {
                groups.push_back({lo, p});
                group_w.push_back(acc);
                lo = p;
                acc = 0;
            }
            acc += cnt[p];
        }
        if (range_hi > lo) {
            groups.push_back({lo, range_hi});
            group_w.push_back(acc);
        }
    }
    const bool parted = groups.size() > 1 || sharded;
    st.super_partitions = (uint32_t)groups.size();
    // With two to four key ranges, the first range's pass 1 also writes each window's range id (two bits
    // per position) and the other ranges' passes select their windows from those bits; with more, each
    // pass 1 tests every window. (The filter-blocked pass 1 tests every window itself.)
    const bool binned_mode = bucketed && !tag && use_filter && firsts_mode && prm.probe_order == 1;
    uint64_t *rid = nullptr;
    uint8_t *d_pg = nullptr;
    bool rid_written = false;
    if (groups.size() >= 2 && groups.size() <= 4 && use_filter && !binned_mode) {
        std::vector<uint8_t> pg(1u << PART_BITS, 0);
        for (size_t g = 0; g < groups.size(); g++)
            for (uint32_t p = groups[g].first; p < groups[g].second; p++) pg[p] = (uint8_t)g;
        d_pg = (uint8_t *)ctx_alloc(c, pg.size(), s);
        ck(cudaMemcpyAsync(d_pg, pg.data(), pg.size(), cudaMemcpyHostToDevice, s));
        rid = (uint64_t *)ctx_alloc(c, 8 * range_id_words(n_bases), s);
    }

    std::vector<PartOut> outs;
    for (size_t g = 0; g < groups.size(); g++) {
        const uint64_t Wg = group_w[g];
        if (Wg == 0) continue;
        const size_t mark = c->scratch.size();  // this super-partition's scratch is freed at its end
        ck(cudaMemsetAsync(ctr + C_CAND, 0, 8 * (C_N - C_CAND), s));
        // pass 1: candidates (and first sightings)
        FilterGeom fg{};
        uint64_t *lib_filter = nullptr;
        if (use_filter) {
            if (tag) {  // one region per library, each sized for that library's windows
                fg.n_sectors = lib_filter_regions(c, lib_w, prm.filter_bits_per_window, &lib_filter, s);
                fg.sector_shift = 64;
            } else {
                const double bits = (double)Wg * prm.filter_bits_per_window;
                fg.n_sectors = pow2_at_least((uint64_t)(bits / 256.0) + 1);
                fg.sector_shift = 64 - log2_exact(fg.n_sectors);
            }
            fg.words = (uint64_t *)ctx_alloc(c, 32 * fg.n_sectors, s);
            ck(cudaMemsetAsync(fg.words, 0, 32 * fg.n_sectors, s));
            fg.patterns = patterns;
            fg.pat_mask = prm.n_patterns - 1;
            st.filter_bytes = 32 * fg.n_sectors > st.filter_bytes ? 32 * fg.n_sectors : st.filter_bytes;
        }
        K *cand = (K *)ctx_alloc(c, sizeof(K) * Wg, s);
        K *firsts = firsts_mode ? cand : nullptr;  // first sightings fill the same buffer from the top
        uint64_t *hist = (uint64_t *)ctx_alloc(c, 8 * 256 * 16, s);
        int bucket_bits = 0;
        BucketGeom bg{};
        if (bucketed && tag) {  // batch: each library its own range of buckets, sized by its windows
            bg = lib_buckets(c, lib_w, k, &bucket_bits, s, bucket_windows_of(prm), tag);
        } else if (bucketed) {  // every window of the range becomes a candidate or a first sighting: Wg of them
            bg = bucket_geom(Wg, parted ? groups[g].first : 0u, parted ? groups[g].second : (1u << PART_BITS),
                             PART_BITS, k, &bucket_bits, bucket_windows_of(prm));
        }
        const int hist_passes = bucketed ? (bucket_bits + 7) / 8 : hashed ? 0 : passes;
        ck(cudaMemsetAsync(hist, 0, 8 * 256 * 16, s));
        tm.start(TURTLE_STAGE_FILTER);
        const uint64_t inj_cap = g_inject.cand_cap.exchange(0);  // failure injection: a smaller candidate room
        const uint64_t cand_cap = inj_cap && inj_cap < Wg ? inj_cap : Wg;
        // filter-blocked pass 1: the windows' keys are binned into what becomes the bucket sort's second
        // buffer (the bins are dead once probed), so it costs no memory
        const bool binned = binned_mode;
        K *bin_keys = nullptr;
        if (binned) {
            bin_keys = (K *)ctx_alloc(c, sizeof(K) * Wg, s);
            unsigned long long *bin_words = (unsigned long long *)ctx_alloc(c, 8 * pass1_bin_words(), s);
            launch_pass1_binned<K>(lc, L, k, P, V, fg, bin_keys, Wg, bin_words, cand, ctr + C_CAND, cand_cap, firsts,
                                   ctr + C_FIRST, Wg, hist, hist_passes, parted ? PART_BITS : 0, groups[g].first,
                                   groups[g].second, err, &bg);
            st.stage_launches[TURTLE_STAGE_FILTER] += 3;  // + the bin-offset scan, counted with the filter stage
        } else {
            // the first range to run writes the range ids that the later ones read
            const bool write_rid = rid && !rid_written;
            launch_pass1<K>(lc, L, k, P, V, use_filter, fg, cand, ctr + C_CAND, cand_cap, firsts, ctr + C_FIRST, Wg,
                            hist, hist_passes, parted ? PART_BITS : 0, groups[g].first, groups[g].second,
                            tag ? tag->lib_starts : nullptr, tag ? tag->n_libs : 0, lib_filter, err,
                            bucketed ? &bg : nullptr, 0, ~0ull, write_rid ? nullptr : rid, (uint32_t)g,
                            tag ? tag->lib_k : nullptr, tag ? tag->tag_shift : 0, write_rid ? rid : nullptr,
                            write_rid ? d_pg : nullptr);
            rid_written |= write_rid;
        }
        tm.stop(TURTLE_STAGE_FILTER);
        st.stage_launches[TURTLE_STAGE_FILTER] += 1;
        if (!bucketed && !hashed) ck(cudaMemcpyAsync(c->h_hist, hist, 8 * 256 * passes, cudaMemcpyDeviceToHost, s));
        read_back(c, s);
        const uint64_t n_cand = c->h_ctr[C_CAND];
        const uint64_t n_first = c->h_ctr[C_FIRST];
        const K *first_keys = firsts_mode ? cand + (Wg - n_first) : nullptr;
        st.n_candidates += n_cand;
        st.n_firsts += n_first;

        PartOut po{};
        if (bucketed) {
            po = bucketed_part<K>(c, lc, tm, st, min_count, cand, n_cand, const_cast<K *>(first_keys), n_first, bg,
                                  bucket_bits, hist, !parted,
                                  sort_variant(prm, true, (int)(sizeof(K) / 8)),
                                  prm.bucket_slots != 4096, s, bin_keys);
        } else if (hashed) {
            po = hashed_part<K>(c, lc, tm, st, min_count, cand, n_cand, first_keys, n_first, key_bits,
                                W >= 0xfffffffeull, !parted, prm, s);
        } else {
        // a4: sort + compact
        SortScratch ss{};
        ss.alt = ctx_alloc(c, sizeof(K) * (n_cand ? n_cand : 1), s);
        ss.hist = hist;
        uint32_t skip = 0;  // digit passes where every candidate has the same digit
        for (int p = 0; p < passes; p++)
            for (int d = 0; d < 256; d++)
                if (c->h_hist[p * 256 + d] == n_cand) skip |= 1u << p;
        ss.lookback_words = sort_lookback_words(n_cand, KW);
        ss.lookback = (uint64_t *)ctx_alloc(c, 8 * ss.lookback_words, s);
        ss.tile_ctr = (uint32_t *)ctx_alloc(c, 4 * 32, s);
        tm.start(TURTLE_STAGE_SORT);
        int passes_run = 0;
        K *sorted = launch_radix_sort<K>(lc, cand, n_cand, key_bits, ss, err, true, skip, &passes_run,
                                         sort_variant(prm, false, (int)(sizeof(K) / 8)));
        tm.stop(TURTLE_STAGE_SORT);
        st.sort_passes = (uint32_t)passes_run;
        st.stage_launches[TURTLE_STAGE_SORT] += n_cand > 1 ? passes_run + 1 : 0;
        K *unique = sorted == cand ? (K *)ss.alt : cand;
        uint64_t *starts = nullptr;
        if (!use_filter || firsts_mode) starts = (uint64_t *)ctx_alloc(c, 8 * (n_cand ? n_cand : 1), s);
        tm.start(TURTLE_STAGE_RLE);
        launch_rle<K>(lc, sorted, n_cand, unique, starts, ctr + C_UNIQUE, ss.lookback, ss.tile_ctr + 20, err);
        tm.stop(TURTLE_STAGE_RLE);
        st.stage_launches[TURTLE_STAGE_RLE] += n_cand ? 1 : 0;

        if (!use_filter) {
            // every window is a candidate: run lengths are the exact counts (min_count == 1)
            uint32_t *counts = (uint32_t *)ctx_alloc(c, 4 * (n_cand ? n_cand : 1), s, !parted);
            tm.start(TURTLE_STAGE_THRESHOLD);
            launch_run_counts(lc, starts, ctr + C_UNIQUE, n_cand, n_cand, counts, err);
            tm.stop(TURTLE_STAGE_THRESHOLD);
            st.stage_launches[TURTLE_STAGE_THRESHOLD] += 1;
            read_back(c, s);
            const uint64_t nu = c->h_ctr[C_UNIQUE];
            if (!parted) {  // keep the buffer holding the unique keys alive as part of the result
                for (auto it = c->scratch.begin(); it != c->scratch.end(); ++it)
                    if (*it == (void *)unique) {
                        c->result.push_back(*it);
                        c->scratch.erase(it);
                        break;
                    }
            }
            po = PartOut{unique, counts, nu};
            st.n_unique += nu;
        } else {
            uint32_t *run = nullptr;  // run lengths of the sorted candidates (first-sighting recount only)
            if (firsts_mode) {
                run = (uint32_t *)ctx_alloc(c, 4 * (n_cand ? n_cand : 1), s);
                launch_run_counts(lc, starts, ctr + C_UNIQUE, n_cand, n_cand, run, err);
                st.stage_launches[TURTLE_STAGE_RLE] += 1;
            }
            read_back(c, s);
            const uint64_t nu = c->h_ctr[C_UNIQUE];
            st.n_unique += nu;
            // load factor <= 0.4: a line overflows into the next one rarely
            uint64_t lines = pow2_at_least((uint64_t)(nu / (0.4 * slots_per_line(KW))) + 1);
            TableGeom tg{lines - 1, nullptr, 0, 0};
            if (tag) {  // one region per library (distinct candidates per library from the sorted tags)
                std::vector<uint64_t> us(tag->n_libs + 1, ~0ull), lr(2 * tag->n_libs);
                uint64_t *d_us = (uint64_t *)ctx_alloc(c, 8 * tag->n_libs, s);
                ck(cudaMemsetAsync(d_us, 0xff, 8 * tag->n_libs, s));
                launch_tag_starts<K>(lc, unique, nu, key_bits - tag->tag_bits, d_us);
                ck(cudaMemcpyAsync(us.data(), d_us, 8 * tag->n_libs, cudaMemcpyDeviceToHost, s));
                read_back(c, s);
                us[tag->n_libs] = nu;
                for (int l = tag->n_libs - 1; l >= 0; l--)
                    if (us[l] == ~0ull) us[l] = us[l + 1];
                lines = 0;
                for (int l = 0; l < tag->n_libs; l++) {
                    const uint64_t nl = pow2_at_least((uint64_t)((us[l + 1] - us[l]) / (0.4 * slots_per_line(KW))) + 1);
                    lr[2 * l] = lines;
                    lr[2 * l + 1] = nl - 1;
                    lines += nl;
                }
                uint64_t *d_lr = (uint64_t *)ctx_alloc(c, 8 * lr.size(), s);
                ck(cudaMemcpyAsync(d_lr, lr.data(), 8 * lr.size(), cudaMemcpyHostToDevice, s));
                tg = TableGeom{0, d_lr, key_bits - tag->tag_bits, tag->n_libs};
            }
            void *table = ctx_alloc(c, 128 * lines, s);
            st.table_bytes = 128 * lines > st.table_bytes ? 128 * lines : st.table_bytes;
            uint64_t member_words = 0;
            uint64_t *member = nullptr;
            if (firsts_mode && prm.member_filter) {  // ~4.5 bits per candidate key: L2-resident
                member_words = pow2_at_least(nu / 16 + 1);
                member = (uint64_t *)ctx_alloc(c, 8 * member_words, s);
                ck(cudaMemsetAsync(member, 0, 8 * member_words, s));
            }
            tm.start(TURTLE_STAGE_TABLE);
            launch_table_clear<K>(lc, table, lines);
            launch_table_insert<K>(lc, unique, run, ctr + C_UNIQUE, nu, table, tg, member, member_words, err);
            tm.stop(TURTLE_STAGE_TABLE);
            st.stage_launches[TURTLE_STAGE_TABLE] += 1;
            tm.start(TURTLE_STAGE_RECOUNT);
            if (firsts_mode)
                launch_add_firsts<K>(lc, first_keys, n_first, table, tg, member, member_words, W >= 0xfffffffeull,
                                     err);
            else
                launch_pass2<K>(lc, L, k, P, V, table, tg, W >= 0xfffffffeull, err);
            tm.stop(TURTLE_STAGE_RECOUNT);
            st.stage_launches[TURTLE_STAGE_RECOUNT] += (!firsts_mode || n_first) ? 1 : 0;
            K *okeys = (K *)ctx_alloc(c, sizeof(K) * (nu ? nu : 1), s, !parted);
            uint32_t *ocounts = (uint32_t *)ctx_alloc(c, 4 * (nu ? nu : 1), s, !parted);
            tm.start(TURTLE_STAGE_THRESHOLD);
            launch_threshold<K>(lc, unique, nu, table, tg, min_count, okeys, ocounts, ctr + C_OUT, ss.lookback,
                                ss.tile_ctr + 21, err);
            tm.stop(TURTLE_STAGE_THRESHOLD);
            st.stage_launches[TURTLE_STAGE_THRESHOLD] += nu ? 1 : 0;
            read_back(c, s);
            po = PartOut{okeys, ocounts, c->h_ctr[C_OUT]};
        }
        }  // global form
        if (prm.timing) {  // accumulate this super-partition's stage times (events are reused per part)
            ck(cudaStreamSynchronize(s));  // the last stage's events may still be pending
            for (int i = TURTLE_STAGE_FILTER; i < TURTLE_STAGE_COUNT; i++) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]) == cudaSuccess) st.stage_ms[i] += ms;
                else cudaGetLastError();
                ck(cudaEventRecord(c->ev[2 * i], s));  // an empty interval unless the stage runs again
                ck(cudaEventRecord(c->ev[2 * i + 1], s));
            }
        }
        if (parted) {
            // keep only this part's output: move it out of the part's scratch range
            for (void *keep : {po.keys, (void *)po.counts})
                for (size_t i = mark; i < c->scratch.size(); i++)
                    if (c->scratch[i] == keep) {
                        c->scratch.erase(c->scratch.begin() + i);
                        break;
                    }
            for (size_t i = mark; i < c->scratch.size(); i++) cudaFreeAsync(c->scratch[i], s);
            c->scratch.resize(mark);
            c->scratch.push_back(po.keys);
            c->scratch.push_back(po.counts);
        }
        outs.push_back(po);
    }
    if (!parted) {
        out.keys = outs.empty() ? ctx_alloc(c, 16, s, true) : outs[0].keys;
        out.counts = outs.empty() ? (uint32_t *)ctx_alloc(c, 16, s, true) : outs[0].counts;
        out.n = outs.empty() ? 0 : outs[0].n;
    } else {
        uint64_t total = 0;
        for (auto &o : outs) total += o.n;
        K *okeys = (K *)ctx_alloc(c, sizeof(K) * (total ? total : 1), s, true);
        uint32_t *ocounts = (uint32_t *)ctx_alloc(c, 4 * (total ? total : 1), s, true);
        uint64_t at = 0;
        for (auto &o : outs) {
            if (o.n) {
                ck(cudaMemcpyAsync(okeys + at, o.keys, sizeof(K) * o.n, cudaMemcpyDeviceToDevice, s));
                ck(cudaMemcpyAsync(ocounts + at, o.counts, 4 * o.n, cudaMemcpyDeviceToDevice, s));
            }
            at += o.n;
        }
        out.keys = okeys;
        out.counts = ocounts;
        out.n = total;
    }
    st.n_out = out.n;
    if (prm.timing) {
        for (int i = 0; i < TURTLE_STAGE_FILTER; i++) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]) == cudaSuccess) st.stage_ms[i] = ms;
            else cudaGetLastError();
        }
    }
    for (int i = 0; i < TURTLE_STAGE_COUNT; i++) st.launches += st.stage_launches[i];
    st.scratch_bytes = c->scratch_bytes;
    c->stats = st;
}

int fail_code(cudaStream_t s, turtle_ctx *c, int code) {
    // leave the context usable: drop this call's buffers
    cudaGetLastError();
    if (c) {
        free_list(c->scratch, s);
        free_list(c->result, s);
        cudaStreamSynchronize(s);
        cudaGetLastError();
    }
    return code;
}

// Scoped L2 fetch-granularity hint: random 8- to 16-byte probes need one 32-byte sector,
// and a larger fetch on every miss multiplies their DRAM traffic.
struct L2Fetch {
    size_t old = 0;
    bool set = false;
    explicit L2Fetch(uint32_t bytes) {
        if (!bytes) return;
        if (cudaDeviceGetLimit(&old, cudaLimitMaxL2FetchGranularity) == cudaSuccess &&
            cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, bytes) == cudaSuccess)
            set = true;
        cudaGetLastError();
    }
    ~L2Fetch() {
        if (set) cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, old);
        cudaGetLastError();
    }
};

int count_device_impl(turtle_ctx *c, const uint8_t *bases, uint64_t n_bases, const uint64_t *offsets,
                      uint64_t n_reads, int k, uint32_t min_count, const turtle_params *params, cudaStream_t s,
                      DeviceOut &o, bool cturtle = false) {
    if (!c || k < 1 || k > 64 || min_count < 1 || !offsets || (n_bases && !bases)) return TURTLE_E_ARG;
    if (!aligned(offsets, 8)) return TURTLE_E_ARG;
    const turtle_params prm = resolve(params);
    if (!params_ok(prm)) return TURTLE_E_ARG;
    try {
        ctx_begin(c, s);
        L2Fetch l2(prm.l2_fetch_bytes);
        if (k <= 32) run_count<uint64_t>(c, bases, n_bases, offsets, n_reads, k, min_count, prm, s, o, nullptr, nullptr,
                                         cturtle);
        else run_count<Key128>(c, bases, n_bases, offsets, n_reads, k, min_count, prm, s, o, nullptr, nullptr, cturtle);
        ctx_end(c, s);
        return TURTLE_OK;
    } catch (Fail f) {
        return fail_code(s, c, f.code);
    } catch (std::bad_alloc &) {
        return fail_code(s, c, TURTLE_E_NOMEM);
    }
}

// Host <-> device copies go straight from and to the caller's memory: on a Grace-based GPU the copy
// engines reach pageable memory through the CPU's page tables, on most boxes at about the rate of
// page-locked memory (~200 GB/s over NVLink-C2C), faster than staging through a page-locked buffer
// with host copies; where they do not, the memory is page-locked for the copy (HostLocks below).
// Host pages that do not exist yet are the exception: the copy engine would fault each one in, an
// order of magnitude slower, so a result buffer is first touched page by page from several threads.

void first_touch(void *p, size_t bytes) {
    const size_t page = (size_t)sysconf(_SC_PAGESIZE);
    const size_t pages = (bytes + page - 1) / page;
    const unsigned hw = std::thread::hardware_concurrency();
    // half the host's threads at most: the executor and the caller's threads keep running meanwhile
    const int T = bytes < ((size_t)4 << 20) ? 1 : (int)std::max(1u, std::min(8u, hw / 2));
    auto touch = [=](size_t a, size_t b) {
        for (size_t i = a; i < b; i++) static_cast<volatile char *>(p)[i * page] = 0;
    };
    if (T == 1) {
        touch(0, pages);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < T; t++) th.emplace_back(touch, pages * t / T, pages * (t + 1) / T);
    for (auto &x : th) x.join();
}

// Result buffers (host) are recycled: turtle_result_free keeps recent ones, up to 8 GiB in all,
// and the next result of a similar size reuses one whose pages already exist, so the device
// writes it at full speed without the first touch.
std::mutex g_rbuf_mu;
std::map<void *, size_t> g_rbuf_live;       // buffers handed out in results: pointer -> capacity
std::multimap<size_t, void *> g_rbuf_idle;  // recycled: capacity -> pointer
size_t g_rbuf_idle_bytes = 0;
constexpr size_t RBUF_IDLE_MAX = (size_t)8 << 30;
constexpr size_t RBUF_MIN = (size_t)1 << 20;  // smaller buffers are not worth keeping

// *fresh: the buffer's pages may not exist yet.
void *result_alloc(size_t bytes, bool *fresh) {
    if (inject_fires(g_inject.host_alloc)) return nullptr;
    {
        std::lock_guard<std::mutex> g(g_rbuf_mu);
        auto it = g_rbuf_idle.lower_bound(bytes);
        if (it != g_rbuf_idle.end() && it->first <= 2 * bytes + RBUF_MIN) {
            void *p = it->second;
            const size_t cap = it->first;
            g_rbuf_idle.erase(it);
            g_rbuf_idle_bytes -= cap;
            g_rbuf_live[p] = cap;
            *fresh = false;
            return p;
        }
    }
    void *p = malloc(bytes ? bytes : 1);
    if (!p) return nullptr;
    std::lock_guard<std::mutex> g(g_rbuf_mu);
    g_rbuf_live[p] = bytes;
    *fresh = true;
    return p;
}

void result_release(void *p) {
    if (!p) return;
    std::lock_guard<std::mutex> g(g_rbuf_mu);
    auto it = g_rbuf_live.find(p);
    if (it == g_rbuf_live.end()) {  // not one of ours
        free(p);
        return;
    }
    const size_t cap = it->second;
    g_rbuf_live.erase(it);
    if (cap < RBUF_MIN || cap > RBUF_IDLE_MAX) {
        free(p);
        return;
    }
    g_rbuf_idle.emplace(cap, p);
    g_rbuf_idle_bytes += cap;
    while (g_rbuf_idle_bytes > RBUF_IDLE_MAX) {  // give back the smallest first
        auto s = g_rbuf_idle.begin();
        g_rbuf_idle_bytes -= s->first;
        free(s->second);
        g_rbuf_idle.erase(s);
    }
}

// Host transfers on Grace: the copy engines reach pageable memory through the CPU's page tables. For
// large arrays the rate of such copies varies from run to run and box to box (8 to 190 GB/s measured,
// even on a box where a fresh 64 MiB buffer copies at 180 GB/s), while copies from page-locked memory
// run at 170-210 GB/s and page-locking (cudaHostRegister) costs 2-3 ms per GB. So the host form
// page-locks its large host arrays for their copies whenever locking is cheap; each context measures
// the rates once on 64 MiB (reported in its statistics).
constexpr double LOCK_MIN_GBS = 100.0;  // page-locking at least this fast: lock large arrays for copies
void calibrate_transfers(turtle_ctx *c, cudaStream_t s) {
    if (c->gbs_pageable > 0) return;
    const size_t n = (size_t)64 << 20;
    std::vector<unsigned char> host(n, 1);  // touched pageable memory
    void *dev = nullptr;
    c->gbs_pageable = 200.0;  // if anything below fails: assume the common fast case
    c->gbs_register = c->gbs_registered = 0.0;
    if (cudaMallocFromPoolAsync(&dev, n, c->pool, s) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    using clk = std::chrono::steady_clock;
    auto secs = [](clk::time_point t) { return std::chrono::duration<double>(clk::now() - t).count(); };
    auto copy_gbs = [&]() {
        double best = 1e30;
        for (int r = 0; r < 2; r++) {
            const clk::time_point t0 = clk::now();
            if (cudaMemcpyAsync(dev, host.data(), n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return 0.0;
            best = std::min(best, secs(t0));
        }
        return n / best / 1e9;
    };
    const double p = copy_gbs();
    if (p > 0) c->gbs_pageable = p;
    const clk::time_point t0 = clk::now();
    if (cudaHostRegister(host.data(), n, cudaHostRegisterDefault) == cudaSuccess) {
        c->gbs_register = n / std::max(secs(t0), 1e-9) / 1e9;
        c->gbs_registered = copy_gbs();
        cudaHostUnregister(host.data());
    }
    cudaFreeAsync(dev, s);
    cudaStreamSynchronize(s);
    cudaGetLastError();
}

// Page-locked parts of a call's host arrays. Only the whole pages inside an array are locked: a page at
// either end may be shared with another allocation (another array of the call, or memory of the caller's
// that is locked already), and locking it twice, or copying a range that starts inside one locked range
// and runs past its end, is an error. Copies therefore go through copy(), which splits them at the locked
// ranges' bounds so that every piece lies wholly inside or wholly outside one locked range. The
// destructor unlocks everything this object locked.
class HostLocks {
public:
    HostLocks(turtle_ctx *c, uint32_t mode) : c_(c), mode_(mode) {}
    HostLocks(const HostLocks &) = delete;
    HostLocks &operator=(const HostLocks &) = delete;
    ~HostLocks() {
        for (auto &r : ranges_) cudaHostUnregister((void *)r.first);
        cudaGetLastError();
    }
    // Lock [p, p + bytes) (its whole pages) when locking is cheap on this machine (mode 0: the context
    // measured page-locking at LOCK_MIN_GBS or more), always (mode 1) or never (mode 2). Arrays below
    // 16 MiB are copied as they are.
    void add(const void *p, size_t bytes) {
        if (!p || bytes < ((size_t)16 << 20) || mode_ == 2) return;
        if (mode_ == 0 && !(c_->gbs_register >= LOCK_MIN_GBS && c_->gbs_registered > 0)) return;
        const uintptr_t page = (uintptr_t)sysconf(_SC_PAGESIZE);
        const uintptr_t a = ((uintptr_t)p + page - 1) & ~(page - 1);
        const uintptr_t e = ((uintptr_t)p + bytes) & ~(page - 1);
        if (e <= a) return;
        for (auto &r : ranges_)
            if (a < r.second && r.first < e) return;  // cannot happen for distinct arrays; keep ranges disjoint
        if (cudaHostRegister((void *)a, e - a, cudaHostRegisterDefault) != cudaSuccess) {
            cudaGetLastError();  // e.g. the caller locked it already: copied as it is
            return;
        }
        ranges_.insert(std::upper_bound(ranges_.begin(), ranges_.end(), std::make_pair(a, e)), std::make_pair(a, e));
    }
    bool locked(const void *p) const {
        for (auto &r : ranges_)
            if ((uintptr_t)p >= r.first && (uintptr_t)p < r.second) return true;
        return false;
    }
    // cudaMemcpyAsync of n bytes between host and device (kind H2D: src is host; D2H: dst is host), split at
    // the locked ranges' bounds.
    void copy(void *dst, const void *src, size_t n, cudaMemcpyKind kind, cudaStream_t s) const {
        const bool h2d = kind == cudaMemcpyHostToDevice;
        const uintptr_t h0 = (uintptr_t)(h2d ? src : dst), h1 = h0 + n;
        uintptr_t pos = h0;
        auto piece = [&](uintptr_t x, uintptr_t y) {
            if (y <= x) return;
            const size_t off = x - h0;
            if (h2d) ck(cudaMemcpyAsync((char *)dst + off, (const char *)src + off, y - x, kind, s));
            else ck(cudaMemcpyAsync((char *)dst + off, (const char *)src + off, y - x, kind, s));
        };
        for (auto &r : ranges_) {
            if (r.second <= pos || r.first >= h1) continue;
            piece(pos, std::min(h1, r.first));
            piece(std::max(pos, r.first), std::min(h1, r.second));
            pos = std::min(h1, r.second);
        }
        piece(pos, h1);
    }

private:
    turtle_ctx *c_;
    uint32_t mode_;
    std::vector<std::pair<uintptr_t, uintptr_t>> ranges_;  // locked [first, second), ascending, disjoint
};

// Into a host result buffer (first touched when fresh), split at the locked ranges of `locks`.
// Synchronises s.
void copy_to_host(const HostLocks &locks, void *dst, const void *src, size_t bytes, cudaStream_t s, bool fresh) {
    if (bytes) {
        if (fresh) first_touch(dst, bytes);
        locks.copy(dst, src, bytes, cudaMemcpyDeviceToHost, s);
    }
    ck(cudaStreamSynchronize(s));
}

// Stream host reads to the device in chunks: chunk i is copied host->device on the copy stream
// while chunk i-1 is packed on `s` (two device staging buffers). Only the 2-bit codes and bitmaps
// stay on the device; the ASCII is never resident as a whole.
void pack_streamed(turtle_ctx *c, const turtle_reads *reads, uint64_t n_bases, const uint64_t *d_off,
                   size_t chunk, cudaStream_t s, PrePacked &pp, const LaunchCfg &lc, const HostLocks &locks) {
    const PackLayout L = PackLayout::of(n_bases);
    pp.P = (uint64_t *)ctx_alloc(c, 8 * L.p_words, s);
    pp.B = (uint64_t *)ctx_alloc(c, 8 * L.b_words, s);
    pp.S = (uint64_t *)ctx_alloc(c, 8 * L.b_words, s);
    ck(cudaMemsetAsync(pp.S, 0, 8 * L.b_words, s));
    chunk = (chunk + 63) & ~(size_t)63;  // chunk starts fall on 64-position boundaries (whole bitmap words)
    uint8_t *stage[2];
    for (auto &st : stage) st = (uint8_t *)ctx_alloc(c, chunk, s);
    for (int i = 0; i < 2; i++) ck(cudaEventRecord(c->ev_packed[i], s));  // both staging buffers start free
    const uint64_t n_chunks = n_bases ? (n_bases + chunk - 1) / chunk : 0;
    for (uint64_t i = 0; i < n_chunks; i++) {
        const int b = (int)(i & 1);
        const uint64_t c0 = i * chunk, c1 = c0 + chunk < n_bases ? c0 + chunk : n_bases;
        ck(cudaStreamWaitEvent(c->copy_stream, c->ev_packed[b], 0));  // its staging buffer was packed
        locks.copy(stage[b], reads->bases + c0, c1 - c0, cudaMemcpyHostToDevice, c->copy_stream);
        ck(cudaEventRecord(c->ev_h2d[b], c->copy_stream));
        ck(cudaStreamWaitEvent(s, c->ev_h2d[b], 0));
        const uint64_t g0 = c0 / 32, g1 = i + 1 == n_chunks ? L.pack_groups() : c1 / 32;
        launch_pack_groups(lc, stage[b] - c0, d_off, reads->n_reads, L, g0, g1, pp.P, pp.B);
        ck(cudaEventRecord(c->ev_packed[b], s));
    }
    ck(cudaEventRecord(c->ev_in[1], c->copy_stream));  // the last chunk has landed
    if (n_chunks == 0) launch_pack_groups(lc, nullptr, d_off, reads->n_reads, L, 0, L.pack_groups(), pp.P, pp.B);
    launch_mark_starts(lc, d_off, reads->n_reads, L, pp.S, c->d_err);
}

// Host-memory input streamed through two device staging buffers, then the path on the packed reads.
int count_streamed_impl(turtle_ctx *c, const turtle_reads *reads, uint64_t n_bases, const uint64_t *d_off, int k,
                        uint32_t min_count, const turtle_params *params, size_t chunk, cudaStream_t s,
                        DeviceOut &o, const HostLocks &locks, bool cturtle = false) {
    const turtle_params prm = resolve(params);
    if (!params_ok(prm)) return TURTLE_E_ARG;
    try {
        ctx_begin(c, s);
        L2Fetch l2(prm.l2_fetch_bytes);
        const LaunchCfg lc{c->sms, s};
        PrePacked pp{};
        pack_streamed(c, reads, n_bases, d_off, chunk, s, pp, lc, locks);
        if (k <= 32)
            run_count<uint64_t>(c, nullptr, n_bases, d_off, reads->n_reads, k, min_count, prm, s, o, &pp, nullptr,
                                cturtle);
        else run_count<Key128>(c, nullptr, n_bases, d_off, reads->n_reads, k, min_count, prm, s, o, &pp, nullptr, cturtle);
        c->stats.stage_launches[TURTLE_STAGE_PACK] = (uint32_t)((n_bases + chunk - 1) / chunk + 1);
        c->stats.launches += c->stats.stage_launches[TURTLE_STAGE_PACK];
        ctx_end(c, s);
        return TURTLE_OK;
    } catch (Fail f) {
        return fail_code(s, c, f.code);
    } catch (std::bad_alloc &) {
        return fail_code(s, c, TURTLE_E_NOMEM);
    }
}

// Host reads (one library, or a batch of them), one key range, bucketed form: the reads are copied
// in chunks on the copy stream while the GPU packs, validates and filters the windows whose bases
// have all arrived, so the input transfer overlaps pass 1. The number of windows is known only
// after the last chunk: the candidate buffer holds n_bases keys (an upper bound), and the filter
// and the buckets are sized from estimates of the windows (the result does not depend on them).
constexpr size_t OVERLAP_MIN = (size_t)64 << 20;  // inputs from this size on overlap their copy

// Positions per chunk: an eighth of the input, 16-256 MiB, a multiple of 128 (whole pass-1 tiles).
uint64_t overlap_chunk(uint64_t n_bases) {
    uint64_t c = (n_bases / 8 + 127) & ~(uint64_t)127;
    return std::min<uint64_t>(std::max<uint64_t>(c, (uint64_t)16 << 20), (uint64_t)256 << 20);
}
struct HostPiece {  // bases [start, start + len) of the concatenated positions live at src
    uint64_t start, len;
    const char *src;
};

template <class K>
void run_count_overlapped(turtle_ctx *c, const std::vector<HostPiece> &pieces, uint64_t n_bases, uint64_t n_reads,
                          uint8_t *d_bases, const uint64_t *d_off, int k, uint32_t min_count,
                          const turtle_params &prm, cudaStream_t s, DeviceOut &out, const HostLocks &locks,
                          const BatchTag *tag = nullptr, const std::vector<unsigned long long> *lib_w_est = nullptr) {
    const LaunchCfg lc{c->sms, s};
    turtle_stats st{};
    Timer tm{c, s, prm.timing != 0};
    uint32_t *err = c->d_err;
    unsigned long long *ctr = c->d_ctr;
    const PackLayout L = PackLayout::of(n_bases);
    uint64_t *P = (uint64_t *)ctx_alloc(c, 8 * L.p_words, s);
    uint64_t *B = (uint64_t *)ctx_alloc(c, 8 * L.b_words, s);
    uint64_t *S = (uint64_t *)ctx_alloc(c, 8 * L.b_words, s);
    uint64_t *V = (uint64_t *)ctx_alloc(c, 8 * L.v_words, s);
    ck(cudaMemsetAsync(S, 0, 8 * L.b_words, s));
    ck(cudaMemsetAsync(V + (L.v_words - 2), 0, 16, s));
    launch_mark_starts(lc, d_off, n_reads, L, S, err);  // read starts (and the offsets check) first
    // buffers: n_bases windows at most; sizes of the filter and of the buckets: n_bases - n_reads (k - 1),
    // the exact count when no read is shorter than k and none holds an ambiguous call
    const uint64_t Wmax = n_bases;
    const uint64_t lost = n_reads * (uint64_t)(k - 1);
    const uint64_t West = std::max<uint64_t>(n_bases > lost ? n_bases - lost : 0, n_bases / 4);
    const bool use_filter = min_count >= 2;
    FilterGeom fg{};
    uint64_t *lib_filter = nullptr;
    if (use_filter) {
        if (tag) {
            fg.n_sectors = lib_filter_regions(c, *lib_w_est, prm.filter_bits_per_window, &lib_filter, s);
            fg.sector_shift = 64;
        } else {
            fg.n_sectors = pow2_at_least((uint64_t)((double)West * prm.filter_bits_per_window / 256.0) + 1);
            fg.sector_shift = 64 - log2_exact(fg.n_sectors);
        }
        fg.words = (uint64_t *)ctx_alloc(c, 32 * fg.n_sectors, s);
        ck(cudaMemsetAsync(fg.words, 0, 32 * fg.n_sectors, s));
        fg.patterns = ctx_patterns(c, prm, s);
        fg.pat_mask = prm.n_patterns - 1;
        st.filter_bytes = 32 * fg.n_sectors;
    }
    constexpr int PART_BITS = 6;
    int bucket_bits = 0;
    const BucketGeom bg = tag ? lib_buckets(c, *lib_w_est, k, &bucket_bits, s, bucket_windows_of(prm))
                              : bucket_geom(West, 0u, 1u << PART_BITS, PART_BITS, k, &bucket_bits,
                                            bucket_windows_of(prm));
    const int hist_passes = (bucket_bits + 7) / 8;
    uint64_t *hist = (uint64_t *)ctx_alloc(c, 8 * 256 * 16, s);
    ck(cudaMemsetAsync(hist, 0, 8 * 256 * 16, s));
    K *cand = (K *)ctx_alloc(c, sizeof(K) * Wmax, s);
    K *firsts = use_filter ? cand : nullptr;  // first sightings fill the same buffer from the top
    ck(cudaMemsetAsync(ctr + C_CAND, 0, 8 * (C_N - C_CAND), s));
    const uint64_t n_words = L.v_words - 2, all_tiles = (n_bases + 127) / 128;
    const uint64_t chunk = overlap_chunk(n_bases);
    const uint64_t n_chunks = (n_bases + chunk - 1) / chunk;
    uint64_t w_done = 0, t_done = 0;
    // d_bases was allocated on s (stream-ordered): the copy stream starts after that point
    ck(cudaEventRecord(c->ev_packed[0], s));
    ck(cudaStreamWaitEvent(c->copy_stream, c->ev_packed[0], 0));
    tm.start(TURTLE_STAGE_FILTER);  // copies, packing, validity and pass 1, overlapped
    size_t pi = 0;  // first piece that may overlap the chunk
    for (uint64_t i = 0; i < n_chunks; i++) {
        const uint64_t c0 = i * chunk, c1 = std::min<uint64_t>(c0 + chunk, n_bases);
        const bool last = i + 1 == n_chunks;
        while (pi < pieces.size() && pieces[pi].start + pieces[pi].len <= c0) pi++;
        for (size_t q = pi; q < pieces.size() && pieces[q].start < c1; q++) {
            const uint64_t a = std::max(c0, pieces[q].start), b = std::min(c1, pieces[q].start + pieces[q].len);
            if (b > a)
                locks.copy(d_bases + a, pieces[q].src + (a - pieces[q].start), b - a, cudaMemcpyHostToDevice,
                           c->copy_stream);
        }
        ck(cudaEventRecord(c->ev_h2d[0], c->copy_stream));
        ck(cudaStreamWaitEvent(s, c->ev_h2d[0], 0));
        launch_pack_groups(lc, d_bases, d_off, n_reads, L, c0 / 32, last ? L.pack_groups() : c1 / 32, P, B);
        // validity word w needs positions below 64 (w + 2); a pass-1 tile covers two words
        const uint64_t w_ready = last ? n_words : (c1 / 64 > 1 ? c1 / 64 - 1 : 0);
        const uint64_t t_ready = last ? all_tiles : w_ready / 2;
        launch_valid(lc, L, k, B, S, V, ctr + C_WINDOWS, w_done, w_ready);
        if (w_ready > w_done) w_done = w_ready;
        launch_pass1<K>(lc, L, k, P, V, use_filter, fg, cand, ctr + C_CAND, Wmax, firsts, ctr + C_FIRST, Wmax, hist,
                        hist_passes, 0, 0u, 1u << PART_BITS, tag ? tag->lib_starts : nullptr, tag ? tag->n_libs : 0,
                        lib_filter, err, &bg, t_done, t_ready);
        if (t_ready > t_done) t_done = t_ready;
    }
    tm.stop(TURTLE_STAGE_FILTER);
    ck(cudaEventRecord(c->ev_in[1], c->copy_stream));  // the last chunk of the reads has landed
    st.stage_launches[TURTLE_STAGE_PACK] = (uint32_t)n_chunks + 1;
    st.stage_launches[TURTLE_STAGE_VALID] = (uint32_t)n_chunks;
    st.stage_launches[TURTLE_STAGE_FILTER] = (uint32_t)n_chunks;
    if (tag) {  // per-library window counts, for the results
        ck(cudaMemsetAsync(tag->lib_windows, 0, 8 * tag->n_libs, s));
        launch_lib_windows(lc, L, V, tag->lib_starts, tag->n_libs, tag->lib_windows);
    }
    read_back(c, s);
    const uint64_t W = c->h_ctr[C_WINDOWS], n_cand = c->h_ctr[C_CAND], n_first = c->h_ctr[C_FIRST];
    st.n_windows = W;
    st.n_candidates = n_cand;
    st.n_firsts = n_first;
    st.super_partitions = 1;
    out.n_windows = W;
    const PartOut po = bucketed_part<K>(c, lc, tm, st, min_count, cand, n_cand, use_filter ? cand + (Wmax - n_first) : nullptr,
                                        n_first, bg, bucket_bits, hist, true,
                                        sort_variant(prm, true, (int)(sizeof(K) / 8)),
                                        prm.bucket_slots != 4096, s);
    out.keys = po.keys;
    out.counts = po.counts;
    out.n = po.n;
    st.n_out = po.n;
    if (prm.timing) ck(cudaStreamSynchronize(s));  // the last stage's events may still be pending
    if (prm.timing)
        for (int i = TURTLE_STAGE_FILTER; i < TURTLE_STAGE_COUNT; i++) {
            float ms = 0.f;
            if ((i == TURTLE_STAGE_FILTER || st.stage_launches[i]) &&
                cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]) == cudaSuccess)
                st.stage_ms[i] = ms;
            else cudaGetLastError();
        }
    for (int i = 0; i < TURTLE_STAGE_COUNT; i++) st.launches += st.stage_launches[i];
    st.scratch_bytes = c->scratch_bytes;
    c->stats = st;
}

// One batched run: libraries `idx` (same k and min_count) concatenated on the device, counted by
// one pipeline with library-tagged keys, results split back per library into outs[] by a host
// thread of bo, which also frees the run's device results. A mixed run (K = Key128) holds libraries
// of different k (same min_count): each starts on a 128-position boundary (the gap filled with N,
// so no window crosses it), windows are keyed with their library's k and the tag sits in the top
// 6 key bits; results of libraries with k <= 32 are narrowed to 64-bit keys on the device.
template <class K>
int batch_run(turtle_ctx *c, const turtle_job *jobs, const std::vector<size_t> &idx, int tag_bits,
              const turtle_params *params, cudaStream_t s, turtle_result *outs, BatchOutput &bo,
              std::function<void(int)> done, bool mixed = false) {
    const int n_libs = (int)idx.size();
    int k = 0;  // the widest k (a mixed run's libraries carry their own)
    std::vector<int> lib_k(n_libs);
    for (int l = 0; l < n_libs; l++) {
        lib_k[l] = jobs[idx[l]].k;
        k = std::max(k, lib_k[l]);
    }
    const uint32_t min_count = jobs[idx[0]].min_count;
    const turtle_params prm = resolve(params);
    if (!params_ok(prm) || prm.shard_count > 1) return TURTLE_E_ARG;
    if (mixed && (sizeof(K) != 16 || n_libs > 64 || k > MIXED_K_MAX || prm.compact != 0)) return TURTLE_E_ARG;
    std::vector<uint64_t> lib_starts(n_libs + 1, 0), entry_starts(n_libs + 1, 0);
    for (int l = 0; l < n_libs; l++) {
        const turtle_job &j = jobs[idx[l]];
        lib_starts[l + 1] = lib_starts[l] + (j.offsets[j.n_reads] - j.offsets[0]);
        if (mixed && l + 1 < n_libs) lib_starts[l + 1] = (lib_starts[l + 1] + 127) & ~127ull;
        entry_starts[l + 1] = entry_starts[l] + j.n_reads;
    }
    const uint64_t n_bases = lib_starts[n_libs], n_reads = entry_starts[n_libs];
    std::vector<unsigned long long> lib_windows(n_libs, 0);
    DeviceOut o;
    if (prm.host_transfer == 0 && cudaSetDevice(c->device) == cudaSuccess) calibrate_transfers(c, s);
    cudaGetLastError();
    HostLocks locks(c, prm.host_transfer);  // the libraries' arrays, page-locked while they are copied
    for (int l = 0; l < n_libs; l++) {
        const turtle_job &j = jobs[idx[l]];
        locks.add(j.bases + j.offsets[0], j.offsets[j.n_reads] - j.offsets[0]);
        locks.add(j.offsets, 8 * (j.n_reads + 1));
    }
    try {
        ctx_begin(c, s);
        const LaunchCfg lc{c->sms, s};
        uint8_t *d_bases = (uint8_t *)ctx_alloc(c, n_bases ? n_bases : 16, s);
        uint64_t *d_src = (uint64_t *)ctx_alloc(c, 8 * (n_reads + n_libs), s);
        uint64_t *d_off = (uint64_t *)ctx_alloc(c, 8 * (n_reads + 1), s);
        uint64_t *d_tab = (uint64_t *)ctx_alloc(c, 8 * 2 * (n_libs + 1), s);  // lib_starts, entry_starts
        unsigned long long *d_lw = (unsigned long long *)ctx_alloc(c, 8 * n_libs, s);
        // the bucketed form overlaps the copy of the bases with pass 1; the global form copies first
        const bool overlapped = prm.compact == 0 && n_bases >= OVERLAP_MIN && !mixed;
        std::vector<HostPiece> pieces;
        std::vector<unsigned long long> w_est(n_libs);
        for (int l = 0; l < n_libs; l++) {
            const turtle_job &j = jobs[idx[l]];
            const uint64_t nb = j.offsets[j.n_reads] - j.offsets[0];
            const uint64_t lost = j.n_reads * (uint64_t)(lib_k[l] - 1);
            w_est[l] = std::max<uint64_t>(nb > lost ? nb - lost : 0, nb / 4);
            if (overlapped) pieces.push_back(HostPiece{lib_starts[l], nb, j.bases + j.offsets[0]});
            else if (nb) locks.copy(d_bases + lib_starts[l], j.bases + j.offsets[0], nb, cudaMemcpyHostToDevice, s);
            if (mixed && lib_starts[l + 1] > lib_starts[l] + nb)  // the gap up to the next library: N
                ck(cudaMemsetAsync(d_bases + lib_starts[l] + nb, 'N', lib_starts[l + 1] - lib_starts[l] - nb, s));
            locks.copy(d_src + entry_starts[l] + l, j.offsets, 8 * (j.n_reads + 1), cudaMemcpyHostToDevice, s);
        }
        int *d_libk = nullptr;
        if (mixed) {
            d_libk = (int *)ctx_alloc(c, 4 * n_libs, s);
            ck(cudaMemcpyAsync(d_libk, lib_k.data(), 4 * n_libs, cudaMemcpyHostToDevice, s));
        }
        ck(cudaMemcpyAsync(d_tab, lib_starts.data(), 8 * (n_libs + 1), cudaMemcpyHostToDevice, s));
        ck(cudaMemcpyAsync(d_tab + n_libs + 1, entry_starts.data(), 8 * (n_libs + 1), cudaMemcpyHostToDevice, s));
        launch_batch_offsets(lc, d_src, d_tab + n_libs + 1, d_tab, n_libs, d_off, n_reads + 1);
        BatchTag tag{d_tab, n_libs, mixed ? MIXED_TAG_BITS : tag_bits, d_lw};
        if (mixed) {
            tag.lib_k = d_libk;
            tag.tag_shift = 128 - MIXED_TAG_BITS;
            tag.host_starts = lib_starts.data();
            tag.host_k = lib_k.data();
        }
        L2Fetch l2(prm.l2_fetch_bytes);
        if (overlapped)
            run_count_overlapped<K>(c, pieces, n_bases, n_reads, d_bases, d_off, k, min_count, prm, s, o, locks, &tag,
                                    &w_est);
        else run_count<K>(c, d_bases, n_bases, d_off, n_reads, k, min_count, prm, s, o, nullptr, &tag);
        // split on the device: library boundaries + tag bits cleared, then one copy per library
        std::vector<uint64_t> starts(n_libs + 1, ~0ull);
        if (tag.tag_bits) {
            uint64_t *d_starts = (uint64_t *)ctx_alloc(c, 8 * n_libs, s);
            ck(cudaMemsetAsync(d_starts, 0xff, 8 * n_libs, s));
            launch_split_tags<K>(lc, (K *)o.keys, o.n, mixed ? tag.tag_shift : 2 * k, d_starts);
            ck(cudaMemcpyAsync(starts.data(), d_starts, 8 * n_libs, cudaMemcpyDeviceToHost, s));
        } else {
            starts[0] = 0;
        }
        ck(cudaMemcpyAsync(lib_windows.data(), d_lw, 8 * n_libs, cudaMemcpyDeviceToHost, s));
        ck(cudaStreamSynchronize(s));
        starts[n_libs] = o.n;
        for (int l = n_libs - 1; l >= 0; l--)
            if (starts[l] == ~0ull) starts[l] = starts[l + 1];  // no entries: an empty range
        // a mixed run: the keys of its libraries with k <= 32, narrowed to 64 bits, at narrow_at[l]
        std::vector<uint64_t> narrow_at(n_libs, ~0ull);
        uint64_t *d_narrow = nullptr;
        if (mixed) {
            uint64_t n_narrow = 0;
            for (int l = 0; l < n_libs; l++)
                if (lib_k[l] <= 32) {
                    narrow_at[l] = n_narrow;
                    n_narrow += starts[l + 1] - starts[l];
                }
            if (n_narrow) {
                d_narrow = (uint64_t *)ctx_alloc(c, 8 * n_narrow, s, true);
                for (int l = 0; l < n_libs; l++)
                    if (lib_k[l] <= 32)
                        launch_narrow_keys(lc, (const Key128 *)o.keys + starts[l], starts[l + 1] - starts[l],
                                           d_narrow + narrow_at[l]);
                ck(cudaStreamSynchronize(s));  // the copy-out runs on its own stream
            }
        }
        // the device results now belong to the copy-out thread (the next run must not free them)
        for (auto it = c->result.begin(); it != c->result.end();)
            it = (*it == o.keys || *it == (void *)o.counts || *it == (void *)d_narrow) ? c->result.erase(it) : it + 1;
        ctx_end(c, s);
        std::vector<size_t> lib_idx = idx;
        const int dev = c->device;
        const uint32_t transfer = prm.host_transfer;
        cudaStream_t os = bo.stream();
        bo.post([=, &bo]() {
            int rc = TURTLE_OK;
            if (cudaSetDevice(dev) != cudaSuccess) rc = TURTLE_E_CUDA;
            for (int l = 0; l < n_libs && rc == TURTLE_OK; l++) {
                turtle_result &r = outs[lib_idx[l]];
                const bool narrowed = narrow_at[l] != ~0ull;
                const int kw = narrowed ? 1 : (int)(sizeof(K) / 8);
                r.k = lib_k[l];
                r.n = starts[l + 1] - starts[l];
                r.n_windows = lib_windows[l];
                bool fk = true, fc = true;
                r.keys = (uint64_t *)result_alloc(8 * kw * (r.n ? r.n : 1), &fk);
                r.counts = (uint32_t *)result_alloc(4 * (r.n ? r.n : 1), &fc);
                if (!r.keys || !r.counts) {
                    rc = TURTLE_E_NOMEM;
                    break;
                }
                if (r.n) {
                    try {
                        if (fk) first_touch(r.keys, 8 * kw * r.n);
                        if (fc) first_touch(r.counts, 4 * r.n);
                        HostLocks rl(c, transfer);
                        rl.add(r.keys, 8 * kw * r.n);
                        rl.add(r.counts, 4 * r.n);
                        const void *src = narrowed ? (const void *)(d_narrow + narrow_at[l])
                                                   : (const void *)((const K *)o.keys + starts[l]);
                        copy_to_host(rl, r.keys, src, 8 * kw * r.n, os, false);
                        copy_to_host(rl, r.counts, o.counts + starts[l], 4 * r.n, os, false);
                    } catch (Fail f) {
                        rc = f.code;
                    }
                }
            }
            cudaFreeAsync(o.keys, os);
            cudaFreeAsync(o.counts, os);
            if (d_narrow) cudaFreeAsync(d_narrow, os);
            cudaGetLastError();
            if (rc) bo.fail(rc);
            if (done) done(rc);
        });
    } catch (Fail f) {
        return fail_code(s, c, f.code);
    } catch (std::exception &) {  // bad_alloc, or no thread for the copy-out
        return fail_code(s, c, TURTLE_E_NOMEM);
    }
    return TURTLE_OK;
}

std::mutex g_default_mu;
turtle_ctx *g_default[64] = {};

// Batched form with params.autotune: the knobs of a group (same k and min_count) come from
// turtle_autotune on the group's largest library, copied to the device for the purpose (tuned once
// per class of input; later groups of the class reuse the cached knobs without a copy).
int tune_group(turtle_ctx *c, const turtle_job *jobs, const std::vector<size_t> &idx, const turtle_params &prm,
               cudaStream_t s, turtle_params *out) {
    size_t big = idx[0];
    for (size_t i : idx)
        if (jobs[i].offsets[jobs[i].n_reads] - jobs[i].offsets[0] > jobs[big].offsets[jobs[big].n_reads] - jobs[big].offsets[0])
            big = i;
    const turtle_job &j = jobs[big];
    const uint64_t nb = j.offsets[j.n_reads] - j.offsets[0];
    turtle_params base0 = prm;
    base0.autotune = 0;
    if (tune_cache_lookup(j.k, j.min_count, base0, nb, out)) return TURTLE_OK;  // tuned before: no copy
    std::vector<uint64_t> off(j.offsets, j.offsets + j.n_reads + 1);
    for (uint64_t &o : off) o -= j.offsets[0];
    turtle_params base = prm;
    base.autotune = 0;
    uint8_t *d_b = nullptr;
    uint64_t *d_o = nullptr;
    int rc = TURTLE_OK;
    if (cudaMalloc(&d_b, nb ? nb : 16) != cudaSuccess || cudaMalloc(&d_o, 8 * off.size()) != cudaSuccess) rc = TURTLE_E_NOMEM;
    if (!rc && ((nb && cudaMemcpyAsync(d_b, j.bases + j.offsets[0], nb, cudaMemcpyHostToDevice, s) != cudaSuccess) ||
                cudaMemcpyAsync(d_o, off.data(), 8 * off.size(), cudaMemcpyHostToDevice, s) != cudaSuccess))
        rc = TURTLE_E_CUDA;
    if (!rc) rc = turtle_autotune(c, d_b, nb, d_o, j.n_reads, j.k, j.min_count, &base, s, out, nullptr);
    cudaStreamSynchronize(s);
    if (d_b) cudaFree(d_b);
    if (d_o) cudaFree(d_o);
    cudaGetLastError();
    out->autotune = 0;
    return rc;
}

}  // namespace

BatchOutput::BatchOutput() {
    if (cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        stream_ = nullptr;
    }
    worker_ = std::thread([this] { loop(); });
}

BatchOutput::~BatchOutput() {
    drain();
    {
        std::lock_guard<std::mutex> g(mu_);
        stop_ = true;
    }
    cv_.notify_all();
    worker_.join();
    if (stream_) cudaStreamDestroy(stream_);
    cudaGetLastError();
}

void BatchOutput::loop() {
    std::unique_lock<std::mutex> lk(mu_);
    for (;;) {
        cv_.wait(lk, [&] { return stop_ || !tasks_.empty(); });
        if (tasks_.empty()) return;  // stop_ with nothing left
        std::function<void()> t = std::move(tasks_.front());
        tasks_.pop_front();
        busy_ = true;
        lk.unlock();
        t();
        lk.lock();
        busy_ = false;
        cv_idle_.notify_all();
    }
}

void BatchOutput::post(std::function<void()> task) {
    {
        std::lock_guard<std::mutex> g(mu_);
        tasks_.push_back(std::move(task));
    }
    cv_.notify_one();
}

void BatchOutput::fail(int code) {
    std::lock_guard<std::mutex> g(mu_);
    if (rc_ == TURTLE_OK) rc_ = code;
}

int BatchOutput::drain() {
    std::unique_lock<std::mutex> lk(mu_);
    cv_idle_.wait(lk, [&] { return tasks_.empty() && !busy_; });
    return rc_;
}

size_t batch_capacity(int k) {
    const int room = (2 * k <= 64 ? 64 : 128) - 2 * k;  // key bits above the 2k of the key
    return room >= 6 ? 64 : ((size_t)1 << room);
}

// Whether libraries idx (same min_count, k <= MIXED_K_MAX) are expected to finish sooner in mixed runs
// than in runs grouped by k. A run costs a fixed time (its launches, host synchronisations and copy
// set-up: RUN_MS) plus time per base; in a mixed run the libraries with k <= 32 are keyed with 128 bits
// instead of 64, which costs them MIX_EXTRA_NS more per base. Both measured on GB300 (host arrays in
// and out): 12 to 48 libraries of 20 kbase to 10 Mbase over 3 to 12 k.
bool mixed_runs_pay(const turtle_job *jobs, const std::vector<size_t> &idx) {
    constexpr double RUN_MS = 0.25, MIX_EXTRA_NS = 0.025;
    std::map<int, size_t> per_k;
    double narrow_bases = 0;
    for (size_t i : idx) {
        per_k[jobs[i].k]++;
        if (jobs[i].k <= 32) narrow_bases += (double)(jobs[i].offsets[jobs[i].n_reads] - jobs[i].offsets[0]);
    }
    size_t grouped = 0;
    for (auto &kv : per_k) grouped += (kv.second + batch_capacity(kv.first) - 1) / batch_capacity(kv.first);
    const size_t mixed = (idx.size() + 63) / 64;
    return grouped > mixed && (double)(grouped - mixed) * RUN_MS > narrow_bases * MIX_EXTRA_NS * 1e-6;
}

int batch_run_jobs(turtle_ctx *c, const turtle_job *jobs, const std::vector<size_t> &idx, const turtle_params *params,
                   cudaStream_t s, turtle_result *outs, BatchOutput &bo, std::function<void(int)> done, bool mixed) {
    if (mixed) {
        if (idx.empty() || idx.size() > 64 || !bo.ok()) return TURTLE_E_ARG;
        for (size_t i : idx)
            if (jobs[i].k > MIXED_K_MAX || jobs[i].min_count != jobs[idx[0]].min_count) return TURTLE_E_ARG;
        return batch_run<Key128>(c, jobs, idx, MIXED_TAG_BITS, params, s, outs, bo, done, true);
    }
    if (idx.empty() || idx.size() > batch_capacity(jobs[idx[0]].k) || !bo.ok()) return TURTLE_E_ARG;
    const int k = jobs[idx[0]].k;
    int tag_bits = 0;
    while (((size_t)1 << tag_bits) < idx.size()) tag_bits++;
    return 2 * k + tag_bits <= 64 ? batch_run<uint64_t>(c, jobs, idx, tag_bits, params, s, outs, bo, done)
                                  : batch_run<Key128>(c, jobs, idx, tag_bits, params, s, outs, bo, done);
}


extern "C" {

void turtle_params_default(turtle_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->struct_size = sizeof(turtle_params);
    p->filter_bits_per_window = 1.0f;
    p->pattern_bits = 4;
    p->n_patterns = 1024;
    p->pattern_seed = 0x7475727469ull;
    p->timing = 0;
    p->l2_fetch_bytes = 0;
}

const char *turtle_strerror(int code) {
    switch (code) {
    case TURTLE_OK: return "ok";
    case TURTLE_E_ARG: return "invalid argument";
    case TURTLE_E_NOMEM: return "out of memory";
    case TURTLE_E_CUDA: return "CUDA runtime error";
    case TURTLE_E_OVERFLOW: return "count overflows uint32";
    case TURTLE_E_TIMEOUT: return "timed out";
    case TURTLE_E_BUSY: return "job does not fit the HBM budget";
    case TURTLE_E_DEVICE: return "device-side check failed";
    case TURTLE_E_NODEV: return "no CUDA device";
    case TURTLE_E_CAPACITY: return "output buffer too small";
    case TURTLE_E_TOO_LARGE: return "input larger than the fixed scratch of the allocation-free entry point";
    default: return "unknown error";
    }
}

const char *turtle_stage_name(int stage) {
    static const char *names[TURTLE_STAGE_COUNT] = {"pack", "valid", "filter", "hist", "sort",
                                                    "rle", "table", "recount", "threshold", "merge"};
    return stage >= 0 && stage < TURTLE_STAGE_COUNT ? names[stage] : "?";
}

int turtle_ctx_create(int device, turtle_ctx **out) {
    if (!out) return TURTLE_E_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return TURTLE_E_NODEV;
    }
    if (device < 0 || device >= n) return TURTLE_E_ARG;
    turtle_ctx *c = new (std::nothrow) turtle_ctx();
    if (!c) return TURTLE_E_NOMEM;
    c->device = device;
    try {
        ck(cudaSetDevice(device));
        ck(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device));
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        ck(cudaMemPoolCreate(&c->pool, &props));
        uint64_t keep = ~0ull;
        ck(cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep));
        ck(cudaMalloc(&c->d_err, 64));
        ck(cudaMalloc(&c->d_ctr, sizeof(unsigned long long) * C_N));
        ck(cudaMallocHost(&c->h_ctr, sizeof(unsigned long long) * C_N));
        ck(cudaMallocHost(&c->h_err, 64));
        ck(cudaMallocHost(&c->h_hist, 8 * 256 * 16));
        for (auto &e : c->ev) ck(cudaEventCreate(&e));
        for (auto &e : c->ev_h2d) ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        for (auto &e : c->ev_packed) ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        for (auto &e : c->ev_in) ck(cudaEventCreate(&e));
        ck(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    } catch (Fail f) {
        turtle_ctx_destroy(c);
        return f.code;
    }
    *out = c;
    return TURTLE_OK;
}

void turtle_ctx_destroy(turtle_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->last_stream) cudaStreamSynchronize(c->last_stream);
    cudaDeviceSynchronize();
    for (void *p : c->scratch) cudaFree(p);
    for (void *p : c->result) cudaFree(p);
    if (c->d_patterns) cudaFree(c->d_patterns);
    if (c->d_err) cudaFree(c->d_err);
    if (c->d_ctr) cudaFree(c->d_ctr);
    if (c->h_ctr) cudaFreeHost(c->h_ctr);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->h_hist) cudaFreeHost(c->h_hist);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    for (auto &e : c->ev_h2d)
        if (e) cudaEventDestroy(e);
    for (auto &e : c->ev_packed)
        if (e) cudaEventDestroy(e);
    for (auto &e : c->ev_in)
        if (e) cudaEventDestroy(e);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->pool) cudaMemPoolDestroy(c->pool);
    cudaGetLastError();
    delete c;
}

void turtle_ctx_trim(turtle_ctx *c) {
    if (!c) return;
    if (cudaSetDevice(c->device) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (c->last_stream) cudaStreamSynchronize(c->last_stream);
    cudaDeviceSynchronize();
    cudaMemPoolTrimTo(c->pool, 0);
    cudaGetLastError();
}

int turtle_ctx_pool_bytes(const turtle_ctx *c, uint64_t *used, uint64_t *reserved) {
    if (!c) return TURTLE_E_ARG;
    uint64_t u = 0, r = 0;
    if (cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrUsedMemCurrent, &u) != cudaSuccess ||
        cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrReservedMemCurrent, &r) != cudaSuccess) {
        cudaGetLastError();
        return TURTLE_E_CUDA;
    }
    if (used) *used = u;
    if (reserved) *reserved = r;
    return TURTLE_OK;
}

int turtle_test_inject(int what, uint64_t value) {
    switch (what) {
    case TURTLE_INJECT_NONE:
        g_inject.device_alloc = -1;
        g_inject.host_alloc = -1;
        g_inject.lookback_spins = 0;
        g_inject.cand_cap = 0;
        return TURTLE_OK;
    case TURTLE_INJECT_DEVICE_ALLOC: g_inject.device_alloc = (int64_t)value; return TURTLE_OK;
    case TURTLE_INJECT_HOST_ALLOC: g_inject.host_alloc = (int64_t)value; return TURTLE_OK;
    case TURTLE_INJECT_LOOKBACK:
        if (value == 0 || value > 0xffffffffull) return TURTLE_E_ARG;
        g_inject.lookback_spins = (uint32_t)value;
        return TURTLE_OK;
    case TURTLE_INJECT_CAND_CAP:
        if (value == 0) return TURTLE_E_ARG;
        g_inject.cand_cap = value;
        return TURTLE_OK;
    default: return TURTLE_E_ARG;
    }
}

int turtle_shard_bounds(const uint64_t *part_windows, uint32_t n_parts, uint32_t n_shards, uint32_t *bounds) {
    if (!part_windows || !bounds || n_parts == 0 || n_shards == 0) return TURTLE_E_ARG;
    shard_bounds(part_windows, n_parts, n_shards, bounds);
    return TURTLE_OK;
}

int turtle_ctx_stats(const turtle_ctx *c, turtle_stats *st) {
    if (!c || !st) return TURTLE_E_ARG;
    *st = c->stats;
    return TURTLE_OK;
}

int turtle_count_device(turtle_ctx *c, const uint8_t *bases, uint64_t n_bases, const uint64_t *offsets,
                        uint64_t n_reads, int k, uint32_t min_count, const turtle_params *params, void *stream,
                        turtle_device_result *out) {
    if (!out) return TURTLE_E_ARG;
    memset(out, 0, sizeof(*out));
    DeviceOut o;
    const int rc = count_device_impl(c, bases, n_bases, offsets, n_reads, k, min_count, params, (cudaStream_t)stream, o);
    if (rc) return rc;
    out->k = k;
    out->key_words = k <= 32 ? 1 : 2;
    out->n = o.n;
    out->keys = (const uint64_t *)o.keys;
    out->counts = o.counts;
    out->n_windows = o.n_windows;
    return TURTLE_OK;
}

int turtle_frequent_device(turtle_ctx *c, const uint8_t *bases, uint64_t n_bases, const uint64_t *offsets,
                           uint64_t n_reads, int k, const turtle_params *params, void *stream,
                           turtle_device_result *out) {
    if (!out) return TURTLE_E_ARG;
    memset(out, 0, sizeof(*out));
    DeviceOut o;
    const int rc = count_device_impl(c, bases, n_bases, offsets, n_reads, k, 2, params, (cudaStream_t)stream, o, true);
    if (rc) return rc;
    out->k = k;
    out->key_words = k <= 32 ? 1 : 2;
    out->n = o.n;
    out->keys = (const uint64_t *)o.keys;
    out->counts = nullptr;
    out->n_windows = o.n_windows;
    return TURTLE_OK;
}

static turtle_ctx *default_ctx(int *rc) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        *rc = TURTLE_E_NODEV;
        return nullptr;
    }
    if (dev < 0 || dev >= 64) {
        *rc = TURTLE_E_ARG;
        return nullptr;
    }
    if (!g_default[dev]) {
        *rc = turtle_ctx_create(dev, &g_default[dev]);
        if (*rc) return nullptr;
    }
    *rc = TURTLE_OK;
    return g_default[dev];
}

}  // extern "C"

uint64_t footprint_estimate(uint64_t n_bases, uint64_t n_reads, int k, uint32_t min_count, const turtle_params *p) {
    turtle_params d;
    turtle_params_default(&d);
    const turtle_params &prm = (p && p->struct_size == sizeof(turtle_params)) ? *p : d;
    const double kb = k <= 32 ? 8.0 : 16.0;
    const double filter = min_count >= 2 ? prm.filter_bits_per_window / 8.0 : 0.0;
    const double per_base = 1.0 + 0.25 + 3.0 / 8.0 + 2.0 * kb + 12.0 + filter + 8.0;  // windows <= bases
    return (uint64_t)(per_base * (double)n_bases) + 8 * (n_reads + 1) + (64ull << 20);
}

// Host-memory form on a given context: copy (or stream) the reads in, run the path, copy the result out.
int count_host_impl(turtle_ctx *c, const turtle_reads *reads, int k, uint32_t min_count, const turtle_params *params,
                    void *stream, turtle_result *out, bool cturtle) {
    if (!out) return TURTLE_E_ARG;
    memset(out, 0, sizeof(*out));
    if (!reads || !reads->offsets || (reads->n_reads && !reads->bases) || k < 1 || k > 64 || min_count < 1)
        return TURTLE_E_ARG;
    // every offsets pair is checked on the device while packing (TURTLE_E_ARG)
    using clk = std::chrono::steady_clock;
    auto ms_since = [](clk::time_point t) { return std::chrono::duration<float, std::milli>(clk::now() - t).count(); };
    const clk::time_point t_call = clk::now();
    float host_ms[TURTLE_HOST_COUNT] = {};
    int rc = 0;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t n_bases = reads->offsets[reads->n_reads];
    const turtle_params prm = resolve(params);
    size_t chunk = (size_t)prm.stream_chunk_mib << 20;
    if (!chunk) {  // stream when the ASCII would take more than a quarter of the free device memory
        size_t free_b = 0, total_b = 0;
        if (cudaSetDevice(c->device) == cudaSuccess && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess &&
            n_bases > free_b / 4)
            chunk = (size_t)1 << 30;
        cudaGetLastError();
    }
    const bool streamed = chunk != 0;
    // large host inputs, one key range, bucketed form: overlap the copy with pass 1
    bool overlapped = false;
    if (!streamed && !cturtle && prm.compact == 0 && (min_count == 1 || !prm.recount_windows) &&
        prm.shard_count <= 1 && n_bases >= OVERLAP_MIN && params_ok(prm)) {
        size_t free_b = 0, total_b = 0;
        if (cudaSetDevice(c->device) == cudaSuccess && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
            const double kb = k <= 32 ? 8.0 : 16.0;
            const double need = (double)n_bases * (1.0 + 0.25 + 0.5 + 3.0 * kb + 8.0 + prm.filter_bits_per_window / 8.0);
            overlapped = need <= 0.7 * (double)free_b;
        }
        cudaGetLastError();
    }
    uint8_t *d_bases = nullptr;
    uint64_t *d_off = nullptr;
    if (cudaSetDevice(c->device) != cudaSuccess) {
        cudaGetLastError();
        return TURTLE_E_CUDA;
    }
    if (prm.host_transfer == 0) calibrate_transfers(c, s);
    // the caller's arrays, page-locked for this call when that is faster (see calibrate_transfers)
    HostLocks locks(c, prm.host_transfer);
    locks.add(reads->bases, n_bases);
    locks.add(reads->offsets, 8 * (reads->n_reads + 1));
    try {
        ck(cudaSetDevice(c->device));
        if (!streamed) ck(cudaMallocFromPoolAsync((void **)&d_bases, n_bases ? n_bases : 16, c->pool, s));
        ck(cudaMallocFromPoolAsync((void **)&d_off, 8 * (reads->n_reads + 1), c->pool, s));
        ck(cudaEventRecord(c->ev_in[0], s));  // the input copies start here
        locks.copy(d_off, reads->offsets, 8 * (reads->n_reads + 1), cudaMemcpyHostToDevice, s);
        if (n_bases && !streamed && !overlapped) locks.copy(d_bases, reads->bases, n_bases, cudaMemcpyHostToDevice, s);
        if (!streamed && !overlapped) ck(cudaEventRecord(c->ev_in[1], s));  // (streamed/overlapped: after the last chunk)
    } catch (Fail f) {
        if (d_bases) cudaFreeAsync(d_bases, s);
        if (d_off) cudaFreeAsync(d_off, s);
        return f.code;
    }
    host_ms[TURTLE_HOST_INPUT] = ms_since(t_call);
    const clk::time_point t_path = clk::now();
    DeviceOut o;
    if (overlapped) {
        try {
            ctx_begin(c, s);
            L2Fetch l2(prm.l2_fetch_bytes);
            const std::vector<HostPiece> pieces{HostPiece{0, n_bases, reads->bases}};
            if (k <= 32)
                run_count_overlapped<uint64_t>(c, pieces, n_bases, reads->n_reads, d_bases, d_off, k, min_count, prm, s,
                                               o, locks);
            else run_count_overlapped<Key128>(c, pieces, n_bases, reads->n_reads, d_bases, d_off, k, min_count, prm, s, o,
                                              locks);
            ctx_end(c, s);
        } catch (Fail f) {
            rc = fail_code(s, c, f.code);
        } catch (std::bad_alloc &) {
            rc = fail_code(s, c, TURTLE_E_NOMEM);
        }
    } else if (streamed) {
        rc = count_streamed_impl(c, reads, n_bases, d_off, k, min_count, params, chunk, s, o, locks, cturtle);
    } else {
        rc = count_device_impl(c, d_bases, n_bases, d_off, reads->n_reads, k, min_count, params, s, o, cturtle);
    }
    if (d_bases) cudaFreeAsync(d_bases, s);
    cudaFreeAsync(d_off, s);
    if (rc) return rc;
    host_ms[TURTLE_HOST_PATH] = ms_since(t_path);
    const int kw = k <= 32 ? 1 : 2;
    bool fk = true, fc = true;
    out->keys = (uint64_t *)result_alloc(8 * kw * (o.n ? o.n : 1), &fk);
    out->counts = o.counts ? (uint32_t *)result_alloc(4 * (o.n ? o.n : 1), &fc) : nullptr;  // cTurtle: no counts
    if (!out->keys || (o.counts && !out->counts)) {
        turtle_result_free(out);
        return TURTLE_E_NOMEM;
    }
    const size_t key_bytes = 8 * kw * o.n, count_bytes = o.counts ? 4 * o.n : 0;
    try {
        const clk::time_point t_touch = clk::now();  // fresh host pages are touched first (see first_touch)
        if (fk && key_bytes) first_touch(out->keys, key_bytes);
        if (fc && count_bytes) first_touch(out->counts, count_bytes);
        host_ms[TURTLE_HOST_TOUCH] = ms_since(t_touch);
        const clk::time_point t_out = clk::now();
        {
            HostLocks rl(c, prm.host_transfer);
            rl.add(out->keys, key_bytes);
            rl.add(out->counts, count_bytes);
            copy_to_host(rl, out->keys, o.keys, key_bytes, s, false);
            if (o.counts) copy_to_host(rl, out->counts, o.counts, count_bytes, s, false);
        }
        host_ms[TURTLE_HOST_OUTPUT] = ms_since(t_out);
    } catch (Fail f) {
        cudaGetLastError();
        turtle_result_free(out);
        return f.code;
    }
    out->k = k;
    out->n = o.n;
    out->n_windows = o.n_windows;
    for (int i = 0; i < TURTLE_HOST_COUNT; i++) c->stats.host_ms[i] = host_ms[i];
    float h2d = 0.f;
    if (cudaEventElapsedTime(&h2d, c->ev_in[0], c->ev_in[1]) != cudaSuccess) {
        cudaGetLastError();
        h2d = 0.f;
    }
    c->stats.h2d_ms = h2d;
    c->stats.h2d_bytes = n_bases + 8 * (reads->n_reads + 1);
    c->stats.d2h_bytes = key_bytes + count_bytes;
    c->stats.host_locked = locks.locked(reads->bases + n_bases / 2) ? 1u : 0u;
    c->stats.transfer_gbs[0] = (float)c->gbs_pageable;
    c->stats.transfer_gbs[1] = (float)c->gbs_register;
    c->stats.transfer_gbs[2] = (float)c->gbs_registered;
    return TURTLE_OK;
}

extern "C" {

int turtle_count_ex(const turtle_reads *reads, int k, uint32_t min_count, const turtle_params *params, void *stream,
                    turtle_result *out) {
    if (!out) return TURTLE_E_ARG;
    memset(out, 0, sizeof(*out));
    if (!reads || !reads->offsets || (reads->n_reads && !reads->bases) || k < 1 || k > 64 || min_count < 1)
        return TURTLE_E_ARG;  // argument errors are reported before any device is touched
    if (reads->offsets[reads->n_reads] < reads->offsets[0]) return TURTLE_E_ARG;  // the device checks every pair
    std::lock_guard<std::mutex> g(g_default_mu);
    int rc = 0;
    turtle_ctx *c = default_ctx(&rc);
    if (!c) return rc;
    return count_host_impl(c, reads, k, min_count, params, stream, out, false);
}

int turtle_ctx_count(turtle_ctx *c, const turtle_reads *reads, int k, uint32_t min_count, const turtle_params *params,
                     void *stream, turtle_result *out) {
    if (!out) return TURTLE_E_ARG;
    memset(out, 0, sizeof(*out));
    if (!c || !reads || !reads->offsets || (reads->n_reads && !reads->bases) || k < 1 || k > 64 || min_count < 1)
        return TURTLE_E_ARG;
    if (reads->offsets[reads->n_reads] < reads->offsets[0]) return TURTLE_E_ARG;  // the device checks every pair
    return count_host_impl(c, reads, k, min_count, params, stream, out, false);
}

int turtle_frequent(const turtle_reads *reads, int k, const turtle_params *params, void *stream, turtle_result *out) {
    if (!out) return TURTLE_E_ARG;
    memset(out, 0, sizeof(*out));
    if (!reads || !reads->offsets || (reads->n_reads && !reads->bases) || k < 1 || k > 64) return TURTLE_E_ARG;
    if (reads->offsets[reads->n_reads] < reads->offsets[0]) return TURTLE_E_ARG;
    std::lock_guard<std::mutex> g(g_default_mu);
    int rc = 0;
    turtle_ctx *c = default_ctx(&rc);
    if (!c) return rc;
    return count_host_impl(c, reads, k, 2, params, stream, out, true);
}

int turtle_count_batch(const turtle_job *jobs, size_t n_jobs, const turtle_params *params, void *stream,
                       turtle_result *outs) {
    if ((n_jobs && (!jobs || !outs))) return TURTLE_E_ARG;
    for (size_t i = 0; i < n_jobs; i++) {
        memset(&outs[i], 0, sizeof(turtle_result));
        const turtle_job &j = jobs[i];
        if (!j.offsets || (j.n_reads && !j.bases) || j.k < 1 || j.k > 64 || j.min_count < 1 ||
            j.offsets[j.n_reads] < j.offsets[0])
            return TURTLE_E_ARG;
    }
    std::lock_guard<std::mutex> g(g_default_mu);
    int rc = 0;
    turtle_ctx *c = default_ctx(&rc);
    if (!c) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    BatchOutput bo;
    if (!bo.ok()) return TURTLE_E_CUDA;
    // group by (k, min_count); a run holds as many libraries as the spare key bits can tag (<= 64)
    const turtle_params prm = resolve(params);
    std::map<std::pair<int, uint32_t>, std::vector<size_t>> groups;
    std::map<uint32_t, std::vector<size_t>> mixed;  // min_count -> libraries counted in mixed runs
    for (size_t i = 0; i < n_jobs; i++) groups[{jobs[i].k, jobs[i].min_count}].push_back(i);
    if (prm.batch_mixed != 2 && prm.compact == 0 && params_ok(prm)) {
        std::map<uint32_t, std::vector<size_t>> cand;  // min_count -> libraries that a mixed run can hold
        for (auto &kv : groups)
            if (kv.first.first <= MIXED_K_MAX) cand[kv.first.second].insert(cand[kv.first.second].end(),
                                                                              kv.second.begin(), kv.second.end());
        for (auto &kv : cand)
            if (prm.batch_mixed == 1 || mixed_runs_pay(jobs, kv.second)) {
                mixed[kv.first] = kv.second;
                for (size_t i : kv.second) groups.erase({jobs[i].k, jobs[i].min_count});
            }
    }
    for (auto &kv : mixed) {
        std::vector<size_t> &all = kv.second;
        // libraries in order of k, so that each run's keys of one width come out together
        std::stable_sort(all.begin(), all.end(), [&](size_t a, size_t b) { return jobs[a].k < jobs[b].k; });
        turtle_params gp = prm;
        if (prm.autotune && rc == TURTLE_OK) rc = tune_group(c, jobs, all, prm, s, &gp);
        for (size_t a = 0; a < all.size() && rc == TURTLE_OK; a += 64) {
            std::vector<size_t> idx(all.begin() + a, all.begin() + std::min(all.size(), a + 64));
            rc = batch_run_jobs(c, jobs, idx, &gp, s, outs, bo, nullptr, true);
        }
    }
    for (auto &kv : groups) {
        const size_t per_run = batch_capacity(kv.first.first);
        const std::vector<size_t> &all = kv.second;
        turtle_params gp = prm;
        if (prm.autotune && rc == TURTLE_OK) rc = tune_group(c, jobs, all, prm, s, &gp);
        for (size_t a = 0; a < all.size() && rc == TURTLE_OK; a += per_run) {
            std::vector<size_t> idx(all.begin() + a, all.begin() + std::min(all.size(), a + per_run));
            rc = batch_run_jobs(c, jobs, idx, &gp, s, outs, bo, nullptr);
        }
    }
    const int rc_out = bo.drain();
    if (rc == TURTLE_OK) rc = rc_out;
    if (rc)
        for (size_t i = 0; i < n_jobs; i++) turtle_result_free(&outs[i]);
    return rc;
}

void turtle_trim(void) {
    {
        std::lock_guard<std::mutex> g(g_default_mu);
        for (turtle_ctx *c : g_default) {
            if (!c) continue;
            if (cudaSetDevice(c->device) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            if (c->last_stream) cudaStreamSynchronize(c->last_stream);
            free_list(c->result, c->last_stream);  // the last device result of the host forms is never handed out
            cudaDeviceSynchronize();
            cudaMemPoolTrimTo(c->pool, 0);
            cudaGetLastError();
        }
    }
    std::lock_guard<std::mutex> g(g_rbuf_mu);
    for (auto &kv : g_rbuf_idle) free(kv.second);
    g_rbuf_idle.clear();
    g_rbuf_idle_bytes = 0;
}

int turtle_count(const turtle_reads *reads, int k, uint32_t min_count, turtle_result *out) {
    return turtle_count_ex(reads, k, min_count, nullptr, nullptr, out);
}

void turtle_result_free(turtle_result *r) {
    if (!r) return;
    result_release(r->keys);
    result_release(r->counts);
    r->keys = nullptr;
    r->counts = nullptr;
    r->n = 0;
}

int turtle_extract(turtle_ctx *c, const uint8_t *bases, uint64_t n_bases, const uint64_t *offsets, uint64_t n_reads,
                   int k, void *stream, uint64_t *keys, uint64_t *valid, uint64_t *n_windows) {
    if (!c || k < 1 || k > 64 || !offsets || (n_bases && (!bases || !keys || !valid))) return TURTLE_E_ARG;
    if (!aligned(offsets, 8) || !aligned(keys, k <= 32 ? 8 : 16) || !aligned(valid, 8)) return TURTLE_E_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    try {
        ctx_begin(c, s);
        const LaunchCfg lc{c->sms, s};
        const PackLayout L = PackLayout::of(n_bases);
        uint64_t *P = (uint64_t *)ctx_alloc(c, 8 * L.p_words, s);
        uint64_t *B = (uint64_t *)ctx_alloc(c, 8 * L.b_words, s);
        uint64_t *S = (uint64_t *)ctx_alloc(c, 8 * L.b_words, s);
        uint64_t *V = (uint64_t *)ctx_alloc(c, 8 * L.v_words, s);
        ck(cudaMemsetAsync(S, 0, 8 * L.b_words, s));
        ck(cudaMemsetAsync(V + (L.v_words - 2), 0, 16, s));
        launch_pack(lc, bases, offsets, n_reads, L, P, B, S, c->d_err);
        launch_valid(lc, L, k, B, S, V, c->d_ctr + C_WINDOWS);
        launch_extract(lc, L, k, P, V, keys);
        if (n_bases) ck(cudaMemcpyAsync(valid, V, 8 * ((n_bases + 63) / 64), cudaMemcpyDeviceToDevice, s));
        read_back(c, s);
        if (n_windows) *n_windows = c->h_ctr[C_WINDOWS];
        ctx_end(c, s);
        return TURTLE_OK;
    } catch (Fail f) {
        return fail_code(s, c, f.code);
    }
}

int turtle_filter(turtle_ctx *c, const uint64_t *keys, uint64_t n, int key_words, uint64_t *filter,
                  uint64_t n_sectors, const turtle_params *params, int set, uint8_t *seen, void *stream) {
    if (!c || (key_words != 1 && key_words != 2) || !filter || n_sectors == 0 || (n_sectors & (n_sectors - 1)) ||
        (n && !keys) || (!set && !seen))
        return TURTLE_E_ARG;
    if (!aligned(keys, 8 * key_words) || !aligned(filter, 8)) return TURTLE_E_ARG;
    const turtle_params prm = resolve(params);
    if (!params_ok(prm)) return TURTLE_E_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    try {
        ctx_begin(c, s);
        const LaunchCfg lc{c->sms, s};
        FilterGeom fg{};
        fg.words = filter;
        fg.n_sectors = n_sectors;
        fg.sector_shift = 64 - log2_exact(n_sectors);
        fg.patterns = ctx_patterns(c, prm, s);
        fg.pat_mask = prm.n_patterns - 1;
        if (n) {
            if (key_words == 1) launch_filter_keys<uint64_t>(lc, keys, n, fg, set, seen);
            else launch_filter_keys<Key128>(lc, reinterpret_cast<const Key128 *>(keys), n, fg, set, seen);
        }
        read_back(c, s);
        ctx_end(c, s);
        return TURTLE_OK;
    } catch (Fail f) {
        return fail_code(s, c, f.code);
    }
}

int turtle_sort_compact(turtle_ctx *c, const uint64_t *keys, uint64_t n, int key_words, int key_bits,
                        uint64_t *unique, uint32_t *counts, uint64_t *n_unique, void *stream) {
    if (!c || (key_words != 1 && key_words != 2) || key_bits < 1 || key_bits > 64 * key_words || !n_unique ||
        (n && (!keys || !unique || !counts)))
        return TURTLE_E_ARG;
    if (!aligned(keys, 8) || !aligned(unique, 8 * key_words) || !aligned(counts, 4)) return TURTLE_E_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    try {
        ctx_begin(c, s);
        *n_unique = 0;
        if (n == 0) {
            ctx_end(c, s);
            return TURTLE_OK;
        }
        const LaunchCfg lc{c->sms, s};
        const size_t kb = 8 * key_words;
        void *a = ctx_alloc(c, kb * n, s);
        SortScratch ss{};
        ss.alt = ctx_alloc(c, kb * n, s);
        ss.hist = (uint64_t *)ctx_alloc(c, 8 * 256 * 16, s);
        ss.lookback_words = sort_lookback_words(n, key_words);
        ss.lookback = (uint64_t *)ctx_alloc(c, 8 * ss.lookback_words, s);
        ss.tile_ctr = (uint32_t *)ctx_alloc(c, 4 * 32, s);
        uint64_t *starts = (uint64_t *)ctx_alloc(c, 8 * n, s);
        ck(cudaMemcpyAsync(a, keys, kb * n, cudaMemcpyDeviceToDevice, s));
        if (key_words == 1) {
            uint64_t *sorted = launch_radix_sort<uint64_t>(lc, (uint64_t *)a, n, key_bits, ss, c->d_err);
            launch_rle<uint64_t>(lc, sorted, n, unique, starts, c->d_ctr + C_UNIQUE, ss.lookback, ss.tile_ctr + 20,
                                 c->d_err);
        } else {
            Key128 *sorted = launch_radix_sort<Key128>(lc, (Key128 *)a, n, key_bits, ss, c->d_err);
            launch_rle<Key128>(lc, sorted, n, (Key128 *)unique, starts, c->d_ctr + C_UNIQUE, ss.lookback,
                               ss.tile_ctr + 20, c->d_err);
        }
        launch_run_counts(lc, starts, c->d_ctr + C_UNIQUE, n, n, counts, c->d_err);
        read_back(c, s);
        *n_unique = c->h_ctr[C_UNIQUE];
        ctx_end(c, s);
        return TURTLE_OK;
    } catch (Fail f) {
        return fail_code(s, c, f.code);
    }
}

}  // extern "C"
