// Autotuner for the knobs that change speed but never the result: the filter's bits per window and
// pattern bits (how full each filter block gets), the onesweep tile shape, the bucket kernel's
// table size and the windows per key-range bucket (how many bucket-index digits the radix passes
// sort by).
//
// Selection is coordinate descent: starting from the caller's params, each knob in turn is set to
// each of its candidate values with the others held, the run is timed, and a value is kept when it
// is faster than the best so far by more than 2% (timing noise). Only measured improvements are
// kept, so the result is never slower, on the run it was measured on, than where it started. The
// device form times turtle_count_device on the caller's library with CUDA events on the call's
// stream (one warm-up, median of three) and caches the result per class of input: key width, with
// or without the filter, the sort-and-compact form and the power of two of the input's bases.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "turtle.h"
#include "host.h"

namespace {

struct Knob {
    void (*set)(turtle_params &, double);
    double (*get)(const turtle_params &);
    std::vector<double> values;
};

const std::vector<Knob> &knobs() {
    static const std::vector<Knob> k = {
        {[](turtle_params &p, double v) { p.filter_bits_per_window = (float)v; },
         [](const turtle_params &p) { return (double)p.filter_bits_per_window; }, {1.0, 0.5, 2.0}},
        {[](turtle_params &p, double v) { p.pattern_bits = (uint32_t)v; },
         [](const turtle_params &p) { return (double)p.pattern_bits; }, {4, 3, 6}},
        {[](turtle_params &p, double v) { p.sort_tile = (uint32_t)v; },
         [](const turtle_params &p) { return (double)p.sort_tile; }, {0, 2, 3}},
        {[](turtle_params &p, double v) { p.bucket_slots = (uint32_t)v; },
         [](const turtle_params &p) { return (double)p.bucket_slots; }, {0, 4096}},
        {[](turtle_params &p, double v) { p.bucket_windows = (uint32_t)v; },
         [](const turtle_params &p) { return (double)(p.bucket_windows ? p.bucket_windows : 16384); },
         {16384, 8192, 32768}},
    };
    return k;
}

constexpr double KEEP_GAIN = 0.98;  // a candidate must beat the best time so far by 2%
constexpr int CONFIRM = 3;          // interleaved re-timings of the start and the choice

std::mutex g_cache_mu;
// (key words, filter on, compact form, log2 bases) -> tuned params
std::map<std::tuple<int, int, uint32_t, int>, turtle_params> g_cache;

struct DeviceRun {
    turtle_ctx *ctx;
    const uint8_t *bases;
    uint64_t n_bases;
    const uint64_t *offsets;
    uint64_t n_reads;
    int k;
    uint32_t min_count;
    cudaStream_t stream;
    cudaEvent_t ev[2];
};

// Median of three timed runs after one warm-up, in ms; -1 when the run fails.
double device_timer(const turtle_params *p, void *user) {
    DeviceRun *r = static_cast<DeviceRun *>(user);
    turtle_device_result out;
    turtle_params q = *p;
    q.timing = 0;
    if (turtle_count_device(r->ctx, r->bases, r->n_bases, r->offsets, r->n_reads, r->k, r->min_count, &q, r->stream,
                            &out))
        return -1.0;
    float t[3];
    for (float &x : t) {
        if (cudaEventRecord(r->ev[0], r->stream) != cudaSuccess) return -1.0;
        if (turtle_count_device(r->ctx, r->bases, r->n_bases, r->offsets, r->n_reads, r->k, r->min_count, &q,
                                r->stream, &out))
            return -1.0;
        if (cudaEventRecord(r->ev[1], r->stream) != cudaSuccess || cudaEventSynchronize(r->ev[1]) != cudaSuccess ||
            cudaEventElapsedTime(&x, r->ev[0], r->ev[1]) != cudaSuccess)
            return -1.0;
    }
    std::sort(t, t + 3);
    return t[1];
}

int log2_floor(uint64_t x) {
    int b = 0;
    while (x >> (b + 1)) b++;
    return b;
}

}  // namespace

extern "C" {

int turtle_tune_select(const turtle_params *base, turtle_tune_timer timer, void *user, turtle_params *best,
                       turtle_tune_report *rep) {
    if (!base || !timer || !best || base->struct_size != sizeof(turtle_params)) return TURTLE_E_ARG;
    turtle_tune_report r{};
    turtle_params cur = *base;
    double t0 = timer(&cur, user);
    r.evaluations = 1;
    if (t0 < 0) return TURTLE_E_DEVICE;
    double best_t = t0;
    for (const Knob &kn : knobs()) {
        const double now = kn.get(cur);
        for (double v : kn.values) {
            if (v == now) continue;
            turtle_params cand = cur;
            kn.set(cand, v);
            const double t = timer(&cand, user);
            r.evaluations++;
            if (t >= 0 && t < best_t * KEEP_GAIN) {
                best_t = t;
                cur = cand;
            }
        }
    }
    // A changed choice is confirmed against the start by interleaved re-timings (start, choice, start,
    // choice, ...): it is kept only if its median still wins by the same margin, so one lucky timing
    // during the sweep cannot select it.
    bool changed = false;
    for (const Knob &kn : knobs()) changed |= kn.get(cur) != kn.get(*base);
    if (changed) {
        double ts[CONFIRM], tc[CONFIRM];
        for (int i = 0; i < CONFIRM; i++) {
            ts[i] = timer(base, user);
            tc[i] = timer(&cur, user);
            r.evaluations += 2;
        }
        std::sort(ts, ts + CONFIRM);
        std::sort(tc, tc + CONFIRM);
        const double ms = ts[CONFIRM / 2], mc = tc[CONFIRM / 2];
        if (mc >= 0 && ms >= 0 && mc < ms * KEEP_GAIN) {
            best_t = mc;
            t0 = ms;
        } else {
            cur = *base;
            best_t = t0 = ms >= 0 ? ms : t0;
        }
    }
    *best = cur;
    r.default_ms = (float)t0;
    r.best_ms = (float)best_t;
    if (rep) *rep = r;
    return TURTLE_OK;
}

}  // extern "C"

bool tune_cache_lookup(int k, uint32_t min_count, const turtle_params &start, uint64_t n_bases, turtle_params *best) {
    const auto key = std::make_tuple(k <= 32 ? 1 : 2, min_count >= 2 ? 1 : 0, start.compact,
                                     log2_floor(n_bases ? n_bases : 1));
    std::lock_guard<std::mutex> g(g_cache_mu);
    auto it = g_cache.find(key);
    if (it == g_cache.end()) return false;
    *best = start;  // the caller's other settings, with the tuned knobs of this class
    best->filter_bits_per_window = it->second.filter_bits_per_window;
    best->pattern_bits = it->second.pattern_bits;
    best->sort_tile = it->second.sort_tile;
    best->bucket_slots = it->second.bucket_slots;
    best->bucket_windows = it->second.bucket_windows;
    return true;
}

extern "C" {

int turtle_autotune(turtle_ctx *ctx, const uint8_t *bases, uint64_t n_bases, const uint64_t *offsets,
                    uint64_t n_reads, int k, uint32_t min_count, const turtle_params *base, void *stream,
                    turtle_params *best, turtle_tune_report *rep) {
    if (!ctx || !best || k < 1 || k > 64 || min_count < 1 || !offsets || (n_bases && !bases)) return TURTLE_E_ARG;
    turtle_params start;
    turtle_params_default(&start);
    if (base) {
        if (base->struct_size != sizeof(turtle_params)) return TURTLE_E_ARG;
        start = *base;
    }
    const auto key = std::make_tuple(k <= 32 ? 1 : 2, min_count >= 2 ? 1 : 0, start.compact,
                                     log2_floor(n_bases ? n_bases : 1));
    if (tune_cache_lookup(k, min_count, start, n_bases, best)) {
        if (rep) {
            memset(rep, 0, sizeof(*rep));
            rep->cached = 1;
        }
        return TURTLE_OK;
    }
    DeviceRun run{ctx, bases, n_bases, offsets, n_reads, k, min_count, (cudaStream_t)stream, {nullptr, nullptr}};
    if (cudaEventCreate(&run.ev[0]) != cudaSuccess || cudaEventCreate(&run.ev[1]) != cudaSuccess) {
        cudaGetLastError();
        if (run.ev[0]) cudaEventDestroy(run.ev[0]);
        return TURTLE_E_CUDA;
    }
    turtle_tune_report r{};
    const int rc = turtle_tune_select(&start, device_timer, &run, best, &r);
    cudaEventDestroy(run.ev[0]);
    cudaEventDestroy(run.ev[1]);
    cudaGetLastError();
    if (rc) return rc;
    r.sample_bases = n_bases;
    if (rep) *rep = r;
    std::lock_guard<std::mutex> g(g_cache_mu);
    g_cache[key] = *best;
    return TURTLE_OK;
}

void turtle_tune_cache_clear(void) {
    std::lock_guard<std::mutex> g(g_cache_mu);
    g_cache.clear();
}

}  // extern "C"
