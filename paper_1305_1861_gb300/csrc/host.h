// Host-side helpers shared by the C-ABI translation units (internal; not part of the C ABI).
#pragma once
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "turtle.h"

// Host-memory form of turtle_count (or, with cturtle, turtle_frequent) on a given context
// (copies or streams the reads in).
int count_host_impl(turtle_ctx *c, const turtle_reads *reads, int k, uint32_t min_count, const turtle_params *params,
                    void *stream, turtle_result *out, bool cturtle);

// Upper estimate of the device memory one call needs for n_bases bases (no key-range split):
// the reads, their packed form and bitmaps, and the per-window buffers of the post-filter stages.
uint64_t footprint_estimate(uint64_t n_bases, uint64_t n_reads, int k, uint32_t min_count, const turtle_params *p);

// Copy-out of finished batched runs: tasks run in posting order on one host thread, with their
// own stream, while later runs execute on the GPU.
class BatchOutput {
public:
    BatchOutput();
    ~BatchOutput();  // drains, then stops the thread
    bool ok() const { return stream_ != nullptr; }
    cudaStream_t stream() const { return stream_; }
    void post(std::function<void()> task);
    void fail(int code);  // record the first error of any task
    int drain();          // wait for every posted task; returns the first recorded error
private:
    void loop();
    cudaStream_t stream_ = nullptr;
    std::thread worker_;
    std::mutex mu_;
    std::condition_variable cv_, cv_idle_;
    std::deque<std::function<void()>> tasks_;
    bool stop_ = false, busy_ = false;
    int rc_ = TURTLE_OK;
};

// Libraries one batched run can hold for this k (the key bits above 2k tag the library).
size_t batch_capacity(int k);

// Mixed runs: libraries of different k share a run with 128-bit keys, the library in the top 6 bits.
constexpr int MIXED_TAG_BITS = 6;                     // up to 64 libraries
constexpr int MIXED_K_MAX = 64 - MIXED_TAG_BITS / 2;  // their keys below the tag: 2k <= 122

// Whether jobs[idx[...]] (same min_count, each k <= MIXED_K_MAX) are expected to finish sooner in mixed
// runs than in runs grouped by k (fewer runs, each with a fixed cost, against 128-bit keys for k <= 32).
bool mixed_runs_pay(const turtle_job *jobs, const std::vector<size_t> &idx);

// One batched run: jobs[idx[...]] (same k and min_count, at most batch_capacity(k)) concatenated
// on the device and counted by one pipeline on stream s. On TURTLE_OK the per-library copy-out
// into outs[idx[...]] is posted to bo and done(rc) is called on bo's thread when it finishes;
// on an error nothing is posted and done is not called. mixed: a run of up to 64 libraries with
// different k (each at most 61) and the same min_count, keyed with 128 bits (bucketed form only).
int batch_run_jobs(turtle_ctx *c, const turtle_job *jobs, const std::vector<size_t> &idx, const turtle_params *params,
                   cudaStream_t s, turtle_result *outs, BatchOutput &bo, std::function<void(int)> done,
                   bool mixed = false);

// Autotuner cache: the tuned knobs of (k's key width, min_count >= 2, start.compact, log2 n_bases) merged into
// *best = start, if that class was tuned before.
bool tune_cache_lookup(int k, uint32_t min_count, const turtle_params &start, uint64_t n_bases, turtle_params *best);
