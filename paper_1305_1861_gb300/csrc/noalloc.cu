// Allocation-free sort-and-compact: the same radix sort and run-length
// compaction as turtle_sort_compact, with every scratch buffer carved from one
// fixed array that lives in the library's own device image.
//
// Who needs this: code that must not call cudaMalloc / cudaFree (or anything
// that allocates device memory behind its back, such as a caching allocator):
// for example a host program that runs under a strict device-memory budget
// decided up front, a plug-in that is handed a stream by a framework that owns
// all allocations, or a real-time loop where an allocation could block on the
// driver or fail part-way through. Such a caller passes its own input and
// output buffers; this call adds no allocation of any kind.
//
// The price is a fixed footprint: every GPU that loads libturtle keeps
// TURTLE_NOALLOC_SCRATCH_BYTES reserved for the array until the process exits,
// and one call handles at most TURTLE_NOALLOC_MAX_KEYS64 64-bit keys or
// TURTLE_NOALLOC_MAX_KEYS128 128-bit keys.
#include <cstring>
#include <mutex>

#include "turtle.h"
#include "common.cuh"
#include "kernels.h"

using namespace turtle;

namespace {

// Scratch layout (bytes): [ key buffer A | key buffer B | run starts | look-back | histograms | words ]
constexpr uint64_t KEY_BUF = 16ull * TURTLE_NOALLOC_MAX_KEYS128;  // == 8 * TURTLE_NOALLOC_MAX_KEYS64
constexpr uint64_t STARTS = 8ull * TURTLE_NOALLOC_MAX_KEYS64;
constexpr uint64_t LOOKBACK_WORDS = (TURTLE_NOALLOC_MAX_KEYS64 / 4096 + 2) * 256;
constexpr uint64_t OFF_A = 0, OFF_B = OFF_A + KEY_BUF, OFF_STARTS = OFF_B + KEY_BUF;
constexpr uint64_t OFF_LB = OFF_STARTS + STARTS, OFF_HIST = OFF_LB + 8 * LOOKBACK_WORDS;
constexpr uint64_t OFF_WORDS = OFF_HIST + 8 * 256 * 16;  // err word, n_unique counter, tile counters
constexpr uint64_t TOTAL = OFF_WORDS + 256;
static_assert(TOTAL == TURTLE_NOALLOC_SCRATCH_BYTES, "header constant out of date");
static_assert(8ull * TURTLE_NOALLOC_MAX_KEYS64 == 16ull * TURTLE_NOALLOC_MAX_KEYS128, "buffers sized for both widths");

}  // namespace

// File-scope device array: part of the module image, so no allocation call ever creates it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TURTLE_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_setup_mu;
unsigned char *g_scratch_addr[256] = {};  // device address of the array, per device ordinal

// Once per device, with that device current: translate the array's host-side
// symbol into its device address. The host symbol itself must never reach a kernel.
int scratch_for_current_device(unsigned char **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        return TURTLE_E_NODEV;
    }
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return TURTLE_E_CUDA;
        }
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return TURTLE_OK;
}

}  // namespace

extern "C" int turtle_sort_compact_noalloc(const uint64_t *keys, uint64_t n, int key_words, int key_bits,
                                           uint64_t *unique, uint32_t *counts, uint64_t *n_unique, void *stream) {
    if ((key_words != 1 && key_words != 2) || key_bits < 1 || key_bits > 64 * key_words || !n_unique ||
        (n && (!keys || !unique || !counts)))
        return TURTLE_E_ARG;
    // unique is written as whole 8- or 16-byte keys and counts as 4-byte words: a misaligned buffer
    // would fault on the device, so it is refused here, before anything is queued
    if (((uintptr_t)keys & 7) || ((uintptr_t)unique & (8 * key_words - 1)) || ((uintptr_t)counts & 3))
        return TURTLE_E_ARG;
    *n_unique = 0;
    if (n > (key_words == 1 ? (uint64_t)TURTLE_NOALLOC_MAX_KEYS64 : (uint64_t)TURTLE_NOALLOC_MAX_KEYS128))
        return TURTLE_E_TOO_LARGE;
    unsigned char *base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc) return rc;
    if (n == 0) return TURTLE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return TURTLE_E_CUDA;
    }
    const LaunchCfg lc{sms, s};
    uint32_t *err = reinterpret_cast<uint32_t *>(base + OFF_WORDS);
    unsigned long long *nu_dev = reinterpret_cast<unsigned long long *>(base + OFF_WORDS + 8);
    SortScratch ss{};
    ss.alt = base + OFF_B;
    ss.hist = reinterpret_cast<uint64_t *>(base + OFF_HIST);
    ss.lookback = reinterpret_cast<uint64_t *>(base + OFF_LB);
    ss.lookback_words = LOOKBACK_WORDS;
    ss.tile_ctr = reinterpret_cast<uint32_t *>(base + OFF_WORDS + 64);
    uint64_t *starts = reinterpret_cast<uint64_t *>(base + OFF_STARTS);
    // The array keeps whatever the previous call left: clear the error word here; the sorter and the
    // compaction clear their own histograms, tile counters, look-back words and the n_unique counter.
    if (cudaMemsetAsync(err, 0, 4, s) != cudaSuccess ||
        cudaMemcpyAsync(base + OFF_A, keys, 8ull * key_words * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return TURTLE_E_CUDA;
    }
    if (key_words == 1) {
        uint64_t *sorted = launch_radix_sort<uint64_t>(lc, reinterpret_cast<uint64_t *>(base + OFF_A), n, key_bits,
                                                       ss, err);
        launch_rle<uint64_t>(lc, sorted, n, unique, starts, nu_dev, ss.lookback, ss.tile_ctr + 20, err);
    } else {
        Key128 *sorted = launch_radix_sort<Key128>(lc, reinterpret_cast<Key128 *>(base + OFF_A), n, key_bits, ss,
                                                   err);
        launch_rle<Key128>(lc, sorted, n, reinterpret_cast<Key128 *>(unique), starts, nu_dev, ss.lookback,
                           ss.tile_ctr + 20, err);
    }
    launch_run_counts(lc, starts, nu_dev, n, n, counts, err);
    uint64_t words[2] = {0, 0};  // host copies of the error word and n_unique (pageable stack memory)
    if (cudaMemcpyAsync(&words[0], err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&words[1], nu_dev, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return TURTLE_E_CUDA;
    }
    if (words[0] & ERR_COUNT_OVERFLOW) return TURTLE_E_OVERFLOW;
    if (words[0]) return TURTLE_E_DEVICE;
    *n_unique = words[1];
    return TURTLE_OK;
}
