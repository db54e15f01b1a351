/*
 * libturtle: frequent canonical k-mer counting on one GB300 GPU (sm_103a).
 *
 * Method: Turtle (Roy, Bhattacharya & Schliep, arXiv:1305.1861). Given a read
 * library and k <= 64, report every canonical k-mer seen at least min_count
 * times, with its exact count, in ascending key order:
 *   - a k-mer and its reverse complement are one object (Sec. 2.1.1);
 *   - k-mers are taken from reads split at ambiguous calls, 2 bits per base,
 *     and represented by the numerically smaller of the k-mer and its reverse
 *     complement (Sec. 2.1.2);
 *   - a pattern-blocked Bloom filter drops first sightings (Sec. 2.1.3);
 *   - the survivors are sorted and compacted (Sec. 2.1.4, Alg. 1);
 *   - an exact second pass recounts every occurrence of each survivor, so the
 *     result is exact and independent of atomic ordering and of Bloom false
 *     positives (the paper instead adds 1 to each count, Sec. 2.1.4).
 *
 * Conventions shared by every call:
 *   Reads      read i is bases[offsets[i] .. offsets[i+1]); offsets has n_reads+1
 *              non-decreasing entries. Bytes other than A/C/G/T/a/c/g/t are
 *              ambiguous calls: windows containing them are skipped. Bytes
 *              outside [offsets[0], offsets[n_reads]) belong to no read.
 *   Encoding   A=0, C=1, G=2, T=3; the first base of a window is the most
 *              significant 2-bit digit of the low 2k bits; complement is 3-x.
 *   Keys       k <= 32: one uint64 per key. 33 <= k <= 64: two uint64 per key,
 *              high word first ({hi, lo}). Keys ascend as unsigned integers.
 *   Counts     uint32. A count that would pass 2^32-2 fails the call with
 *              TURTLE_E_OVERFLOW.
 *   Errors     every int-returning call returns TURTLE_OK (0) or a negative
 *              TURTLE_E_* code and never throws or aborts. On error, outputs
 *              hold nothing that needs freeing.
 *   Streams    `stream` is a cudaStream_t passed as void* (NULL = legacy
 *              default stream). Calls are stream-ordered; calls that return
 *              host-visible results synchronise the stream before returning.
 *   Threads    a turtle_ctx is used by one host thread at a time; distinct
 *              contexts may be used concurrently.
 */
#ifndef TURTLE_H
#define TURTLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TURTLE_OK 0
#define TURTLE_E_ARG (-1)       /* invalid argument (k outside 1..64, min_count 0, NULL, bad offsets) */
#define TURTLE_E_NOMEM (-2)     /* device or host allocation failed */
#define TURTLE_E_CUDA (-3)      /* a CUDA runtime call failed */
#define TURTLE_E_OVERFLOW (-4)  /* a count would not fit in uint32 */
#define TURTLE_E_TIMEOUT (-5)   /* turtle_poll: the job did not finish in time */
#define TURTLE_E_BUSY (-6)      /* turtle_submit: the job does not fit the server's HBM budget */
#define TURTLE_E_DEVICE (-7)    /* a device-side check failed (bounded wait expired, table full) */
#define TURTLE_E_NODEV (-8)     /* no CUDA device is visible */
#define TURTLE_E_CAPACITY (-9)  /* an output buffer is too small */
#define TURTLE_E_TOO_LARGE (-10) /* input exceeds the fixed scratch of turtle_sort_compact_noalloc */

/* ------------------------------------------------------------------ params */
/* Tuning knobs. None of them changes the result, only speed and memory. */
typedef struct {
    uint32_t struct_size;          /* sizeof(turtle_params); set by turtle_params_default */
    float filter_bits_per_window;  /* Bloom filter bits per valid window (rounded up to a power of two
                                      number of 32-byte sectors); default 1: a small filter stays partly
                                      in L2, and the few extra false-positive candidates cost less
                                      than the DRAM lines a larger filter's probes would move */
    uint32_t pattern_bits;         /* bits per precomputed pattern (1..64); default 4 */
    uint32_t n_patterns;           /* pattern-table entries, power of two, 1..4096; default 1024 */
    uint64_t pattern_seed;         /* SplitMix64 seed of the pattern table */
    uint32_t timing;               /* 1: record per-stage CUDA events (see turtle_stats) */
    uint32_t l2_fetch_bytes;       /* L2 fetch granularity hint for the call (cudaLimitMaxL2FetchGranularity:
                                      32..128; 0 = leave the context's setting). It is a context-wide
                                      limit: set at the start of a call and restored before it returns. */
    uint32_t recount_windows;      /* exact recount (step a5) by: 0 = first sightings (default): each key's
                                      count is its run length among the sorted candidates plus 1 if one of
                                      its windows was a first sighting, found by probing the recount table
                                      with the first-sighting keys only; 1 = re-extracting every window and
                                      counting it in the table. Both are exact. */
    uint32_t member_filter;        /* 1: screen first-sighting keys with a small membership bitmap of the
                                      candidates before probing the recount table (default 0: probe all) */
    uint32_t budget_mib;           /* device-memory budget (MiB) for one super-partition's working set;
                                      0 = 80% of the free memory at the start of the call. Inputs whose
                                      working set exceeds it are processed in consecutive key ranges. */
    uint32_t stream_chunk_mib;     /* host-memory calls: n > 0 streams the reads to the device in chunks of
                                      n MiB through two device staging buffers, packing each chunk as it
                                      lands (the ASCII is never resident whole); 0 = automatic: reads larger
                                      than a quarter of the free device memory stream in 1 GiB chunks;
                                      otherwise reads of 64 MiB or more (bucketed form, one key range) are
                                      copied in chunks that overlap pass 1, and smaller ones at once. Every
                                      copy reads the caller's memory directly, pageable or page-locked. */
    uint32_t sort_tile;            /* onesweep tile shape (256 threads): 0 = default (global sort: 32 keys per
                                      thread, 16 for 128-bit keys, 2 CTAs/SM; bucket sort: 16, 4 CTAs/SM for
                                      64-bit keys, 16, 2 CTAs/SM for 128-bit keys);
                                      1 = 16, 4/SM (8, 3/SM); 2 = 24 (12), 2/SM; 3 = 32 (16), 2/SM;
                                      4 = persistent, 16 (8), 2/SM: each CTA's next tile is bulk-copied
                                      (cp.async.bulk) into shared memory while it sorts the current one */
    uint32_t compact;              /* form of sort-and-compact (step a4, with a5 and a6): 0 = bucketed
                                      (default): one MSD radix pass moves candidates and first sightings
                                      into key-range buckets; per bucket, in shared memory, duplicates are
                                      merged into run lengths, first sightings add one, counts below
                                      min_count are dropped and the rest sorted. 1 = global: LSD radix sort
                                      of all candidates, run-length compaction, recount table, threshold.
                                      2 = hash table (the hash-table side of Table 1): candidates are
                                      counted in an open-addressing table sized from a HyperLogLog
                                      estimate of their distinct keys, first sightings add one, the keys
                                      whose count reaches min_count are extracted and radix-sorted.
                                      3 = lazy sort-and-compact phases (Sec. 2.1.4, Alg. 1), the
                                      memory-capped form: the reads are taken in chunks of window tiles
                                      through one shared filter; each chunk's candidates are sorted and
                                      compacted on their own and merged (merge path) into a running
                                      sorted array of distinct candidates with counts; then the second
                                      pass re-extracts every window and counts it in a table of those
                                      keys. Memory: the packed reads, the filter, the running array
                                      twice and one chunk, whose size follows budget_mib.
                                      All four are exact. recount_windows = 1 uses the global form
                                      (0) or is ignored (2: first sightings; 3: always window recount). */
    uint32_t bucket_slots;         /* bucketed form: shared-memory table of one bucket CTA: 0 or 8192 =
                                      8192 slots (1024 threads, one CTA per SM; default), 4096 = 4096 slots
                                      (512 threads, two CTAs per SM; half the distinct keys per bucket
                                      before a bucket is split) */
    uint32_t cturtle_bits_per_window; /* turtle_frequent: bits of its two-stage filter per valid window
                                         (rounded up to a power of two of 32-byte sectors); 0 = 8. Its
                                         false-positive and false-negative rates fall as this grows. */
    uint32_t hash_slots_log2;      /* compact = 2: 0 = size the table from the distinct-key estimate (load
                                      at most 1/2); n = start with 2^n slots. A table in which a key finds
                                      no free slot within 32 lines is doubled and the counting redone. */
    uint32_t shard_count;          /* key-range shards (the paper's routing of k-mers by key to consumers,
                                      Sec. 2.1.5, across processes or GPUs): 0 or 1 = the whole key space;
                                      n in 2..TURTLE_PARTS = the call counts only the keys of shard
                                      shard_index, one of n consecutive key ranges balanced by window
                                      counts (see turtle_shard_bounds). Every shard reads all the reads;
                                      concatenating shards 0 .. n-1 in order gives the whole result. Not
                                      with compact = 3 or the batched form (TURTLE_E_ARG). */
    uint32_t shard_index;          /* 0 .. shard_count - 1 */
    uint32_t probe_order;          /* pass 1 with a filter, bucketed form (compact = 0), one library: 0 = in window
                                      order (default); 1 = by filter block: the windows are first binned by the
                                      top 8 bits of their hash, i.e. by the 1/256 of the filter their block lies
                                      in, and then probed bin after bin, so the blocks being probed stay in L2.
                                      The result is the same either way; on GB300 the window order is faster
                                      (the binning passes cost more than the DRAM misses they save). */
    uint32_t bucket_windows;       /* bucketed form: windows per key-range bucket, about (sets how many bucket-
                                      index digits the radix passes sort by); 0 = 16384, else 1024 .. 2^20 */
    uint32_t autotune;             /* turtle_count_batch: 1 = run each group of libraries (same k and min_count)
                                      with knobs chosen by turtle_autotune on its largest library (tuned once
                                      per class of input, then cached); 0 = as given */
    uint32_t host_transfer;        /* host-memory calls: how the caller's reads and the result arrays (those
                                      of 16 MiB or more) move between host and device. 0 = automatic: each
                                      context measures once how fast page-locking (cudaHostRegister) runs, and
                                      when it costs little (100 GB/s or more, as on Grace) the arrays' whole
                                      pages are page-locked for their copies: pageable copies of large arrays
                                      vary from run to run and box to box (8 to 190 GB/s measured), locked ones
                                      run at 170-210 GB/s; 1 = always page-lock them; 2 = copy pageable
                                      memory directly. Memory the caller locked already is used as it is. */
    uint32_t batch_mixed;          /* turtle_count_batch, bucketed form (compact = 0): libraries with different k
                                      (each at most 61) and the same min_count in one run, keyed with 128 bits
                                      and tagged in the top 6: fewer runs (each has a fixed cost), but 128-bit
                                      work for libraries with k <= 32. 0 = when a cost model expects it to be
                                      faster (many small libraries over several k), 1 = always, 2 = never
                                      (one run per k, as many libraries as its key bits can tag). */
} turtle_params;

/* Fill *p with the defaults above. */
void turtle_params_default(turtle_params *p);

/* Key-range parts: the canonical key's top 31 bits v (of its 2k bits) map to f(v) = v (2^32 - v),
 * which is increasing in v and splits the canonical keys of random sequence into about equal
 * numbers; part p of TURTLE_PARTS holds the keys with f(v) >> 56 == p, so parts are consecutive key
 * ranges in ascending order. Super-partitions (budget_mib) and shards are unions of parts. */
#define TURTLE_PARTS 64

/*
 * Shard bounds (host only, no device): given the valid windows of each of the n_parts key-range parts
 * (part_windows[0 .. n_parts)), split the parts into n_shards consecutive ranges of about equal
 * windows: shard s takes parts [bounds[s], bounds[s+1]); bounds has n_shards + 1 entries, bounds[0] = 0,
 * bounds[n_shards] = n_parts, non-decreasing; bounds[s] is the first part p at which the windows of
 * parts below p reach s/n_shards of all windows. A shard may be empty. TURTLE_E_ARG for NULL
 * pointers, n_parts = 0 or n_shards = 0.
 */
int turtle_shard_bounds(const uint64_t *part_windows, uint32_t n_parts, uint32_t n_shards, uint32_t *bounds);

/* ------------------------------------------------------------------ host-memory form */
typedef struct {
    const char *bases;        /* host, caller-owned */
    const uint64_t *offsets;  /* host, n_reads + 1 entries */
    uint64_t n_reads;
} turtle_reads;

typedef struct {
    int k;
    uint64_t n;          /* reported pairs */
    uint64_t *keys;      /* host, library-allocated: n (k <= 32) or 2n (k > 32) words */
    uint32_t *counts;    /* host, library-allocated: n */
    uint64_t n_windows;  /* valid windows processed */
} turtle_result;

/*
 * Count the canonical k-mers of `reads` (host memory) with count >= min_count.
 * Copies the reads to the device, runs the whole path there and copies the
 * result back into library-allocated host arrays owned by *out (free with
 * turtle_result_free). Uses an internal context on the current device.
 * min_count == 1 reports every k-mer (the Bloom filter is skipped).
 */
int turtle_count(const turtle_reads *reads, int k, uint32_t min_count, turtle_result *out);

/* As turtle_count, with explicit params (NULL = defaults) and stream. */
int turtle_count_ex(const turtle_reads *reads, int k, uint32_t min_count, const turtle_params *params,
                    void *stream, turtle_result *out);

/* Free the arrays of a turtle_result (safe on a zeroed or already freed result). The library
 * keeps recently freed result arrays (up to 8 GiB in all) and hands them out again for later
 * results of a similar size: their pages already exist, so the device fills them without first
 * faulting every page in. */
void turtle_result_free(turtle_result *r);

/* Static description of an error code. */
const char *turtle_strerror(int code);

/* Give back what the library keeps between calls of its host-memory and batched forms: the device
 * memory that the internal per-device contexts' pools hold unused, and the recycled host result
 * arrays. Later calls allocate again as needed. Waits for those contexts' work. Contexts created
 * with turtle_ctx_create are not touched (turtle_ctx_destroy releases theirs). */
void turtle_trim(void);

/* ------------------------------------------------------------------ contexts and the device form */
/* A context owns device scratch (a memory pool grown on demand and kept between calls: its idle
 * memory counts as free for the context's own budget; turtle_ctx_trim gives it back), the device
 * result of its last call, an error word and timing events. */
typedef struct turtle_ctx turtle_ctx;

/* Create a context on CUDA device `device`. */
int turtle_ctx_create(int device, turtle_ctx **ctx);
/* Destroy a context and free its device memory (synchronises its last stream). */
void turtle_ctx_destroy(turtle_ctx *ctx);

typedef struct {
    int k;
    int key_words;           /* 1 or 2 */
    uint64_t n;              /* reported pairs */
    const uint64_t *keys;    /* DEVICE, owned by the context, valid until its next call */
    const uint32_t *counts;  /* DEVICE, same ownership */
    uint64_t n_windows;
} turtle_device_result;

/*
 * Device-resident form: bases (n_bases bytes) and offsets (n_reads + 1 entries)
 * are DEVICE pointers, caller-owned, left unchanged. The result stays on the
 * device in context-owned memory (*out describes it). Synchronises `stream`.
 */
int turtle_count_device(turtle_ctx *ctx, const uint8_t *bases, uint64_t n_bases, const uint64_t *offsets,
                        uint64_t n_reads, int k, uint32_t min_count, const turtle_params *params, void *stream,
                        turtle_device_result *out);

/*
 * cTurtle (Sec. 2.2 of the paper): the k-mers seen at least twice, without counts, from a
 * two-stage counting pattern-blocked Bloom filter in one pass over the windows. A key's
 * first sighting sets its pattern in its block; a later sighting that finds that pattern
 * complete tests and sets a second pattern in the adjacent block, and the sighting that
 * completes the second pattern reports the key (each key at most once). Approximate, as in
 * the paper: a singleton whose first pattern other keys have completed is reported (false
 * positive); a repeated key whose second pattern other keys have completed is not (false
 * negative); which colliding keys these are depends on the order the GPU takes the windows
 * in. Keys come out ascending; the result's counts pointer is NULL. Memory: the filter
 * (params.cturtle_bits_per_window) plus room for the reported keys (one key per valid window,
 * at most 40% of the free device memory; TURTLE_E_CAPACITY if more keys are reported).
 */
int turtle_frequent(const turtle_reads *reads, int k, const turtle_params *params, void *stream,
                    turtle_result *out);
/* Device-resident form of turtle_frequent (arguments as turtle_count_device; out->counts NULL). */
int turtle_frequent_device(turtle_ctx *ctx, const uint8_t *bases, uint64_t n_bases, const uint64_t *offsets,
                           uint64_t n_reads, int k, const turtle_params *params, void *stream,
                           turtle_device_result *out);

/* Stages of one turtle_count_device call, in launch order. */
enum {
    TURTLE_STAGE_PACK = 0,      /* ASCII -> 2-bit codes, ambiguous-call and read-start bitmaps */
    TURTLE_STAGE_VALID,         /* valid-window bitmap and window count */
    TURTLE_STAGE_FILTER,        /* pass 1: extraction + Bloom test-and-set + candidate emission */
    TURTLE_STAGE_HIST,          /* radix sort: digit histograms of all passes + scan */
    TURTLE_STAGE_SORT,          /* radix sort: onesweep digit passes */
    TURTLE_STAGE_RLE,           /* run-length compaction of sorted candidates */
    TURTLE_STAGE_TABLE,         /* insert unique candidates into the recount table */
    TURTLE_STAGE_RECOUNT,       /* exact recount: first sightings, or pass 2 over every window */
    TURTLE_STAGE_THRESHOLD,     /* keep count >= min_count in key order */
    TURTLE_STAGE_MERGE,         /* lazy form (compact = 3): merge a chunk's compacted keys into the running set */
    TURTLE_STAGE_COUNT
};

/* Where the wall time of a host-memory call (turtle_ctx_count) went, in call order. */
enum {
    TURTLE_HOST_INPUT = 0,  /* device buffers for the reads, their offsets copied, and the reads' copy queued
                               (when it overlaps pass 1 it runs inside TURTLE_HOST_PATH) */
    TURTLE_HOST_PATH,       /* the device path, until the result is complete in device memory */
    TURTLE_HOST_TOUCH,      /* first touch of host result pages that did not exist yet */
    TURTLE_HOST_OUTPUT,     /* the result's copy from device to host memory */
    TURTLE_HOST_COUNT
};

typedef struct {
    uint64_t n_windows, n_candidates, n_firsts, n_unique, n_out;
    uint64_t filter_bytes, table_bytes, scratch_bytes;
    uint32_t sort_passes;                       /* LSD digit passes run (8-bit digits), last super-partition */
    uint32_t super_partitions;                  /* key ranges the call was split into (1 = none) */
    uint32_t launches;                          /* kernels launched by the last call */
    uint32_t stage_launches[TURTLE_STAGE_COUNT];
    float stage_ms[TURTLE_STAGE_COUNT];         /* CUDA-event time per stage (params->timing) */
    float host_ms[TURTLE_HOST_COUNT];           /* host-memory calls: wall time per phase (always recorded) */
    float h2d_ms;                               /* host-memory calls: CUDA-event span of the reads' copy to
                                                   the device, first byte queued to last byte landed */
    uint64_t h2d_bytes, d2h_bytes;              /* host-memory calls: bytes copied in and out */
    uint32_t chunks;                            /* lazy form (compact = 3): read chunks merged into the
                                                   running set (0 in the other forms) */
    uint32_t host_locked;                       /* host-memory calls: 1 if the call page-locked the caller's
                                                   reads for their copy (params.host_transfer) */
    float transfer_gbs[3];                      /* this context's measured host transfer rates (GB/s): pageable
                                                   copy, page-locking, copy from page-locked memory (0 = not
                                                   measured) */
    uint32_t pad_;
} turtle_stats;

/* Statistics of the context's last successful call. */
int turtle_ctx_stats(const turtle_ctx *ctx, turtle_stats *st);

/* Give back to the device the memory the context's pool keeps unused between calls (its last
 * device result stays valid). Waits for the context's work. */
void turtle_ctx_trim(turtle_ctx *ctx);

/* Device memory of the context's pool: *used = bytes held by live buffers (the last call's device
 * result, between calls), *reserved = bytes the pool keeps from the driver for later calls. After a
 * failed call, used returns to what it was before the call. Either pointer may be NULL. */
int turtle_ctx_pool_bytes(const turtle_ctx *ctx, uint64_t *used, uint64_t *reserved);

/* Host-memory form on a caller-owned context: as turtle_count_ex (reads in host memory, result in
 * library-allocated host arrays owned by *out, free with turtle_result_free), run on `ctx`, whose
 * statistics then also hold the host-side phases (host_ms, h2d_ms, h2d_bytes, d2h_bytes). */
int turtle_ctx_count(turtle_ctx *ctx, const turtle_reads *reads, int k, uint32_t min_count,
                     const turtle_params *params, void *stream, turtle_result *out);
/* Name of a stage ("pack", "valid", "filter", ...). */
const char *turtle_stage_name(int stage);

/* ------------------------------------------------------------------ per-step entry points
 * Each runs one step of the path on caller-owned DEVICE buffers, for step-wise
 * checking and reuse. All are stream-ordered and synchronise `stream`.
 * Alignment: buffers of keys are read and written as whole keys, so they must be
 * aligned to the key width (8 bytes for 64-bit keys, 16 bytes for 128-bit keys);
 * offsets, bitmaps and filter words to 8 bytes; counts to 4 bytes. A misaligned
 * buffer returns TURTLE_E_ARG before any work is queued. (turtle_count_device
 * needs offsets aligned to 8 bytes; its bases may start at any byte.)
 */

/*
 * Steps a1-a2 (Sec. 2.1.2): canonical key of every window start. For every
 * position s in [0, n_bases): valid bit s (bit s&63 of valid[s>>6]) is 1 iff
 * bases[s .. s+k) lies inside one read and holds no ambiguous call; then
 * keys[s*key_words ..] is its canonical key (other entries are unspecified).
 * keys: n_bases * key_words uint64; valid: ceil(n_bases/64) uint64.
 * *n_windows receives the number of valid windows.
 */
int turtle_extract(turtle_ctx *ctx, const uint8_t *bases, uint64_t n_bases, const uint64_t *offsets,
                   uint64_t n_reads, int k, void *stream, uint64_t *keys, uint64_t *valid, uint64_t *n_windows);

/*
 * Step a3 (Sec. 2.1.3): pattern-blocked Bloom filter on caller-owned filter
 * words (4 * n_sectors uint64; n_sectors a power of two; zero it to start).
 * Block = one 32-byte sector chosen by the top bits of fmix64(key) (128-bit
 * keys: fmix64(lo ^ fmix64(hi))); the pattern (params->pattern_bits bits from a
 * SplitMix64 table seeded by params->pattern_seed, entry = low bits of the hash)
 * lies in the 64-bit word (hash >> 16) & 3 of the sector.
 * set != 0: test-and-set, seen[i] = 1 iff every pattern bit was already set
 * when key i's single atomicOr ran (order among concurrent keys unspecified).
 * set == 0: membership test only. seen: n bytes (may be NULL when set != 0).
 */
int turtle_filter(turtle_ctx *ctx, const uint64_t *keys, uint64_t n, int key_words, uint64_t *filter,
                  uint64_t n_sectors, const turtle_params *params, int set, uint8_t *seen, void *stream);

/*
 * Step a4 (Sec. 2.1.4): sort-and-compact. Sorts n keys (onesweep LSD radix
 * sort, 8-bit digits, over the low key_bits bits; key_bits = 2k) and writes the
 * distinct keys ascending to unique (capacity n keys) with their run lengths to
 * counts (uint32). keys is not modified. *n_unique receives the distinct count.
 * Scratch comes from the context.
 */
int turtle_sort_compact(turtle_ctx *ctx, const uint64_t *keys, uint64_t n, int key_words, int key_bits,
                        uint64_t *unique, uint32_t *counts, uint64_t *n_unique, void *stream);

/* ------------------------------------------------------------------ served form
 * A request loop for many counting jobs (continuous batching). Jobs queue in arrival order;
 * whenever an executor is free, the oldest job is admitted together with every queued job of
 * the same k and min_count whose device-memory footprint estimate still fits the HBM budget
 * (at most max_batch of them, and at most as many as turtle_count_batch puts in one run), and
 * they run as one batched pipeline on that executor's stream. Runs of different executors are on
 * the device at the same time; a finished run's results are copied to the host while its
 * executor's next run executes. Each result equals turtle_count on the same reads. Reads stay in
 * caller-owned host memory until the job's poll returns.
 */
typedef struct turtle_server turtle_server;

typedef struct {
    const char *bases;        /* host, caller-owned, valid until turtle_poll returns the result */
    const uint64_t *offsets;  /* host, n_reads + 1 entries */
    uint64_t n_reads;
    int k;
    uint32_t min_count;
} turtle_job;

/*
 * Batched form: count many libraries (jobs, host memory) with one pipeline per group
 * instead of one per library. Libraries with the same k and min_count are concatenated
 * on the device and every window's key carries its library index in the key bits above
 * 2k, so each stage is one launch for the whole group and libraries never mix; a group
 * holds up to 64 libraries (fewer when 2k leaves less room: k = 31 takes 4 per run,
 * k = 32 and k = 64 one). With params->batch_mixed, libraries of different k (at most 61)
 * and the same min_count can share a run instead: 128-bit keys, the library in the top 6
 * bits, up to 64 libraries per run. outs[i] receives job i's result, identical to
 * turtle_count on that job (free each with turtle_result_free). Uses the internal context
 * of the current device.
 */
int turtle_count_batch(const turtle_job *jobs, size_t n_jobs, const turtle_params *params, void *stream,
                       turtle_result *outs);

typedef struct {
    double queue_ms;  /* submit -> admitted */
    double run_ms;    /* admitted -> result ready */
    double total_ms;  /* submit -> result ready */
    double start_ms, end_ms;  /* admission and completion on one steady clock (ms): jobs of different
                                 runs whose [start, end) intervals intersect ran at the same time */
} turtle_job_times;

typedef struct {
    uint64_t budget_bytes, admitted_bytes, peak_admitted_bytes;
    uint64_t submitted, completed, failed, queued, running, peak_running, peak_queued;
    uint64_t batches, largest_batch;  /* batched runs started; most jobs in one run */
    uint64_t executors;               /* runs that can be on the device at once */
    uint64_t peak_running_batches;    /* most runs whose device work was in progress at the same time */
} turtle_server_stats;

/* Start a server on `device` with 2 executors (turtle_server_create_ex). */
int turtle_server_create(int device, uint64_t hbm_budget_bytes, int max_batch, const turtle_params *params,
                         turtle_server **server);
/* Start a server on `device`: up to max_batch jobs (1..64) share one run (1 = every job alone),
 * and up to `executors` runs (1..16) are on the device at once, each executor with its own
 * context, stream and copy-out thread, all admitting from one queue (oldest job first) within one
 * HBM budget: a run is admitted only while the footprint estimates of every admitted job fit
 * hbm_budget_bytes (0 = half of the free device memory). executors = 1 runs one batch at a time.
 * params may be NULL. */
int turtle_server_create_ex(int device, uint64_t hbm_budget_bytes, int max_batch, int executors,
                            const turtle_params *params, turtle_server **server);
/* Queue a job; *ticket identifies it. TURTLE_E_BUSY: its footprint estimate exceeds the whole
 * budget, so it could never be admitted. */
int turtle_submit(turtle_server *server, const turtle_job *job, uint64_t *ticket);
/* Wait up to timeout_ms (< 0: forever) for a job. On completion fills *out (free with
 * turtle_result_free), optionally *times, forgets the ticket and returns the job's status;
 * TURTLE_E_TIMEOUT if it is not done yet (the ticket stays valid); TURTLE_E_ARG for an
 * unknown ticket. */
int turtle_poll(turtle_server *server, uint64_t ticket, int timeout_ms, turtle_result *out, turtle_job_times *times);
int turtle_server_stats_get(turtle_server *server, turtle_server_stats *stats);
/* Stop accepting work, let running jobs finish, drop queued ones, free everything. */
void turtle_server_destroy(turtle_server *server);

/* ------------------------------------------------------------------ autotuner
 * Chooses the knobs that change speed but not the result -- filter bits per window and pattern bits
 * (the filter block's fill), the onesweep tile shape (sort_tile), the bucket kernel's table size
 * (bucket_slots) and the windows per bucket (bucket_windows: how many bucket-index radix digits are
 * sorted) -- by coordinate descent: each knob in turn takes each of its candidate values with the
 * others held; a value is kept when its measured time beats the best so far by more than 2%. The
 * result is therefore never slower than the starting params on the measured runs.
 */
typedef struct {
    uint32_t evaluations;  /* configurations timed (0 when taken from the cache) */
    uint32_t cached;       /* 1: the class was tuned before; its knobs were reused, nothing was timed */
    float default_ms;      /* time of the starting params */
    float best_ms;         /* time of the chosen params */
    uint64_t sample_bases; /* bases of the library the times were measured on */
} turtle_tune_report;

/* Timer of one configuration: milliseconds, or a negative value when the configuration cannot run. */
typedef double (*turtle_tune_timer)(const turtle_params *p, void *user);

/* The selection alone (host only): coordinate descent from *base with `timer`; *best receives the
 * chosen params, *rep (may be NULL) the evaluations and times. TURTLE_E_DEVICE when the timer fails
 * on *base itself; TURTLE_E_ARG for NULL pointers or a base without struct_size set. */
int turtle_tune_select(const turtle_params *base, turtle_tune_timer timer, void *user, turtle_params *best,
                       turtle_tune_report *rep);

/* Device form: tune on a device-resident library (arguments as turtle_count_device; base may be NULL =
 * defaults), timing turtle_count_device on `ctx` and `stream` with CUDA events (one warm-up, median of
 * three runs per configuration). *best = base with the tuned knobs. Results are cached per class of
 * input -- key width, filter used (min_count >= 2), base->compact and floor(log2(n_bases)) -- and a
 * later call of the same class returns the cached knobs at once (rep->cached = 1). The context's
 * last device result is invalidated. */
int turtle_autotune(turtle_ctx *ctx, const uint8_t *bases, uint64_t n_bases, const uint64_t *offsets,
                    uint64_t n_reads, int k, uint32_t min_count, const turtle_params *base, void *stream,
                    turtle_params *best, turtle_tune_report *rep);

/* Forget every cached tuning. */
void turtle_tune_cache_clear(void);

/*
 * Allocation-free variant of turtle_sort_compact (no counterpart in the paper:
 * it exists for callers, not for the method).
 *
 * For callers that may not allocate device memory at all -- no cudaMalloc,
 * cudaFree, memory pool or caching allocator, not even through a context
 * (turtle_ctx_create allocates) -- because a fixed device-memory budget is
 * decided up front, because a host framework owns every allocation and only
 * lends them a stream, or because an allocation could block or fail in a
 * latency-critical loop. Arguments, results and errors are those of
 * turtle_sort_compact, without the context.
 *
 * Scratch is one array of TURTLE_NOALLOC_SCRATCH_BYTES compiled into the
 * library's device image: every GPU that loads libturtle keeps it reserved
 * until the process exits. Limits: n <= TURTLE_NOALLOC_MAX_KEYS64 for 64-bit
 * keys, n <= TURTLE_NOALLOC_MAX_KEYS128 for 128-bit keys; larger n returns
 * TURTLE_E_TOO_LARGE before any work is queued.
 * Alignment as for turtle_sort_compact (keys 8 bytes, unique 8 * key_words
 * bytes, counts 4 bytes; TURTLE_E_ARG otherwise, before any work is queued).
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture begins. Every call waits for its own work: it synchronises `stream`
 * and reads the error word and n_unique back to host memory before returning.
 * All calls share the one array: calls whose work overlaps on the GPU
 * (different streams or threads at the same time) race and corrupt each
 * other's results; serialise them. The array keeps the previous call's
 * contents; the call clears what must start at zero itself.
 */
#define TURTLE_NOALLOC_MAX_KEYS64 (1u << 20)
#define TURTLE_NOALLOC_MAX_KEYS128 (1u << 19)
#define TURTLE_NOALLOC_SCRATCH_BYTES 25727232ull
int turtle_sort_compact_noalloc(const uint64_t *keys, uint64_t n, int key_words, int key_bits, uint64_t *unique,
                                uint32_t *counts, uint64_t *n_unique, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TURTLE_H */
