// Host-side launchers of the libturtle kernels (internal; not part of the C ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace turtle {

struct Key128;

// Layout sizes derived from n_bases (all in uint64 words).
struct PackLayout {
    uint64_t n_bases;
    uint64_t p_words;  // packed 2-bit codes: 32 bases/word, one per pack group (2 * b_words)
    uint64_t b_words;  // ambiguous-call bitmap and read-start bitmap: 64 positions/word, +2 padding
    uint64_t v_words;  // valid-window bitmap: 64 positions/word, +2 padding
    static PackLayout of(uint64_t n_bases) {
        PackLayout L;
        L.n_bases = n_bases;
        L.b_words = (n_bases + 63) / 64 + 2;
        L.p_words = 2 * L.b_words;
        L.v_words = (n_bases + 63) / 64 + 2;
        return L;
    }
    uint64_t pack_groups() const { return 2 * b_words; }  // groups of 32 positions, padding included
};

// Bucket of a key (bucketed sort-and-compact): ((f(top31(key)) - f_lo) >> shift), clamped to
// [0, n_buckets), with the monotone map f(v) = v (2^32 - v) of the key-range parts: buckets are
// consecutive key ranges. Batches (lib != null): library l = the key's tag owns the buckets
// [lib[l].x, lib[l].x + lib[l].y), indexed by f >> lib[l].z; lib[l].w = the library's k in a mixed
// batch (0: every library has k).
struct BucketGeom {
    uint64_t f_lo;
    int shift;
    uint32_t n_buckets;
    int k;
    int tag_shift;
    const uint4 *lib;
};

struct LaunchCfg {
    int sms;            // multiprocessors on the device
    cudaStream_t stream;
};

// a1: P <- 2-bit codes, B <- ambiguous/out-of-read bits, S <- read-start bits (S must be zero on entry).
void launch_pack(const LaunchCfg &c, const uint8_t *bases, const uint64_t *offsets, uint64_t n_reads,
                 const PackLayout &L, uint64_t *P, uint64_t *B, uint64_t *S, uint32_t *err);
// a1 in pieces: groups [g_begin, g_end) of 32 positions (bases indexed by absolute position), and S.
void launch_pack_groups(const LaunchCfg &c, const uint8_t *bases, const uint64_t *offsets, uint64_t n_reads,
                        const PackLayout &L, uint64_t g_begin, uint64_t g_end, uint64_t *P, uint64_t *B);
void launch_mark_starts(const LaunchCfg &c, const uint64_t *offsets, uint64_t n_reads, const PackLayout &L,
                        uint64_t *S, uint32_t *err);
// a1/a2: V <- valid-window bits for k; *n_windows += popcount(V) (zero it first).
// Words [w_begin, w_end) only (window starts 64 w_begin ..): word w needs positions below 64 (w + 2) packed.
void launch_valid(const LaunchCfg &c, const PackLayout &L, int k, const uint64_t *B, const uint64_t *S,
                  uint64_t *V, unsigned long long *n_windows, uint64_t w_begin = 0, uint64_t w_end = ~0ull);
// a2 alone: keys[s] <- canonical key of every valid window start s.
void launch_extract(const LaunchCfg &c, const PackLayout &L, int k, const uint64_t *P, const uint64_t *V,
                    uint64_t *keys);

struct FilterGeom {
    uint64_t *words;        // 4 * n_sectors uint64
    uint64_t n_sectors;     // power of two
    int sector_shift;       // 64 - log2(n_sectors); 64 when n_sectors == 1
    const uint64_t *patterns;  // device, n_patterns masks
    uint32_t pat_mask;      // n_patterns - 1
};

// a2+a3: pass 1. Emits the canonical key of every valid window whose filter test says "seen"
// (every valid window when use_filter is false) to cand[0 .. *cand_count); with a filter and a
// non-null firsts buffer, the other windows (first sightings) fill firsts[first_cap - *first_count ..
// first_cap) from the top, so firsts may be the candidate buffer itself (cand + first_cap == end).
// hist (non-null): += the 256-bin digit counts of the candidates for radix passes 0..hist_passes-1.
// part_bits > 0: only windows whose key lies in key-range parts [part_lo, part_hi) of 2^part_bits take part.
// n_libs > 0 (batched form, <= 64): positions [lib_starts[l], lib_starts[l+1]) belong to library l, whose
// index is added to every key above its 2k bits; lib_filter (optional, 2 * n_libs entries: first
// sector, hash shift) gives each library its own filter region.
template <class K>
void launch_pass1(const LaunchCfg &c, const PackLayout &L, int k, const uint64_t *P, const uint64_t *V,
                  bool use_filter, const FilterGeom &f, K *cand, unsigned long long *cand_count, uint64_t cand_cap,
                  K *firsts, unsigned long long *first_count, uint64_t first_cap, uint64_t *hist, int hist_passes,
                  int part_bits, uint32_t part_lo, uint32_t part_hi, const uint64_t *lib_starts, int n_libs,
                  const uint64_t *lib_filter, uint32_t *err, const BucketGeom *bucket = nullptr, uint64_t t_begin = 0,
                  uint64_t t_end = ~0ull, const uint64_t *rid = nullptr, uint32_t rid_value = 0,
                  const int *lib_k = nullptr, int tag_shift = 0, uint64_t *rid_out = nullptr,
                  const uint8_t *part_group = nullptr);
// (lib_k: mixed batches, each library's k (device, n_libs entries); the library tag then sits at bit tag_shift.
// rid_out: a key range's pass (rid == nullptr) that also writes every window's range id, part_group[part of
// its key], for the passes of the other ranges; word w holds positions 32w .. 32w+31, bit j of its low
// half the low bit of position 32w + j's id, bit j of its high half the high bit.)
// 64-bit keys of a mixed batch's libraries with k <= 32: out[i] <- in[i].lo.
void launch_narrow_keys(const LaunchCfg &c, const Key128 *in, uint64_t n, uint64_t *out);
// Words of the range ids a key range's pass 1 writes (rid_out of launch_pass1): two bits per position, as
// two bit planes per 32 positions.
uint64_t range_id_words(uint64_t n_bases);
// a2+a3, filter-blocked form of pass 1 (one library, bucketed sort-and-compact): the valid windows (of
// parts [part_lo, part_hi) when part_bits > 0) are binned by the top 8 bits of their hash into bin_keys
// (room for every such window), then probed bin after bin, so the filter blocks being probed stay in L2;
// outputs as launch_pass1. bin_words: pass1_bin_words() device words of scratch.
uint64_t pass1_bin_words();
template <class K>
void launch_pass1_binned(const LaunchCfg &c, const PackLayout &L, int k, const uint64_t *P, const uint64_t *V,
                         const FilterGeom &f, K *bin_keys, uint64_t bin_cap, unsigned long long *bin_words, K *cand,
                         unsigned long long *cand_count, uint64_t cand_cap, K *firsts,
                         unsigned long long *first_count, uint64_t first_cap, uint64_t *hist, int hist_passes,
                         int part_bits, uint32_t part_lo, uint32_t part_hi, uint32_t *err, const BucketGeom *bucket);
// Valid windows of each library of a batch (counts: n_libs zeroed counters).
void launch_lib_windows(const LaunchCfg &c, const PackLayout &L, const uint64_t *V, const uint64_t *lib_starts,
                        int n_libs, unsigned long long *counts);
// Batch offsets: library l's offsets (n_reads_l + 1 entries each, concatenated in src) become positions
// in the concatenated bases: dst[first_l + r] = src[first_l + l + r] - src[first_l + l] + lib_starts[l].
void launch_batch_offsets(const LaunchCfg &c, const uint64_t *src, const uint64_t *entry_starts,
                          const uint64_t *lib_starts, int n_libs, uint64_t *dst, uint64_t n_entries);
// Batched output sorted by library tag: starts[l] <- first entry of library l (starts pre-set to
// UINT64_MAX; libraries without entries keep it), and the tag bits (at bit `shift` and up) are cleared.
template <class K>
void launch_split_tags(const LaunchCfg &c, K *keys, uint64_t n, int shift, uint64_t *starts);
// Only the library starts (tags kept).
template <class K>
void launch_tag_starts(const LaunchCfg &c, const K *keys, uint64_t n, int shift, uint64_t *starts);
// Valid windows per key-range part (counts: 2^part_bits zeroed counters).
// cTurtle (Sec. 2.2): two-stage counting filter; keys whose second pattern a window completes
// are appended to out (stage 2 in sector (s + 1) & sector_mask).
template <class K>
void launch_cturtle(const LaunchCfg &c, const PackLayout &L, int k, const uint64_t *P, const uint64_t *V,
                    const FilterGeom &f, uint64_t sector_mask, K *out, unsigned long long *out_count,
                    uint64_t out_cap, uint32_t *err);
template <class K>
void launch_part_count(const LaunchCfg &c, const PackLayout &L, int k, const uint64_t *P, const uint64_t *V,
                       int part_bits, unsigned long long *counts);
// a3 alone on a key array.
template <class K>
void launch_filter_keys(const LaunchCfg &c, const K *keys, uint64_t n, const FilterGeom &f, int set, uint8_t *seen);

// a4: radix sort + run-length compaction.
struct SortScratch {
    void *alt;               // n keys
    uint64_t *hist;          // passes * 256
    uint64_t *lookback;      // max(tiles) * 256 status words (zeroed by the sorter)
    uint32_t *tile_ctr;      // passes + 2 counters (zeroed by the sorter)
    uint64_t lookback_words;
};
int sort_passes_for(int key_bits);
uint64_t sort_lookback_words(uint64_t n, int key_words);
// Sorts keys[0..n) by their low key_bits bits. Returns the buffer that holds the result (keys or scratch.alt).
// hist_ready: s.hist already holds the digit counts of every pass (e.g. accumulated by pass 1);
// bit p of skip_mask skips digit pass p (only valid when every key has the same digit p).
template <class K>
K *launch_radix_sort(const LaunchCfg &c, K *keys, uint64_t n, int key_bits, const SortScratch &s, uint32_t *err,
                     bool hist_ready = false, uint32_t skip_mask = 0, int *passes_run = nullptr, int variant = 0);
// unique/starts from sorted keys; *n_unique (device) receives the distinct count.
template <class K>
void launch_rle(const LaunchCfg &c, const K *sorted, uint64_t n, K *unique, uint64_t *starts,
                unsigned long long *n_unique, uint64_t *lookback, uint32_t *tile_ctr, uint32_t *err);
// counts[j] <- starts[j+1] - starts[j] (starts[n_unique] = n), with overflow check.
void launch_run_counts(const LaunchCfg &c, const uint64_t *starts, const unsigned long long *n_unique, uint64_t n,
                       uint64_t cap, uint32_t *counts, uint32_t *err);

// a5: recount table: lines of 128 bytes (8 slots of 16 B for 64-bit keys, 4 of 32 B for 128-bit).
// One region (lines [0, mask]) or, for a batch, one region per library: lib_regions[2l] = first line,
// lib_regions[2l+1] = line mask, the library taken from the key's tag at bit tag_shift.
struct TableGeom {
    uint64_t mask;
    const uint64_t *lib_regions;  // device, 2 * n_libs (batched form) or nullptr
    int tag_shift;
    int n_libs;
};
template <class K> struct Slot;
size_t slot_bytes(int key_words);
int slots_per_line(int key_words);
template <class K>
void launch_table_clear(const LaunchCfg &c, void *table, uint64_t lines);
// counts == nullptr: every slot starts at 0; otherwise slot j starts at counts[j]. member (optional,
// member_words a power of two, zeroed) receives the membership bitmap of the inserted keys.
template <class K>
void launch_table_insert(const LaunchCfg &c, const K *unique, const uint32_t *counts,
                         const unsigned long long *n_unique, uint64_t cap, void *table, const TableGeom &tg,
                         uint64_t *member, uint64_t member_words, uint32_t *err);
// a5 (first-sighting form): +1 on the slot of every key of firsts[0 .. n) that is in the table.
template <class K>
void launch_add_firsts(const LaunchCfg &c, const K *firsts, uint64_t n, void *table, const TableGeom &tg,
                       const uint64_t *member, uint64_t member_words, bool check_overflow, uint32_t *err);
template <class K>
void launch_pass2(const LaunchCfg &c, const PackLayout &L, int k, const uint64_t *P, const uint64_t *V,
                  void *table, const TableGeom &tg, bool check_overflow, uint32_t *err);
// a6: keep count >= min_count in key order.
template <class K>
void launch_threshold(const LaunchCfg &c, const K *unique, uint64_t n_unique, const void *table, const TableGeom &tg,
                      uint32_t min_count, K *out_keys, uint32_t *out_counts, unsigned long long *n_out,
                      uint64_t *lookback, uint32_t *tile_ctr, uint32_t *err);

// ---------------------------------------------------------------- bucketed sort-and-compact (bucket.cu)
// Stable sort of keys[0 .. n) by bucket index (8 bits per onesweep pass); returns keys or s.alt.
template <class K>
K *launch_bucket_sort(const LaunchCfg &c, K *keys, uint64_t n, const BucketGeom &g, int bits, const SortScratch &s,
                      uint32_t *err, int *passes_run, bool hist_ready, int variant = 0);
// off[b] <- first position of bucket b in bucket-sorted keys, b = 0 .. n_buckets (off[n_buckets] = n).
template <class K>
void launch_bucket_bounds(const LaunchCfg &c, const K *keys, uint64_t n, const BucketGeom &g,
                          unsigned long long *off);
// out[0 .. n] <- exclusive scan of in[0 .. n), out[n] = total (one CTA).
void launch_scan_u64(const LaunchCfg &c, const unsigned long long *in, uint64_t n, unsigned long long *out);
// Per bucket: merge candidates, add first sightings (first may be null), keep count >= min_count,
// sort; results at tmp_*[off_c[b] ..], their number at n_rep[b]. ticket must be zero on entry.
template <class K>
void launch_bucket_count(const LaunchCfg &c, const K *cand, const unsigned long long *off_c, const K *first,
                         const unsigned long long *off_f, uint32_t B, uint32_t min_count, K *tmp_keys,
                         uint32_t *tmp_counts, unsigned long long *n_rep, uint32_t *ticket,
                         unsigned long long *n_distinct, uint32_t *err, int large = 0);
// Dense output: bucket b's n_rep entries from tmp_*[off[b] ..] to out[out_off[b] ..].
template <class K>
void launch_bucket_gather(const LaunchCfg &c, const K *tmp_keys, const uint32_t *tmp_counts,
                          const unsigned long long *off, const unsigned long long *out_off, uint32_t B, K *okeys,
                          uint32_t *ocounts);

// ---------------------------------------------------------------- lazy sort-and-compact phases (merge.cu)
// Merge the ascending runs of distinct keys A[0 .. na) and B[0 .. nb) (counts ca, cb) into out/cout, a key in
// both inputs once with its counts added; *n_out <- the merged length. Scratch: split (merge_tiles(na + nb) + 1
// words), lookback (merge_tiles(na + nb) words), tile_ctr (one word). out must not alias A or B.
// skip_tile0 / spin_limit (failure-injection tests only): start the tile tickets at 1, so the look-back
// waits of tiles 1.. run out after spin_limit rounds (0 = the default limit) and ERR_LOOKBACK is set.
uint64_t merge_tiles(uint64_t n);
template <class K>
void launch_merge_counts(const LaunchCfg &c, const K *A, const uint32_t *ca, uint64_t na, const K *B,
                         const uint32_t *cb, uint64_t nb, K *out, uint32_t *cout, unsigned long long *n_out,
                         uint64_t *split, uint64_t *lookback, uint32_t *tile_ctr, uint32_t *err,
                         bool skip_tile0 = false, uint32_t spin_limit = 0);

// ---------------------------------------------------------------- hash-table counting (hashcount.cu)
// Open-addressing table of 128-byte lines (8 slots of 16 B for 64-bit keys, 4 of 32 B for 128-bit),
// lines a power of two. regs: 2^hash_sketch_bits() zeroed uint32 HyperLogLog registers.
int hash_sketch_bits();
int hash_slots_per_line(int key_words);
template <class K>
void launch_hash_sketch(const LaunchCfg &c, const K *keys, uint64_t n, uint32_t *regs);
template <class K>
void launch_hash_clear(const LaunchCfg &c, void *table, uint64_t lines);
// +1 on the slot of every key of keys[0 .. n); *n_distinct += slots taken; *full = 1 when a key found
// no slot within its probe bound (the counts are then incomplete: clear a larger table and redo).
template <class K>
void launch_hash_insert(const LaunchCfg &c, const K *keys, uint64_t n, void *table, uint64_t lines,
                        bool check_overflow, unsigned long long *n_distinct, uint32_t *full, uint32_t *err);
// +1 on the slot of every key of keys[0 .. n) that is in the table.
template <class K>
void launch_hash_firsts(const LaunchCfg &c, const K *keys, uint64_t n, void *table, uint64_t lines,
                        bool check_overflow, uint32_t *err);
// out[0 .. *n_out) <- the keys whose count >= min_count (in no particular order; *n_out zeroed first).
template <class K>
void launch_hash_extract(const LaunchCfg &c, const void *table, uint64_t lines, uint32_t min_count, K *out,
                         uint64_t cap, unsigned long long *n_out, uint32_t *err);
// counts[i] <- count of keys[i] (every key must be in the table).
template <class K>
void launch_hash_lookup(const LaunchCfg &c, const K *keys, uint64_t n, const void *table, uint64_t lines,
                        uint32_t *counts, uint32_t *err);

}  // namespace turtle
