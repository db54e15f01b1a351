// Steps a2+a3: canonical extraction and the pattern-blocked Bloom filter (Sec. 2.1.3).
//
// Block = one 32-byte DRAM sector chosen by the top bits of the key hash; the
// precomputed pattern (from a table kept in shared memory, indexed by the low
// hash bits) lies inside one 64-bit word of that sector, chosen by hash bits
// 16..17. A probe therefore costs one sector, and test-and-set is a single
// atomicOr on one word.
//
// Why one word: "seen before" must be decided by one linearizable operation.
// If a pattern spanned several words with one atomic each, two concurrent first
// sightings of a key could each find a different word not yet set and both
// conclude "first sighting"; the key would then never become a candidate and
// the recount could not repair the miss. With one atomicOr per key, among all
// occurrences of a key at most one can observe its pattern incomplete, so every
// key seen twice emits at least one candidate (no false negatives, for any
// interleaving). A plain load that already shows every pattern bit set proves
// "seen" without the atomic, because bits are never cleared.
#include <algorithm>

#include "bucket.cuh"

namespace turtle {

constexpr int P1_BLOCK = 256;
constexpr int P1_WARPS = P1_BLOCK / WARP;
constexpr int P1_ILP = 4;                    // window starts per lane per warp tile
constexpr int P1_TILE = WARP * P1_ILP;       // 128 starts per warp tile (two V words)
constexpr int P1_STAGE = 256;                // keys per candidate flush
constexpr int P1_BUF = P1_STAGE + WARP;      // warp staging buffer capacity

// A stream written with `down` fills its buffer from the top: entry j lands at cap-1-j, so
// candidates (from the bottom) and first sightings (from the top) can share one buffer.
template <class K>
__device__ __forceinline__ void flush_full(K *wbuf, int &nbuf, K *out, unsigned long long *cursor,
                                           uint64_t cap, uint32_t *err, int lane, bool down = false) {
    __syncwarp();
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(cursor, (unsigned long long)P1_STAGE);
    base = __shfl_sync(FULL, base, 0);
    if (base + P1_STAGE <= cap) {
        if (down) base = cap - base - P1_STAGE;
#pragma unroll
        for (int j = 0; j < P1_STAGE / WARP; j++) store_key(out + base + lane + WARP * j, wbuf[lane + WARP * j]);
    } else if (lane == 0) {
        atomicOr(err, ERR_CAND_OVERFLOW);
    }
    const int rem = nbuf - P1_STAGE;
    K tail;
    if (lane < rem) tail = wbuf[P1_STAGE + lane];
    __syncwarp();
    if (lane < rem) wbuf[lane] = tail;
    __syncwarp();
    nbuf = rem;
}

template <class K>
__device__ __forceinline__ void flush_rest(K *wbuf, int nbuf, K *out, unsigned long long *cursor, uint64_t cap,
                                           uint32_t *err, int lane, bool down = false) {
    __syncwarp();
    if (nbuf <= 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(cursor, (unsigned long long)nbuf);
    base = __shfl_sync(FULL, base, 0);
    if (base + nbuf <= cap) {
        if (down) base = cap - base - nbuf;
        for (int j = lane; j < nbuf; j += WARP) store_key(out + base + j, wbuf[j]);
    } else if (lane == 0) {
        atomicOr(err, ERR_CAND_OVERFLOW);
    }
}

// Digit counts of every radix pass for the keys being flushed (fused into pass 1 so the
// sorter does not have to read the keys once more just to histogram them): digits of the key
// itself, or (by_bucket) of its bucket index for the bucketed sort-and-compact.
template <class K>
__device__ __forceinline__ void hist_keys(const K *buf, int count, uint32_t *s_hist, int passes, int lane,
                                          const BucketGeom &bg, bool by_bucket) {
    for (int j = lane; j < count; j += WARP) {
        const K key = buf[j];
        if (by_bucket) {
            const uint32_t b = bucket_of(key, bg);
            for (int p = 0; p < passes; p++) atomicAdd(&s_hist[p * 256 + ((b >> (8 * p)) & 0xffu)], 1u);
        } else {
            for (int p = 0; p < passes; p++) atomicAdd(&s_hist[p * 256 + KeyT<K>::digit(key, 8 * p)], 1u);
        }
    }
}

// Every valid window lands in exactly one stream: "seen" windows go to cand, and
// (when EMIT_FIRSTS) the windows whose atomicOr completed their pattern go to
// firsts. Since that atomicOr is one linearizable operation, at most one
// occurrence of a key can ever be a first.
// MODE bits: P1_BATCHED (windows tagged with their library), P1_PARTED (only the windows of key-range
// parts [part_lo, part_hi)), P1_BY_BUCKET (histograms of the bucket index rather than the key). Each
// combination is its own kernel, so none carries the lookups of the forms it does not serve.
constexpr int P1_BATCHED = 1, P1_PARTED = 2, P1_BY_BUCKET = 4;

template <class K, bool USE_FILTER, bool EMIT_FIRSTS, int MODE>
__global__ void __launch_bounds__(P1_BLOCK) k_pass1(const uint64_t *__restrict__ P, const uint64_t *__restrict__ V,
                                                    uint64_t n_pos, int k, uint64_t *filter, int sector_shift,
                                                    const uint64_t *__restrict__ patterns, uint32_t pat_mask,
                                                    K *cand, unsigned long long *cand_count, uint64_t cand_cap,
                                                    K *firsts, unsigned long long *first_count, uint64_t first_cap,
                                                    uint64_t *hist, int hist_passes, int part_bits, uint32_t part_lo,
                                                    uint32_t part_hi, const uint64_t *__restrict__ lib_starts,
                                                    int n_libs, const uint64_t *__restrict__ lib_filter,
                                                    const int *__restrict__ lib_k, int tag_shift,
                                                    BucketGeom bg, int by_bucket, uint64_t t_begin, uint64_t t_end,
                                                    uint32_t *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NBUF = EMIT_FIRSTS ? 2 : 1;
    constexpr bool BATCHED = (MODE & P1_BATCHED) != 0, PARTED = (MODE & P1_PARTED) != 0;
    constexpr bool BY_BUCKET = (MODE & P1_BY_BUCKET) != 0;
    (void)by_bucket;
    // by_bucket: first sightings get their own histograms, after the candidates'
    const int n_hist = 256 * hist_passes * (BY_BUCKET && EMIT_FIRSTS ? 2 : 1);
    K *s_buf = reinterpret_cast<K *>(smem);
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(smem + sizeof(K) * P1_BUF * P1_WARPS * NBUF);
    uint32_t *s_fhist = s_hist + 256 * hist_passes;
    uint64_t *s_pat = reinterpret_cast<uint64_t *>(s_hist + n_hist);
    __shared__ uint64_t s_lib[65];
    __shared__ uint64_t s_lf[128];  // per-library filter region: first sector, shift of the hash
    __shared__ int s_libk[64];      // mixed batches: each library's k
    if (BATCHED)
        for (int i = threadIdx.x; i <= n_libs; i += P1_BLOCK) s_lib[i] = lib_starts[i];
    if (BATCHED && lib_k)
        for (int i = threadIdx.x; i < n_libs; i += P1_BLOCK) s_libk[i] = lib_k[i];
    if (BATCHED && lib_filter)
        for (int i = threadIdx.x; i < 2 * n_libs; i += P1_BLOCK) s_lf[i] = lib_filter[i];
    if (USE_FILTER)
        for (uint32_t i = threadIdx.x; i <= pat_mask; i += P1_BLOCK) s_pat[i] = patterns[i];
    for (int i = threadIdx.x; i < n_hist; i += P1_BLOCK) s_hist[i] = 0;
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    K *wbuf = s_buf + warp * P1_BUF * NBUF;
    K *fbuf = wbuf + P1_BUF;  // firsts staging (EMIT_FIRSTS only)
    int nbuf = 0, nfirst = 0;
    for (uint64_t t = t_begin + (uint64_t)blockIdx.x * P1_WARPS + warp; t < t_end; t += (uint64_t)gridDim.x * P1_WARPS) {
        const uint64_t base = t * P1_TILE;
        const uint64_t v0 = V[2 * t], v1 = V[2 * t + 1];
        bool ok[P1_ILP];
        K key[P1_ILP];
        uint64_t *addr[P1_ILP];
        uint64_t mask[P1_ILP];
        uint32_t libi[P1_ILP];
        int lib0 = 0;  // batched form: library of the tile's first position (binary search, once per tile)
        if (BATCHED) {
            int hi = n_libs;
            while (hi - lib0 > 1) {
                const int mid = (lib0 + hi) >> 1;
                if (s_lib[mid] <= base) lib0 = mid;
                else hi = mid;
            }
        }
#pragma unroll
        for (int i = 0; i < P1_ILP; i++) {
            const int r = lane + WARP * i;
            const uint64_t s = base + r;
            ok[i] = s < n_pos && (((r < 64 ? v0 : v1) >> (r & 63)) & 1);
            if (ok[i]) {
                if (BATCHED) {  // batched form: tag the key with its library (the tile's, or a later one)
                    int lo = lib0;
                    while (lo + 1 < n_libs && s_lib[lo + 1] <= s) lo++;
                    // mixed batches: every library its own k, the tag in the key's top bits
                    key[i] = canonical<K>(P, s, lib_k ? s_libk[lo] : k);
                    key[i] = add_tag(key[i], (uint32_t)lo, lib_k ? tag_shift : 2 * k);
                    libi[i] = (uint32_t)lo;
                } else {
                    key[i] = canonical<K>(P, s, k);
                }
                if (PARTED) {  // keys of other key ranges wait for their own super-partition
                    const uint32_t pt = key_part(key[i], k, part_bits);
                    ok[i] = pt >= part_lo && pt < part_hi;
                }
            }
            if (ok[i]) {
                if (USE_FILTER) {
                    const uint64_t h = key_hash(key[i]);
                    uint64_t sector;
                    if (BATCHED && lib_filter) {  // batched: each library has its own region, hot in L2 while its
                        const uint64_t sh = s_lf[2 * libi[i] + 1];  // windows are being processed
                        sector = s_lf[2 * libi[i]] + (sh < 64 ? (h >> sh) : 0);
                    } else {
                        sector = sector_shift < 64 ? (h >> sector_shift) : 0;
                    }
                    addr[i] = filter + sector * 4 + ((h >> 16) & 3);
                    mask[i] = s_pat[h & pat_mask];
                }
            }
        }
        bool seen[P1_ILP];
        if (USE_FILTER) {
            uint64_t w[P1_ILP];
#pragma unroll
            for (int i = 0; i < P1_ILP; i++) w[i] = ok[i] ? __ldcg(addr[i]) : 0;
#pragma unroll
            for (int i = 0; i < P1_ILP; i++) {
                seen[i] = ok[i];
                if (ok[i] && (w[i] & mask[i]) != mask[i]) {
                    const uint64_t old = atomicOr((unsigned long long *)addr[i], (unsigned long long)mask[i]);
                    seen[i] = (old & mask[i]) == mask[i];
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < P1_ILP; i++) seen[i] = ok[i];
        }
#pragma unroll
        for (int i = 0; i < P1_ILP; i++) {
            const uint32_t b = __ballot_sync(FULL, seen[i]);
            if (seen[i]) wbuf[nbuf + __popc(b & lt)] = key[i];
            nbuf += __popc(b);
            if (nbuf >= P1_STAGE) {
                __syncwarp();
                hist_keys(wbuf, P1_STAGE, s_hist, hist_passes, lane, bg, BY_BUCKET);
                flush_full(wbuf, nbuf, cand, cand_count, cand_cap, err, lane);
            }
            if (EMIT_FIRSTS) {
                const bool f = ok[i] && !seen[i];
                const uint32_t bf = __ballot_sync(FULL, f);
                if (f) fbuf[nfirst + __popc(bf & lt)] = key[i];
                nfirst += __popc(bf);
                if (nfirst >= P1_STAGE) {
                    if (BY_BUCKET) {
                        __syncwarp();
                        hist_keys(fbuf, P1_STAGE, s_fhist, hist_passes, lane, bg, true);
                    }
                    flush_full(fbuf, nfirst, firsts, first_count, first_cap, err, lane, true);
                }
            }
        }
    }
    __syncwarp();
    hist_keys(wbuf, nbuf, s_hist, hist_passes, lane, bg, BY_BUCKET);
    flush_rest(wbuf, nbuf, cand, cand_count, cand_cap, err, lane);
    if (EMIT_FIRSTS) {
        if (BY_BUCKET) hist_keys(fbuf, nfirst, s_fhist, hist_passes, lane, bg, true);
        flush_rest(fbuf, nfirst, firsts, first_count, first_cap, err, lane, true);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_hist; i += P1_BLOCK)
        if (s_hist[i]) atomicAdd((unsigned long long *)&hist[i], (unsigned long long)s_hist[i]);
}

// cTurtle (Sec. 2.2): a two-stage counting filter. Stage 1 is pass 1's test-and-set in the key's
// block; a window that finds its stage-1 pattern complete tests and sets a second pattern in the
// adjacent block (sector s + 1, word (h >> 18) & 3, pattern (h >> 20) & mask), and the window whose
// atomicOr completes that pattern reports the key. Each stage is one atomic on one word, so a key
// is reported at most once; which colliding keys are missed or reported as singletons depends on
// the order of the windows, as in the paper's sequential tool.
template <class K>
__global__ void __launch_bounds__(P1_BLOCK) k_cturtle(const uint64_t *__restrict__ P, const uint64_t *__restrict__ V,
                                                      uint64_t n_pos, int k, uint64_t *filter, int sector_shift,
                                                      uint64_t sector_mask, const uint64_t *__restrict__ patterns,
                                                      uint32_t pat_mask, K *out, unsigned long long *out_count,
                                                      uint64_t out_cap, uint32_t *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    K *s_buf = reinterpret_cast<K *>(smem);
    uint64_t *s_pat = reinterpret_cast<uint64_t *>(smem + sizeof(K) * P1_BUF * P1_WARPS);
    for (uint32_t i = threadIdx.x; i <= pat_mask; i += P1_BLOCK) s_pat[i] = patterns[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    K *wbuf = s_buf + warp * P1_BUF;
    int nbuf = 0;
    const uint64_t tiles = (n_pos + P1_TILE - 1) / P1_TILE;
    for (uint64_t t = (uint64_t)blockIdx.x * P1_WARPS + warp; t < tiles; t += (uint64_t)gridDim.x * P1_WARPS) {
        const uint64_t base = t * P1_TILE;
        const uint64_t v0 = V[2 * t], v1 = V[2 * t + 1];
#pragma unroll
        for (int i = 0; i < P1_ILP; i++) {
            const int r = lane + WARP * i;
            const uint64_t s = base + r;
            const bool ok = s < n_pos && (((r < 64 ? v0 : v1) >> (r & 63)) & 1);
            K key{};
            bool emit = false;
            if (ok) {
                key = canonical<K>(P, s, k);
                const uint64_t h = key_hash(key);
                const uint64_t s1 = sector_shift < 64 ? (h >> sector_shift) : 0;
                uint64_t *a1 = filter + s1 * 4 + ((h >> 16) & 3);
                const uint64_t m1 = s_pat[h & pat_mask];
                bool seen = (__ldcg(a1) & m1) == m1;
                if (!seen) seen = (atomicOr((unsigned long long *)a1, (unsigned long long)m1) & m1) == m1;
                if (seen) {
                    uint64_t *a2 = filter + ((s1 + 1) & sector_mask) * 4 + ((h >> 18) & 3);
                    const uint64_t m2 = s_pat[(h >> 20) & pat_mask];
                    if ((__ldcg(a2) & m2) != m2)
                        emit = (atomicOr((unsigned long long *)a2, (unsigned long long)m2) & m2) != m2;
                }
            }
            const uint32_t b = __ballot_sync(FULL, emit);
            if (emit) wbuf[nbuf + __popc(b & lt)] = key;
            nbuf += __popc(b);
            if (nbuf >= P1_STAGE) flush_full(wbuf, nbuf, out, out_count, out_cap, err, lane);
        }
    }
    __syncwarp();
    flush_rest(wbuf, nbuf, out, out_count, out_cap, err, lane);
}

template <class K>
void launch_cturtle(const LaunchCfg &c, const PackLayout &L, int k, const uint64_t *P, const uint64_t *V,
                    const FilterGeom &f, uint64_t sector_mask, K *out, unsigned long long *out_count,
                    uint64_t out_cap, uint32_t *err) {
    const uint64_t tiles = (L.n_bases + P1_TILE - 1) / P1_TILE;
    const size_t smem = sizeof(K) * P1_BUF * P1_WARPS + sizeof(uint64_t) * (f.pat_mask + 1);
    cudaFuncSetAttribute(k_cturtle<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cturtle<K>, P1_BLOCK, smem);
    if (per_sm < 1) per_sm = 1;
    const uint64_t need = (tiles + P1_WARPS - 1) / P1_WARPS, cap = (uint64_t)c.sms * per_sm;
    const int grid = (int)(need < cap ? (need ? need : 1) : cap);
    k_cturtle<K><<<grid, P1_BLOCK, smem, c.stream>>>(P, V, L.n_bases, k, f.words, f.sector_shift, sector_mask,
                                                     f.patterns, f.pat_mask, out, out_count, out_cap, err);
}
template void launch_cturtle<uint64_t>(const LaunchCfg &, const PackLayout &, int, const uint64_t *,
                                       const uint64_t *, const FilterGeom &, uint64_t, uint64_t *,
                                       unsigned long long *, uint64_t, uint32_t *);
template void launch_cturtle<Key128>(const LaunchCfg &, const PackLayout &, int, const uint64_t *, const uint64_t *,
                                     const FilterGeom &, uint64_t, Key128 *, unsigned long long *, uint64_t,
                                     uint32_t *);

// Part (of 2^part_bits) of the canonical key of the window at s, exactly as key_part of that key. The top 31
// bits of the canonical key are the smaller of the top 31 bits of the forward encoding and of the reverse
// complement (if those differ, the smaller belongs to the smaller key; if equal, both keys share them); for
// 128-bit keys they come from the window's first 32 bases and its last 32 bases, without building the keys.
template <class K>
__device__ __forceinline__ uint32_t window_part(const uint64_t *__restrict__ P, uint64_t s, int k, int part_bits);
template <>
__device__ __forceinline__ uint32_t window_part<uint64_t>(const uint64_t *__restrict__ P, uint64_t s, int k,
                                                          int part_bits) {
    return key_part(canonical_at(P, s, k), k, part_bits);
}
template <>
__device__ __forceinline__ uint32_t window_part<Key128>(const uint64_t *__restrict__ P, uint64_t s, int k,
                                                        int part_bits) {
    const uint64_t e = s + (uint64_t)k - 16;  // k >= 33: the window's last 16 bases start at e > s
    const uint64_t a = stream_bits(__ldg(P + (s >> 5)), __ldg(P + (s >> 5) + 1), (int)(s & 31) << 1);
    const uint32_t b = (uint32_t)(stream_bits(__ldg(P + (e >> 5)), __ldg(P + (e >> 5) + 1), (int)(e & 31) << 1) >> 32);
    // the reverse complement begins with the complements of the last 16 bases, last first
    uint32_t r = __brev(b);
    r = ((r >> 1) & 0x55555555u) | ((r & 0x55555555u) << 1);
    const uint32_t vf = (uint32_t)(a >> 33), vr = (~r) >> 1;  // top 31 bits of forward / reverse complement
    const uint32_t v = vf < vr ? vf : vr;
    // (v (2^32 - v)) >> (62 - part_bits), from the high word of the 32 x 32-bit product (v < 2^31)
    return v ? __umulhi(v, 0u - v) >> (30 - part_bits) : 0u;
}

// Number of valid windows in each of the 2^part_bits key-range parts (sizes the super-partitions and the
// shards). Warp tiles of 128 positions read their two validity words once; the part comes from the exact
// end-bases test of window_part (no full 128-bit key is built); each warp counts into its own shared
// histogram, so lanes of different warps never contend for a bin.
template <class K>
__global__ void __launch_bounds__(256) k_part_count(const uint64_t *__restrict__ P, const uint64_t *__restrict__ V,
                                                    uint64_t n_pos, int k, int part_bits,
                                                    unsigned long long *counts) {
    extern __shared__ uint32_t s_cnt[];  // 8 warps x 2^part_bits
    const int nparts = 1 << part_bits;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 8 * nparts; i += blockDim.x) s_cnt[i] = 0;
    __syncthreads();
    uint32_t *mine = s_cnt + warp * nparts;
    const uint64_t tiles = (n_pos + P1_TILE - 1) / P1_TILE;
    for (uint64_t t = (uint64_t)blockIdx.x * 8 + warp; t < tiles; t += (uint64_t)gridDim.x * 8) {
        const uint64_t base = t * P1_TILE;
        const uint64_t v0 = V[2 * t], v1 = V[2 * t + 1];
#pragma unroll
        for (int i = 0; i < P1_ILP; i++) {
            const int r = lane + WARP * i;
            const uint64_t s = base + r;
            if (s < n_pos && (((r < 64 ? v0 : v1) >> (r & 63)) & 1)) atomicAdd(&mine[window_part<K>(P, s, k, part_bits)], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        uint32_t c = 0;
        for (int w = 0; w < 8; w++) c += s_cnt[w * nparts + i];
        if (c) atomicAdd(&counts[i], (unsigned long long)c);
    }
}

template <class K>
void launch_part_count(const LaunchCfg &c, const PackLayout &L, int k, const uint64_t *P, const uint64_t *V,
                       int part_bits, unsigned long long *counts) {
    const uint64_t tiles = (L.n_bases + P1_TILE - 1) / P1_TILE;
    const uint64_t need = (tiles + 7) / 8, cap = (uint64_t)c.sms * 8;
    k_part_count<K><<<(int)(need < cap ? (need ? need : 1) : cap), 256, 32u << part_bits, c.stream>>>(
        P, V, L.n_bases, k, part_bits, counts);
}
template void launch_part_count<uint64_t>(const LaunchCfg &, const PackLayout &, int, const uint64_t *,
                                          const uint64_t *, int, unsigned long long *);
template void launch_part_count<Key128>(const LaunchCfg &, const PackLayout &, int, const uint64_t *,
                                        const uint64_t *, int, unsigned long long *);

// Key range of every window, two bits per position, for up to four ranges: range id = group[part of the
// window's key], written by the first range's pass 1. Word w covers positions 32w .. 32w+31 as two bit
// planes: bit j of its low half is the low bit of position 32w + j's id, bit j of its high half the high
// bit. The other ranges' passes select their windows from these words and the validity bitmap, without
// computing any other key.
constexpr int MAX_PARTS = 64;  // key-range parts of a library (part_bits <= 6)

// 16-byte asynchronous copy global -> shared (both addresses 16-byte aligned), and its group bookkeeping.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

uint64_t range_id_words(uint64_t n_bases) { return 4 * ((n_bases + P1_TILE - 1) / P1_TILE) + 4; }

template <class K>
__global__ void __launch_bounds__(256) k_filter_keys(const K *__restrict__ keys, uint64_t n, uint64_t *filter,
                                                     int sector_shift, const uint64_t *__restrict__ patterns,
                                                     uint32_t pat_mask, int set, uint8_t *seen) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const K key = keys[i];
        const uint64_t h = key_hash(key);
        const uint64_t sector = sector_shift < 64 ? (h >> sector_shift) : 0;
        uint64_t *addr = filter + sector * 4 + ((h >> 16) & 3);
        const uint64_t m = patterns[h & pat_mask];
        uint64_t w = __ldcg(addr);
        bool s = (w & m) == m;
        if (set && !s) s = (atomicOr((unsigned long long *)addr, (unsigned long long)m) & m) == m;
        if (seen) seen[i] = s ? 1 : 0;
    }
}

// ---------------------------------------------------------------- pass 1 for one key range (super-partitions, shards)
// A key range holds a fraction of the windows. Testing each window where it is and probing the filter
// only for those in range would leave most lanes of a warp idle during the probe round trips, which
// are what pass 1 waits on. Instead, each warp first tests a tile of 128 windows for the range and
// appends the positions of those in range to a queue in shared memory; whenever the queue holds 128
// positions, the warp extracts their keys and probes them four per lane, as pass 1 does for a full
// tile. The range test needs only the top 31 bits of the canonical key, which are the smaller of
// the top 31 bits of the forward encoding and of the reverse complement (if those differ, the
// smaller one belongs to the smaller key; if they are equal, both keys share them). For 128-bit keys
// those come from the window's first 32 bases and from its last 32 bases, without building either
// full key; the probe phase checks every key against the range once more.
constexpr int PQ_CAP = 2 * P1_TILE;  // queue of in-range positions per warp: one tile's worth beyond a full batch

template <class K, bool EMIT_FIRSTS, bool BY_BUCKET, bool WRITE_RID>
__global__ void __launch_bounds__(P1_BLOCK) k_pass1_range(const uint64_t *__restrict__ P, const uint64_t *__restrict__ V,
                                                          uint64_t n_pos, int k, uint64_t *filter, int sector_shift,
                                                          const uint64_t *__restrict__ patterns, uint32_t pat_mask,
                                                          K *cand, unsigned long long *cand_count, uint64_t cand_cap,
                                                          K *firsts, unsigned long long *first_count,
                                                          uint64_t first_cap, uint64_t *hist, int hist_passes,
                                                          int part_bits, uint32_t part_lo, uint32_t part_hi,
                                                          const uint64_t *__restrict__ rid, uint32_t rid_value,
                                                          uint64_t *rid_out, const uint8_t *__restrict__ part_group,
                                                          BucketGeom bg, uint64_t t_begin, uint64_t t_end,
                                                          uint32_t *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NBUF = EMIT_FIRSTS ? 2 : 1;
    const int n_hist = 256 * hist_passes * (BY_BUCKET && EMIT_FIRSTS ? 2 : 1);
    K *s_buf = reinterpret_cast<K *>(smem);
    uint64_t *s_queue = reinterpret_cast<uint64_t *>(smem + sizeof(K) * P1_BUF * P1_WARPS * NBUF);
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(s_queue + PQ_CAP * P1_WARPS);
    uint32_t *s_fhist = s_hist + 256 * hist_passes;
    uint64_t *s_pat = reinterpret_cast<uint64_t *>(s_hist + n_hist);
    __shared__ uint8_t s_pg[MAX_PARTS];  // WRITE_RID: range of each key-range part
    __shared__ __align__(16) uint64_t s_stage[P1_WARPS][2][6];  // each warp's next tiles' words
    for (uint32_t i = threadIdx.x; i <= pat_mask; i += P1_BLOCK) s_pat[i] = patterns[i];
    for (int i = threadIdx.x; i < n_hist; i += P1_BLOCK) s_hist[i] = 0;
    if (WRITE_RID)
        for (int i = threadIdx.x; i < (1 << part_bits); i += P1_BLOCK) s_pg[i] = part_group[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    K *wbuf = s_buf + warp * P1_BUF * NBUF;
    K *fbuf = wbuf + P1_BUF;
    uint64_t *q = s_queue + warp * PQ_CAP;
    int nbuf = 0, nfirst = 0, nq = 0;
    // extract, test-and-set and emit the first `count` queued positions (count <= P1_TILE)
    auto probe = [&](int count) {
        bool ok[P1_ILP], seen[P1_ILP];
        K key[P1_ILP];
        uint64_t *addr[P1_ILP];
        uint64_t mask[P1_ILP], w[P1_ILP];
#pragma unroll
        for (int i = 0; i < P1_ILP; i++) {
            const int j = lane + WARP * i;
            ok[i] = j < count;
            if (ok[i]) {
                key[i] = canonical<K>(P, q[j], k);
                const uint32_t pt = key_part(key[i], k, part_bits);
                if (pt < part_lo || pt >= part_hi) {  // cannot happen: the range test is exact
                    atomicOr(err, ERR_PART_MISMATCH);
                    ok[i] = false;
                }
            }
            if (ok[i]) {
                const uint64_t h = key_hash(key[i]);
                const uint64_t sector = sector_shift < 64 ? (h >> sector_shift) : 0;
                addr[i] = filter + sector * 4 + ((h >> 16) & 3);
                mask[i] = s_pat[h & pat_mask];
            }
        }
#pragma unroll
        for (int i = 0; i < P1_ILP; i++) w[i] = ok[i] ? __ldcg(addr[i]) : 0;
#pragma unroll
        for (int i = 0; i < P1_ILP; i++) {
            seen[i] = ok[i];
            if (ok[i] && (w[i] & mask[i]) != mask[i]) {
                const uint64_t old = atomicOr((unsigned long long *)addr[i], (unsigned long long)mask[i]);
                seen[i] = (old & mask[i]) == mask[i];
            }
        }
#pragma unroll
        for (int i = 0; i < P1_ILP; i++) {
            const uint32_t b = __ballot_sync(FULL, seen[i]);
            if (seen[i]) wbuf[nbuf + __popc(b & lt)] = key[i];
            nbuf += __popc(b);
            if (nbuf >= P1_STAGE) {
                __syncwarp();
                hist_keys(wbuf, P1_STAGE, s_hist, hist_passes, lane, bg, BY_BUCKET);
                flush_full(wbuf, nbuf, cand, cand_count, cand_cap, err, lane);
            }
            if (EMIT_FIRSTS) {
                const bool f = ok[i] && !seen[i];
                const uint32_t bf = __ballot_sync(FULL, f);
                if (f) fbuf[nfirst + __popc(bf & lt)] = key[i];
                nfirst += __popc(bf);
                if (nfirst >= P1_STAGE) {
                    if (BY_BUCKET) {
                        __syncwarp();
                        hist_keys(fbuf, P1_STAGE, s_fhist, hist_passes, lane, bg, true);
                    }
                    flush_full(fbuf, nfirst, firsts, first_count, first_cap, err, lane, true);
                }
            }
        }
    };
    // A warp's tiles are strided across the grid; each tile's two validity words and (with range ids) its
    // four range-id words are copied to shared memory (cp.async, lanes 0-2) while the warp works on the
    // previous tile, so a tile's test does not wait for its words and the copy overlaps the probes.
    uint64_t(*stage)[6] = s_stage[warp];
    const uint64_t stride = (uint64_t)gridDim.x * P1_WARPS;
    auto fetch = [&](uint64_t tt, int b) {
        if (tt < t_end) {
            if (lane == 0) cp_async16(&stage[b][0], V + 2 * tt);
            else if (rid && lane < 3) cp_async16(&stage[b][2 * lane], rid + 4 * tt + 2 * (lane - 1));
        }
        cp_async_commit();
    };
    uint64_t t = t_begin + (uint64_t)blockIdx.x * P1_WARPS + warp;
    int sb = 0;
    fetch(t, 0);
    for (; t < t_end; t += stride, sb ^= 1) {
        cp_async_wait_all();
        __syncwarp();  // the tile's words have landed; every lane is done with the other buffer
        const uint64_t base = t * P1_TILE;
        const uint64_t v0 = stage[sb][0], v1 = stage[sb][1];
        uint64_t rw[P1_ILP];
        if (rid)
#pragma unroll
            for (int i = 0; i < P1_ILP; i++) rw[i] = stage[sb][2 + i];
        fetch(t + stride, sb ^ 1);
        bool in[P1_ILP];  // all four windows' tests first, so their loads overlap; then the ballots
        if (WRITE_RID) {  // the first range's pass: every window's range id, written for the later passes
            uint32_t g[P1_ILP];
#pragma unroll
            for (int i = 0; i < P1_ILP; i++) {
                const int r = lane + WARP * i;
                const uint64_t s = base + r;
                const bool valid = s < n_pos && (((r < 64 ? v0 : v1) >> (r & 63)) & 1);
                g[i] = valid ? s_pg[window_part<K>(P, s, k, part_bits)] : 0u;
                in[i] = valid && g[i] == rid_value;
            }
#pragma unroll
            for (int i = 0; i < P1_ILP; i++) {
                const uint32_t lo = __ballot_sync(FULL, g[i] & 1u), hi = __ballot_sync(FULL, (g[i] >> 1) & 1u);
                if (lane == 0) rid_out[4 * t + i] = (uint64_t)lo | ((uint64_t)hi << 32);
            }
        } else {
#pragma unroll
            for (int i = 0; i < P1_ILP; i++) {
                const int r = lane + WARP * i;
                const uint64_t s = base + r;
                in[i] = s < n_pos && (((r < 64 ? v0 : v1) >> (r & 63)) & 1);
                if (in[i] && rid) {  // the window's range id, written by the first range's pass
                    const uint32_t id = (uint32_t)(((rw[i] >> lane) & 1u) | (((rw[i] >> (32 + lane)) & 1u) << 1));
                    in[i] = id == rid_value;
                } else if (in[i]) {
                    const uint32_t pt = window_part<K>(P, s, k, part_bits);
                    in[i] = pt >= part_lo && pt < part_hi;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < P1_ILP; i++) {
            const uint32_t m = __ballot_sync(FULL, in[i]);
            if (in[i]) q[nq + __popc(m & lt)] = base + lane + WARP * i;
            nq += __popc(m);
        }
        __syncwarp();
        if (nq >= P1_TILE) {
            probe(P1_TILE);
            __syncwarp();
            const int rest = nq - P1_TILE;  // < P1_TILE: move the remainder to the front
            uint64_t tail[P1_ILP];
#pragma unroll
            for (int i = 0; i < P1_ILP; i++)
                if (lane + WARP * i < rest) tail[i] = q[P1_TILE + lane + WARP * i];
            __syncwarp();
#pragma unroll
            for (int i = 0; i < P1_ILP; i++)
                if (lane + WARP * i < rest) q[lane + WARP * i] = tail[i];
            __syncwarp();
            nq = rest;
        }
    }
    if (nq > 0) probe(nq);
    __syncwarp();
    hist_keys(wbuf, nbuf, s_hist, hist_passes, lane, bg, BY_BUCKET);
    flush_rest(wbuf, nbuf, cand, cand_count, cand_cap, err, lane);
    if (EMIT_FIRSTS) {
        if (BY_BUCKET) hist_keys(fbuf, nfirst, s_fhist, hist_passes, lane, bg, true);
        flush_rest(fbuf, nfirst, firsts, first_count, first_cap, err, lane, true);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_hist; i += P1_BLOCK)
        if (s_hist[i]) atomicAdd((unsigned long long *)&hist[i], (unsigned long long)s_hist[i]);
}

template <class K, bool F, bool E>
static auto pass1_by_mode(int mode) -> decltype(&k_pass1<K, F, E, 0>) {
    switch (mode) {  // the combinations the pipeline uses (batches are never split into key ranges)
    case P1_BATCHED: return k_pass1<K, F, E, P1_BATCHED>;
    case P1_PARTED: return k_pass1<K, F, E, P1_PARTED>;
    case P1_BY_BUCKET: return k_pass1<K, F, E, P1_BY_BUCKET>;
    case P1_BATCHED | P1_BY_BUCKET: return k_pass1<K, F, E, P1_BATCHED | P1_BY_BUCKET>;
    case P1_PARTED | P1_BY_BUCKET: return k_pass1<K, F, E, P1_PARTED | P1_BY_BUCKET>;
    case P1_BATCHED | P1_PARTED: return k_pass1<K, F, E, P1_BATCHED | P1_PARTED>;
    case P1_BATCHED | P1_PARTED | P1_BY_BUCKET: return k_pass1<K, F, E, P1_BATCHED | P1_PARTED | P1_BY_BUCKET>;
    default: return k_pass1<K, F, E, 0>;
    }
}
template <class K>
static auto pass1_kernel(bool use_filter, bool emit_firsts, int mode) -> decltype(&k_pass1<K, true, true, 0>) {
    if (emit_firsts) return pass1_by_mode<K, true, true>(mode);
    if (use_filter) return pass1_by_mode<K, true, false>(mode);
    return pass1_by_mode<K, false, false>(mode);
}

template <class K>
void launch_pass1(const LaunchCfg &c, const PackLayout &L, int k, const uint64_t *P, const uint64_t *V,
                  bool use_filter, const FilterGeom &f, K *cand, unsigned long long *cand_count, uint64_t cand_cap,
                  K *firsts, unsigned long long *first_count, uint64_t first_cap, uint64_t *hist, int hist_passes,
                  int part_bits, uint32_t part_lo, uint32_t part_hi, const uint64_t *lib_starts, int n_libs,
                  const uint64_t *lib_filter, uint32_t *err, const BucketGeom *bucket, uint64_t t_begin,
                  uint64_t t_end, const uint64_t *rid, uint32_t rid_value, const int *lib_k, int tag_shift,
                  uint64_t *rid_out, const uint8_t *part_group) {
    const uint64_t all_tiles = (L.n_bases + P1_TILE - 1) / P1_TILE;
    if (t_end > all_tiles) t_end = all_tiles;
    if (t_begin >= t_end) return;
    const uint64_t tiles = t_end - t_begin;
    const bool emit_firsts = use_filter && firsts != nullptr;
    if (!hist) hist_passes = 0;
    const BucketGeom bg = bucket ? *bucket : BucketGeom{};
    const int by_bucket = bucket != nullptr;
    const size_t smem = sizeof(K) * P1_BUF * P1_WARPS * (emit_firsts ? 2 : 1) +
                        4 * 256 * hist_passes * (by_bucket && emit_firsts ? 2 : 1) +
                        (use_filter ? sizeof(uint64_t) * (f.pat_mask + 1) : 0);
    if (part_bits && !n_libs && use_filter) {  // one key range of a library: the compacting form
        const size_t rsmem = sizeof(K) * P1_BUF * P1_WARPS * (emit_firsts ? 2 : 1) + 8 * PQ_CAP * P1_WARPS +
                             4 * 256 * hist_passes * (by_bucket && emit_firsts ? 2 : 1) +
                             sizeof(uint64_t) * (f.pat_mask + 1);
        auto rk = rid_out ? (emit_firsts ? (by_bucket ? k_pass1_range<K, true, true, true>
                                                      : k_pass1_range<K, true, false, true>)
                                         : (by_bucket ? k_pass1_range<K, false, true, true>
                                                      : k_pass1_range<K, false, false, true>))
                          : (emit_firsts ? (by_bucket ? k_pass1_range<K, true, true, false>
                                                      : k_pass1_range<K, true, false, false>)
                                         : (by_bucket ? k_pass1_range<K, false, true, false>
                                                      : k_pass1_range<K, false, false, false>));
        cudaFuncSetAttribute(rk, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rk, P1_BLOCK, rsmem);
        if (per_sm < 1) per_sm = 1;
        const uint64_t need = (tiles + P1_WARPS - 1) / P1_WARPS, cap = (uint64_t)c.sms * per_sm;
        rk<<<(int)(need < cap ? (need ? need : 1) : cap), P1_BLOCK, rsmem, c.stream>>>(
            P, V, L.n_bases, k, f.words, f.sector_shift, f.patterns, f.pat_mask, cand, cand_count, cand_cap, firsts,
            first_count, first_cap, hist, hist_passes, part_bits, part_lo, part_hi, rid, rid_value, rid_out,
            part_group, bg, t_begin, t_end, err);
        return;
    }
    const int mode = (n_libs ? P1_BATCHED : 0) | (part_bits ? P1_PARTED : 0) | (by_bucket ? P1_BY_BUCKET : 0);
    auto kern = pass1_kernel<K>(use_filter, emit_firsts, mode);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, P1_BLOCK, smem);
    if (per_sm < 1) per_sm = 1;
    uint64_t need = (tiles + P1_WARPS - 1) / P1_WARPS;
    uint64_t cap = (uint64_t)c.sms * per_sm;
    int grid = (int)(need < cap ? (need ? need : 1) : cap);
    kern<<<grid, P1_BLOCK, smem, c.stream>>>(P, V, L.n_bases, k, f.words, f.sector_shift, f.patterns, f.pat_mask,
                                             cand, cand_count, cand_cap, firsts, first_count, first_cap, hist,
                                             hist_passes, part_bits, part_lo, part_hi, lib_starts, n_libs,
                                             lib_filter, lib_k, tag_shift, bg, by_bucket, t_begin, t_end, err);
}

template <class K>
void launch_filter_keys(const LaunchCfg &c, const K *keys, uint64_t n, const FilterGeom &f, int set, uint8_t *seen) {
    uint64_t need = (n + 255) / 256;
    uint64_t cap = (uint64_t)c.sms * 8;
    int grid = (int)(need < cap ? (need ? need : 1) : cap);
    k_filter_keys<K><<<grid, 256, 0, c.stream>>>(keys, n, f.words, f.sector_shift, f.patterns, f.pat_mask, set, seen);
}

template void launch_pass1<uint64_t>(const LaunchCfg &, const PackLayout &, int, const uint64_t *, const uint64_t *,
                                     bool, const FilterGeom &, uint64_t *, unsigned long long *, uint64_t, uint64_t *,
                                     unsigned long long *, uint64_t, uint64_t *, int, int, uint32_t, uint32_t, const uint64_t *, int,
                                     const uint64_t *, uint32_t *, const BucketGeom *, uint64_t, uint64_t,
                                     const uint64_t *, uint32_t, const int *, int, uint64_t *, const uint8_t *);
template void launch_pass1<Key128>(const LaunchCfg &, const PackLayout &, int, const uint64_t *, const uint64_t *,
                                   bool, const FilterGeom &, Key128 *, unsigned long long *, uint64_t, Key128 *,
                                   unsigned long long *, uint64_t, uint64_t *, int, int, uint32_t, uint32_t,
                                   const uint64_t *, int, const uint64_t *, uint32_t *, const BucketGeom *, uint64_t,
                                   uint64_t, const uint64_t *, uint32_t, const int *, int, uint64_t *,
                                   const uint8_t *);
template void launch_filter_keys<uint64_t>(const LaunchCfg &, const uint64_t *, uint64_t, const FilterGeom &, int,
                                           uint8_t *);
template void launch_filter_keys<Key128>(const LaunchCfg &, const Key128 *, uint64_t, const FilterGeom &, int,
                                         uint8_t *);

// ---------------------------------------------------------------- pass 1, filter-blocked (binned) form
// The filter is far larger than L2, and in window order every probe lands on a random sector: most
// probes miss L2 and move a whole DRAM line. The Turtle filter is designed for caches (Sec. 2.1.3:
// one block per k-mer, so a probe touches one cache line); here the probes are also ORDERED so
// that the cache holds the blocks being probed. Window keys are first binned by the top 8 bits of
// their hash -- the top bits of their filter sector, so bin b holds exactly the keys whose blocks
// lie in the b-th 1/256 of the filter -- and then probed bin after bin by all warps together: at
// any moment the whole GPU works inside one or two bins, a few MiB of filter that stay in L2. The
// order in which windows test-and-set the filter does not change the result: every valid window
// still leaves as exactly one candidate or first sighting, and at most one occurrence of a key can
// be a first sighting (see above).
//   k_bin_count   extract + hash every valid (in-range) window, count it in its bin
//   (scan)        exact bin offsets
//   k_bin_scatter extract + hash again, rank inside the CTA's tile per bin, reserve each bin's run
//                 of slots with one atomic per bin and tile, write the keys
//   k_probe_bins  stream the binned keys in order: filter test-and-set and candidate / first-sighting
//                 emission exactly as in k_pass1 (same staging, same bucket-index histograms)
constexpr int BIN_BITS = 8;
constexpr int N_BINS = 1 << BIN_BITS;
constexpr int BT_THREADS = 256;
constexpr int BT_ITEMS = 16;                   // positions per thread per tile
constexpr int BT_POS = BT_THREADS * BT_ITEMS;  // 4096 positions per tile: 64 validity words
static_assert(BT_THREADS == N_BINS, "one thread per bin in the scatter's reservation step");

__device__ __forceinline__ uint32_t bin_of(uint64_t h) { return (uint32_t)(h >> (64 - BIN_BITS)); }

// Validity words of the tile starting at position `base` into s_v (words past the bitmap read as 0).
__device__ __forceinline__ void load_tile_valid(const uint64_t *__restrict__ V, uint64_t base, uint64_t n_vwords,
                                                uint64_t *s_v) {
    if (threadIdx.x < BT_POS / 64) {
        const uint64_t w = base / 64 + threadIdx.x;
        s_v[threadIdx.x] = w < n_vwords ? V[w] : 0ull;
    }
}

template <class K, bool PARTED>
__global__ void __launch_bounds__(BT_THREADS) k_bin_count(const uint64_t *__restrict__ P, const uint64_t *__restrict__ V,
                                                          uint64_t n_pos, int k, int part_bits, uint32_t part_lo,
                                                          uint32_t part_hi, unsigned long long *bin_count) {
    __shared__ uint32_t s_hist[N_BINS];
    __shared__ uint64_t s_v[BT_POS / 64];
    const int tid = threadIdx.x;
    s_hist[tid] = 0;
    const uint64_t tiles = (n_pos + BT_POS - 1) / BT_POS, n_vwords = (n_pos + 63) / 64;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint64_t base = t * BT_POS;
        __syncthreads();
        load_tile_valid(V, base, n_vwords, s_v);
        __syncthreads();
#pragma unroll 4
        for (int i = 0; i < BT_ITEMS; i++) {
            const int r = tid + BT_THREADS * i;
            const uint64_t s = base + r;
            if (s >= n_pos || !((s_v[r >> 6] >> (r & 63)) & 1)) continue;
            const K key = canonical<K>(P, s, k);
            if (PARTED) {
                const uint32_t pt = key_part(key, k, part_bits);
                if (pt < part_lo || pt >= part_hi) continue;
            }
            atomicAdd(&s_hist[bin_of(key_hash(key))], 1u);
        }
    }
    __syncthreads();
    if (s_hist[tid]) atomicAdd(&bin_count[tid], (unsigned long long)s_hist[tid]);
}

// The tile's keys are first placed in shared memory grouped by bin (bin-major, each bin's keys in one
// run), so that the writes of one bin's run are consecutive addresses: a warp's stores coalesce into
// a few requests instead of one request per key.
template <class K, bool PARTED>
__global__ void __launch_bounds__(BT_THREADS) k_bin_scatter(const uint64_t *__restrict__ P,
                                                            const uint64_t *__restrict__ V, uint64_t n_pos, int k,
                                                            int part_bits, uint32_t part_lo, uint32_t part_hi,
                                                            unsigned long long *cursor,
                                                            const unsigned long long *__restrict__ bin_off,
                                                            K *__restrict__ out, uint64_t out_cap, uint32_t *err) {
    extern __shared__ __align__(16) unsigned char bs_smem[];
    K *s_key = reinterpret_cast<K *>(bs_smem);                            // BT_POS keys, grouped by bin
    uint8_t *s_bin = reinterpret_cast<uint8_t *>(s_key + BT_POS);         // bin of each staged key
    __shared__ uint32_t s_cnt[N_BINS], s_start[N_BINS], s_scan[BT_THREADS / WARP];
    __shared__ unsigned long long s_base[N_BINS];
    __shared__ uint64_t s_v[BT_POS / 64];
    __shared__ uint32_t s_total;
    const int tid = threadIdx.x;
    const uint64_t tiles = (n_pos + BT_POS - 1) / BT_POS, n_vwords = (n_pos + 63) / 64;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint64_t base = t * BT_POS;
        __syncthreads();
        s_cnt[tid] = 0;
        load_tile_valid(V, base, n_vwords, s_v);
        __syncthreads();
        K key[BT_ITEMS];
        uint32_t slot[BT_ITEMS];  // bin | rank << 8 inside the tile's run of that bin; ~0 = no key
#pragma unroll
        for (int i = 0; i < BT_ITEMS; i++) {
            const int r = tid + BT_THREADS * i;
            const uint64_t s = base + r;
            slot[i] = ~0u;
            if (s >= n_pos || !((s_v[r >> 6] >> (r & 63)) & 1)) continue;
            key[i] = canonical<K>(P, s, k);
            if (PARTED) {
                const uint32_t pt = key_part(key[i], k, part_bits);
                if (pt < part_lo || pt >= part_hi) continue;
            }
            const uint32_t b = bin_of(key_hash(key[i]));
            slot[i] = b | (atomicAdd(&s_cnt[b], 1u) << BIN_BITS);
        }
        __syncthreads();
        // thread b: the start of bin b's run in the staging area, and its slots in the output
        const uint32_t cnt = s_cnt[tid];
        uint32_t total;
        const uint32_t st = block_exclusive_scan<BT_THREADS>(cnt, s_scan, &total);
        s_start[tid] = st;
        if (cnt) s_base[tid] = atomicAdd(&cursor[tid], (unsigned long long)cnt);
        if (tid == 0) s_total = total;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < BT_ITEMS; i++) {
            if (slot[i] == ~0u) continue;
            const uint32_t b = slot[i] & (N_BINS - 1), j = s_start[b] + (slot[i] >> BIN_BITS);
            s_key[j] = key[i];
            s_bin[j] = (uint8_t)b;
        }
        __syncthreads();
        // consecutive staged keys of one bin go to consecutive output slots
        for (uint32_t j = tid; j < s_total; j += BT_THREADS) {
            const uint32_t b = s_bin[j];
            const unsigned long long o = s_base[b] + (j - s_start[b]);
            if (o < bin_off[b + 1] && o < out_cap) store_key(out + o, s_key[j]);  // the counting pass sized every bin
            else atomicOr(err, ERR_CAND_OVERFLOW);
        }
    }
}

template <class K, bool EMIT_FIRSTS, bool BY_BUCKET>
__global__ void __launch_bounds__(P1_BLOCK, sizeof(K) == 8 ? 4 : 2) k_probe_bins(const K *__restrict__ keys, const unsigned long long *n_keys,
                                                         uint64_t *filter, int sector_shift,
                                                         const uint64_t *__restrict__ patterns, uint32_t pat_mask,
                                                         K *cand, unsigned long long *cand_count, uint64_t cand_cap,
                                                         K *firsts, unsigned long long *first_count,
                                                         uint64_t first_cap, uint64_t *hist, int hist_passes,
                                                         BucketGeom bg, uint32_t *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NBUF = EMIT_FIRSTS ? 2 : 1;
    const int n_hist = 256 * hist_passes * (BY_BUCKET && EMIT_FIRSTS ? 2 : 1);
    K *s_buf = reinterpret_cast<K *>(smem);
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(smem + sizeof(K) * P1_BUF * P1_WARPS * NBUF);
    uint32_t *s_fhist = s_hist + 256 * hist_passes;
    uint64_t *s_pat = reinterpret_cast<uint64_t *>(s_hist + n_hist);
    for (uint32_t i = threadIdx.x; i <= pat_mask; i += P1_BLOCK) s_pat[i] = patterns[i];
    for (int i = threadIdx.x; i < n_hist; i += P1_BLOCK) s_hist[i] = 0;
    __syncthreads();
    const uint64_t n = *n_keys;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    K *wbuf = s_buf + warp * P1_BUF * NBUF;
    K *fbuf = wbuf + P1_BUF;
    int nbuf = 0, nfirst = 0;
    // every warp of the grid takes the next 128 keys: together they sweep the bins front to back. The
    // keys of a warp's next chunk are loaded while the current chunk is probed.
    const uint64_t stride = (uint64_t)gridDim.x * P1_WARPS;
    uint64_t t = (uint64_t)blockIdx.x * P1_WARPS + warp;
    K next[P1_ILP];
#pragma unroll
    for (int i = 0; i < P1_ILP; i++) {
        const uint64_t j = t * P1_TILE + lane + WARP * i;
        if (j < n) next[i] = load_stream(keys + j);
    }
    for (; t * P1_TILE < n; t += stride) {
        const uint64_t base = t * P1_TILE;
        bool ok[P1_ILP];
        K key[P1_ILP];
#pragma unroll
        for (int i = 0; i < P1_ILP; i++) {
            ok[i] = base + lane + WARP * i < n;
            key[i] = next[i];
            const uint64_t j = base + stride * P1_TILE + lane + WARP * i;
            if (j < n) next[i] = load_stream(keys + j);
        }
        // the probed blocks are in L2 (the bins are swept in order), so the test-and-set goes straight to
        // the atomic: its old value says whether every pattern bit was already set
        bool seen[P1_ILP];
        uint64_t old[P1_ILP], mask[P1_ILP];
#pragma unroll
        for (int i = 0; i < P1_ILP; i++) {
            if (ok[i]) {
                const uint64_t h = key_hash(key[i]);
                const uint64_t sector = sector_shift < 64 ? (h >> sector_shift) : 0;
                mask[i] = s_pat[h & pat_mask];
                old[i] = atomicOr((unsigned long long *)(filter + sector * 4 + ((h >> 16) & 3)),
                                  (unsigned long long)mask[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < P1_ILP; i++) seen[i] = ok[i] && (old[i] & mask[i]) == mask[i];
#pragma unroll
        for (int i = 0; i < P1_ILP; i++) {
            const uint32_t b = __ballot_sync(FULL, seen[i]);
            if (seen[i]) wbuf[nbuf + __popc(b & lt)] = key[i];
            nbuf += __popc(b);
            if (nbuf >= P1_STAGE) {
                __syncwarp();
                hist_keys(wbuf, P1_STAGE, s_hist, hist_passes, lane, bg, BY_BUCKET);
                flush_full(wbuf, nbuf, cand, cand_count, cand_cap, err, lane);
            }
            if (EMIT_FIRSTS) {
                const bool f = ok[i] && !seen[i];
                const uint32_t bf = __ballot_sync(FULL, f);
                if (f) fbuf[nfirst + __popc(bf & lt)] = key[i];
                nfirst += __popc(bf);
                if (nfirst >= P1_STAGE) {
                    if (BY_BUCKET) {
                        __syncwarp();
                        hist_keys(fbuf, P1_STAGE, s_fhist, hist_passes, lane, bg, true);
                    }
                    flush_full(fbuf, nfirst, firsts, first_count, first_cap, err, lane, true);
                }
            }
        }
    }
    __syncwarp();
    hist_keys(wbuf, nbuf, s_hist, hist_passes, lane, bg, BY_BUCKET);
    flush_rest(wbuf, nbuf, cand, cand_count, cand_cap, err, lane);
    if (EMIT_FIRSTS) {
        if (BY_BUCKET) hist_keys(fbuf, nfirst, s_fhist, hist_passes, lane, bg, true);
        flush_rest(fbuf, nfirst, firsts, first_count, first_cap, err, lane, true);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_hist; i += P1_BLOCK)
        if (s_hist[i]) atomicAdd((unsigned long long *)&hist[i], (unsigned long long)s_hist[i]);
}

uint64_t pass1_bin_words() { return 3 * (N_BINS + 1); }

template <class K>
void launch_pass1_binned(const LaunchCfg &c, const PackLayout &L, int k, const uint64_t *P, const uint64_t *V,
                         const FilterGeom &f, K *bin_keys, uint64_t bin_cap, unsigned long long *bin_words, K *cand,
                         unsigned long long *cand_count, uint64_t cand_cap, K *firsts,
                         unsigned long long *first_count, uint64_t first_cap, uint64_t *hist, int hist_passes,
                         int part_bits, uint32_t part_lo, uint32_t part_hi, uint32_t *err, const BucketGeom *bucket) {
    unsigned long long *count = bin_words, *off = bin_words + (N_BINS + 1), *cursor = bin_words + 2 * (N_BINS + 1);
    cudaMemsetAsync(count, 0, sizeof(unsigned long long) * N_BINS, c.stream);
    const uint64_t tiles = (L.n_bases + BT_POS - 1) / BT_POS;
    if (tiles) {
        auto kc = part_bits ? k_bin_count<K, true> : k_bin_count<K, false>;
        auto ks = part_bits ? k_bin_scatter<K, true> : k_bin_scatter<K, false>;
        const size_t smem = (sizeof(K) + 1) * BT_POS;
        cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm_c = 0, per_sm_s = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_c, kc, BT_THREADS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_s, ks, BT_THREADS, smem);
        const int grid_c = (int)std::min<uint64_t>(tiles, (uint64_t)c.sms * std::max(per_sm_c, 1));
        const int grid_s = (int)std::min<uint64_t>(tiles, (uint64_t)c.sms * std::max(per_sm_s, 1));
        kc<<<grid_c, BT_THREADS, 0, c.stream>>>(P, V, L.n_bases, k, part_bits, part_lo, part_hi, count);
        launch_scan_u64(c, count, N_BINS, off);
        cudaMemcpyAsync(cursor, off, sizeof(unsigned long long) * N_BINS, cudaMemcpyDeviceToDevice, c.stream);
        ks<<<grid_s, BT_THREADS, smem, c.stream>>>(P, V, L.n_bases, k, part_bits, part_lo, part_hi, cursor, off,
                                                   bin_keys, bin_cap, err);
    } else {
        cudaMemsetAsync(off, 0, sizeof(unsigned long long) * (N_BINS + 1), c.stream);
    }
    const bool emit_firsts = firsts != nullptr;
    if (!hist) hist_passes = 0;
    const BucketGeom bg = bucket ? *bucket : BucketGeom{};
    const bool by_bucket = bucket != nullptr;
    const size_t smem = sizeof(K) * P1_BUF * P1_WARPS * (emit_firsts ? 2 : 1) +
                        4 * 256 * hist_passes * (by_bucket && emit_firsts ? 2 : 1) + sizeof(uint64_t) * (f.pat_mask + 1);
    auto kp = emit_firsts ? (by_bucket ? k_probe_bins<K, true, true> : k_probe_bins<K, true, false>)
                          : (by_bucket ? k_probe_bins<K, false, true> : k_probe_bins<K, false, false>);
    cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kp, P1_BLOCK, smem);
    if (per_sm < 1) per_sm = 1;
    const uint64_t need = (L.n_bases / P1_TILE + P1_WARPS) / P1_WARPS;  // keys <= positions
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)c.sms * per_sm));
    kp<<<grid, P1_BLOCK, smem, c.stream>>>(bin_keys, off + N_BINS, f.words, f.sector_shift, f.patterns, f.pat_mask, cand,
                                           cand_count, cand_cap, firsts, first_count, first_cap, hist, hist_passes, bg,
                                           err);
}

template void launch_pass1_binned<uint64_t>(const LaunchCfg &, const PackLayout &, int, const uint64_t *,
                                            const uint64_t *, const FilterGeom &, uint64_t *, uint64_t,
                                            unsigned long long *, uint64_t *, unsigned long long *, uint64_t, uint64_t *,
                                            unsigned long long *, uint64_t, uint64_t *, int, int, uint32_t, uint32_t,
                                            uint32_t *, const BucketGeom *);
template void launch_pass1_binned<Key128>(const LaunchCfg &, const PackLayout &, int, const uint64_t *,
                                          const uint64_t *, const FilterGeom &, Key128 *, uint64_t,
                                          unsigned long long *, Key128 *, unsigned long long *, uint64_t, Key128 *,
                                          unsigned long long *,
                                          uint64_t, uint64_t *, int, int, uint32_t, uint32_t, uint32_t *,
                                          const BucketGeom *);

}  // namespace turtle
