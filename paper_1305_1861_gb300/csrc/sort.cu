// Step a4: sort-and-compact of the candidate keys (Sec. 2.1.4, Alg. 1).
//
// The paper sorts its candidate array in place with a comparison sort and then
// merges runs of equal keys. On the GPU the sort is a least-significant-digit
// radix sort in the onesweep style (Adinets & Merrill 2022): one kernel reads the
// keys once and builds the 256-bin histograms of every 8-bit digit; then each
// digit pass is ONE kernel in which a tile ranks its keys locally (warp ballots +
// per-warp counters, stable), publishes its per-digit counts, obtains the counts
// of all earlier tiles through decoupled look-back (one status chain per digit)
// and scatters its keys, staged through shared memory so that each run of equal
// digits is written contiguously. Each pass reads and writes every key once.
// Run-length compaction then keeps the first key of each run (flag = key differs
// from its predecessor) with an order-preserving single-pass scan.
#include "bucket.cuh"

namespace turtle {

constexpr int S_BLOCK = 256;
constexpr int S_WARPS = S_BLOCK / WARP;
constexpr int BINS = 256;
constexpr int MAX_PASSES = 16;

// Onesweep tile shapes (keys per thread, CTAs per SM), selected at run time (params.sort_tile).
// Variant 0 is the default; the others trade tile size against occupancy.
template <class K> struct SortCfg;
constexpr int min3(const int (&v)[3]) { return v[0] < v[1] ? (v[0] < v[2] ? v[0] : v[2]) : (v[1] < v[2] ? v[1] : v[2]); }
// Variant 3 (BULK_VARIANT) is the persistent form with bulk-copied tiles, BULK_ITEMS keys per thread,
// 2 CTAs/SM.
template <> struct SortCfg<uint64_t> {
    static constexpr int V_ITEMS[3] = {32, 16, 24};  // default: 8192 keys (64 KB) per tile, 2 CTAs/SM
    static constexpr int V_MINB[3] = {2, 4, 2};
    static constexpr int BULK_ITEMS = 16;
    static constexpr int MIN_TILE = 256 * min3(V_ITEMS);  // sizes the look-back status array
};
template <> struct SortCfg<Key128> {
    static constexpr int V_ITEMS[3] = {16, 8, 12};   // default: 4096 keys (64 KB) per tile
    static constexpr int V_MINB[3] = {2, 3, 2};
    static constexpr int BULK_ITEMS = 8;
    static constexpr int MIN_TILE = 256 * min3(V_ITEMS);
};
constexpr int BULK_VARIANT = 3;

int sort_passes_for(int key_bits) { return (key_bits + 7) / 8; }

uint64_t sort_lookback_words(uint64_t n, int key_words) {  // sized for the smallest tile of any variant
    const uint64_t tile = key_words == 1 ? SortCfg<uint64_t>::MIN_TILE : SortCfg<Key128>::MIN_TILE;
    return ((n + tile - 1) / tile + 1) * BINS;
}

template <class K, class D>
__global__ void __launch_bounds__(S_BLOCK) k_hist(const K *__restrict__ keys, uint64_t n, int passes,
                                                  uint64_t *__restrict__ hist, D dig) {
    __shared__ uint32_t sh[MAX_PASSES * BINS];
    for (int i = threadIdx.x; i < passes * BINS; i += S_BLOCK) sh[i] = 0;
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)S_BLOCK + threadIdx.x; i < n; i += (uint64_t)gridDim.x * S_BLOCK) {
        const K key = keys[i];
        for (int p = 0; p < passes; p++) atomicAdd(&sh[p * BINS + dig(key, 8 * p)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * BINS; i += S_BLOCK)
        if (sh[i]) atomicAdd((unsigned long long *)&hist[i], (unsigned long long)sh[i]);
}

// hist[p][d] -> exclusive prefix over d (in place). One block per pass.
__global__ void k_scan_bins(uint64_t *hist) {
    __shared__ uint64_t s[BINS];
    uint64_t *h = hist + (uint64_t)blockIdx.x * BINS;
    s[threadIdx.x] = h[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t run = 0;
        for (int d = 0; d < BINS; d++) {
            const uint64_t v = s[d];
            s[d] = run;
            run += v;
        }
    }
    __syncthreads();
    h[threadIdx.x] = s[threadIdx.x];
}

// Shared state of one onesweep tile, besides the staged keys and their digits.
struct OsShared {
    uint32_t whist[S_WARPS][BINS];  // per-warp digit counters
    uint32_t texcl[BINS];
    uint64_t glob[BINS];
    uint32_t scan[S_WARPS];
    uint32_t uniform;
};

// One onesweep tile: keys src[0 .. min(TILE, n - start)) (global memory, or a shared-memory copy) are
// ranked by digit into skeys/sdig and scattered to out. On entry sh.whist is zero and a barrier has
// passed since; skeys may be the buffer src points into (every read of src ends before the first
// barrier here, every write of skeys comes after it). The caller synchronises before reusing skeys,
// sdig or sh.
//
// STABLE = false: the first pass of a sort, whose input order carries no information. Each key
// then takes its place with one shared-memory atomic on its warp's digit counter, in any order
// among the warp's keys of the same digit, without the warp match and broadcast.
template <class K, int ITEMS, class D, bool STABLE>
__device__ __forceinline__ void onesweep_tile(const K *src, uint64_t start, uint64_t n, K *skeys, uint8_t *sdig,
                                              OsShared &sh, K *__restrict__ out, int shift,
                                              const uint64_t *__restrict__ bin_base, uint64_t *lookback,
                                              uint64_t tile, uint32_t epoch, uint32_t *err, D digit) {
    constexpr int TILE = S_BLOCK * ITEMS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t wofs = (uint32_t)warp * ITEMS * WARP;  // warp w owns a contiguous run of the tile
    const uint32_t lt = lanemask_lt();

    // A full tile (every tile but the last) needs no bounds checks.
    const bool full = start + TILE <= n;
    const uint64_t wstart = start + wofs;
    const uint32_t n_in_warp = full ? (uint32_t)(ITEMS * WARP)
                                    : (uint32_t)(wstart >= n ? 0 : (n - wstart < (uint64_t)ITEMS * WARP ? n - wstart
                                                                                                       : ITEMS * WARP));
    K key[ITEMS];
    uint32_t dig[(ITEMS + 3) / 4];  // digits packed four to a register, computed once
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
        const uint32_t r = (uint32_t)(i * WARP + lane);
        if (full || r < n_in_warp) key[i] = src[wofs + r];
    }
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
        const uint32_t r = (uint32_t)(i * WARP + lane);
        const uint32_t d = (full || r < n_in_warp) ? digit(key[i], shift) : 0u;
        if ((i & 3) == 0) dig[i >> 2] = d;
        else dig[i >> 2] |= d << (8 * (i & 3));
    }
    // A stable pass's input is sorted by the lower digits, so its tile holds one value of them
    // exactly when the tile's first and last keys agree. Then no two keys of the tile need a
    // relative order (equal digits there mean equal sort keys so far), and the tile ranks like a
    // first pass: one shared atomic per key.
    if (STABLE && tid == 0) {
        const uint64_t last = (full ? TILE : n - start) - 1;
        sh.uniform = digit.same_low(src[0], src[last], shift) ? 1u : 0u;
    }
    // 1. early counts: per-warp digit counts (order-free shared atomics)
#pragma unroll
    for (int i = 0; i < ITEMS; i++)
        if (full || (uint32_t)(i * WARP + lane) < n_in_warp)
            atomicAdd(&sh.whist[warp][(dig[i >> 2] >> (8 * (i & 3))) & 0xffu], 1u);
    __syncthreads();
    // 2. thread tid owns digit tid: tile count, publish it, tile-local start, per-warp starts
    uint32_t tcount = 0;
#pragma unroll
    for (int w = 0; w < S_WARPS; w++) tcount += sh.whist[w][tid];
    if (tile > 0) st_relaxed(lookback + tile * BINS + tid, lb_pack(LB_AGG, epoch, tcount));
    const uint32_t texcl = block_exclusive_scan<S_BLOCK>(tcount, sh.scan, nullptr);
    sh.texcl[tid] = texcl;
    {
        uint32_t run = texcl;
#pragma unroll
        for (int w = 0; w < S_WARPS; w++) {
            const uint32_t v = sh.whist[w][tid];
            sh.whist[w][tid] = run;
            run += v;
        }
    }
    __syncthreads();
    // 3. ranking straight into shared memory. Unstable (a first pass, or a tile with one value of
    //    the lower digits): one shared atomic per key. Stable: rows in order, lanes in order within
    //    a row, equal digits found by ballots.
    const bool by_atomics = !STABLE || sh.uniform;  // read after the barriers that follow its write
    if (by_atomics) {
#pragma unroll
        for (int i = 0; i < ITEMS; i++) {
            if (full || (uint32_t)(i * WARP + lane) < n_in_warp) {
                const uint32_t d = (dig[i >> 2] >> (8 * (i & 3))) & 0xffu;
                const uint32_t pos = atomicAdd(&sh.whist[warp][d], 1u);
                skeys[pos] = key[i];
                sdig[pos] = (uint8_t)d;
            }
        }
    } else if (STABLE) {
#pragma unroll
        for (int i = 0; i < ITEMS; i++) {
            const bool valid = full || (uint32_t)(i * WARP + lane) < n_in_warp;
            const uint32_t d = valid ? ((dig[i >> 2] >> (8 * (i & 3))) & 0xffu) : (BINS + lane);
            uint32_t peers = FULL;  // lanes whose digit equals this lane's: one ballot per digit bit
#pragma unroll
            for (int b = 0; b < 9; b++) {
                if (b == 8 && full) break;  // bit 8 only separates the invalid lanes of a partial tile
                const bool bit = (d >> b) & 1u;
                const uint32_t bal = __ballot_sync(FULL, bit);
                peers &= bit ? bal : ~bal;
            }
            // Every peer reads the warp's counter for its digit; then the group's highest lane advances
            // it by the group size (one writer per digit: the warp owns its counters).
            const int leader = 31 - __clz(peers);
            uint32_t pos = 0;
            if (valid) pos = sh.whist[warp][d];
            __syncwarp();
            if (valid && lane == leader) sh.whist[warp][d] = pos + (uint32_t)__popc(peers);
            __syncwarp();
            if (valid) {
                skeys[pos + __popc(peers & lt)] = key[i];
                sdig[pos + __popc(peers & lt)] = (uint8_t)d;
            }
        }
    }
    // 4. global offsets of this tile's digits (predecessors have usually published by now)
    const uint64_t excl = lookback_prefix(lookback + tid, BINS, tile, tcount, epoch, err);
    sh.glob[tid] = bin_base[tid] + excl - texcl;
    __syncthreads();
    if (full) {
#pragma unroll 4
        for (uint32_t p = tid; p < (uint32_t)TILE; p += S_BLOCK) {
            out[sh.glob[sdig[p]] + p] = skeys[p];
        }
    } else {
        const uint32_t tile_n = (uint32_t)(n - start);
        for (uint32_t p = tid; p < tile_n; p += S_BLOCK) {
            out[sh.glob[sdig[p]] + p] = skeys[p];
        }
    }
}

// One CTA per tile, the tile's keys loaded by its threads.
template <class K, int ITEMS, int MINB, class D, bool STABLE>
__global__ void __launch_bounds__(S_BLOCK, MINB) k_onesweep(const K *__restrict__ in, K *__restrict__ out, uint64_t n,
                                                            int shift, const uint64_t *__restrict__ bin_base,
                                                            uint64_t *lookback, uint32_t *tile_ctr, uint32_t epoch,
                                                            uint32_t *err, D digit) {
    constexpr int TILE = S_BLOCK * ITEMS;
    extern __shared__ __align__(16) unsigned char os_smem[];
    K *skeys = reinterpret_cast<K *>(os_smem);  // TILE keys (dynamic: up to 64 KB)
    __shared__ uint8_t sdig[TILE];  // digit of each staged key: the scatter does not recompute it
    __shared__ OsShared sh;
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x;
    for (int i = tid; i < S_WARPS * BINS; i += S_BLOCK) (&sh.whist[0][0])[i] = 0;
    if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);  // tiles start in launch order: look-back always progresses
    __syncthreads();
    const uint64_t tile = s_tile, start = tile * TILE;
    onesweep_tile<K, ITEMS, D, STABLE>(in + start, start, n, skeys, sdig, sh, out, shift, bin_base, lookback, tile,
                                       epoch, err, digit);
}

// ---------------------------------------------------------------- bulk-copy (TMA) tile loads
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Make the barriers' initialisation visible to the copy engine.
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// Order this thread's earlier generic accesses of shared memory before later bulk copies into it.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from global to shared memory,
// completing on `bar`, which expects this many bytes in its current phase.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
// Wait until `bar` has completed the phase of the given parity: at most `limit` polls, each of
// which may suspend the thread for a short, hardware-defined time. False when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit) {
    const uint32_t a = smem_addr(bar);
    for (uint32_t i = 0; i < limit; i++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
constexpr uint32_t BULK_WAIT_LIMIT = 1u << 22;
constexpr uint32_t NO_BULK = ~0u;

// Persistent form: each CTA takes tiles by ticket, and while it ranks and scatters one tile the copy
// engine already loads its next one into the other of two shared-memory buffers (cp.async.bulk,
// completion counted on an mbarrier), so the next tile's loads do not wait for this one's scatter. A
// tile is taken before the one it prefetches is processed and every CTA processes its current tile
// before its prefetched one, so the lowest unfinished ticket is always some CTA's current tile and the
// look-back chain always progresses. The buffer a tile was loaded into also stages its ranked keys.
// Bulk copies need 16-byte aligned addresses: a tile of 64-bit keys that starts between two 16-byte
// boundaries is copied from the boundary below, one key earlier; the first and the last full tile,
// where that could read outside the keys, and a partial last tile are loaded by the threads.
template <class K, int ITEMS, class D, bool STABLE>
__global__ void __launch_bounds__(S_BLOCK, 2) k_onesweep_bulk(const K *__restrict__ in, K *__restrict__ out,
                                                              uint64_t n, int shift,
                                                              const uint64_t *__restrict__ bin_base,
                                                              uint64_t *lookback, uint32_t *tile_ctr, uint32_t epoch,
                                                              uint32_t *err, D digit) {
    constexpr int TILE = S_BLOCK * ITEMS;
    constexpr int SLACK = 16 / (int)sizeof(K) - 1;  // keys before and after a tile copied from a boundary
    constexpr int BUF = TILE + 2 * SLACK;
    extern __shared__ __align__(16) unsigned char os_smem[];
    K *buf[2] = {reinterpret_cast<K *>(os_smem), reinterpret_cast<K *>(os_smem) + BUF};
    uint8_t *sdig = reinterpret_cast<uint8_t *>(reinterpret_cast<K *>(os_smem) + 2 * BUF);
    __shared__ OsShared sh;
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t s_tile[2], s_off[2];  // tile staged in each buffer; its key offset, or NO_BULK
    const int tid = threadIdx.x;
    const uint64_t tiles = (n + TILE - 1) / TILE;

    // tid 0: take the next ticket into buffer b and start its copy (full tiles whose aligned span
    // stays inside the keys)
    auto stage = [&](int b) {
        const uint32_t t = atomicAdd(tile_ctr, 1u);
        uint32_t how = NO_BULK;
        if (t < tiles) {
            const uint64_t start = (uint64_t)t * TILE;
            const uint32_t off = (uint32_t)((reinterpret_cast<uintptr_t>(in + start) & 15) / sizeof(K));
            const uint32_t bytes = (uint32_t)(((uint64_t)(TILE + off) * sizeof(K) + 15) & ~(uint64_t)15);
            const bool aligned = (reinterpret_cast<uintptr_t>(in + (start - off)) & 15) == 0;
            if (aligned && start >= off && start - off + bytes / sizeof(K) <= n) {
                bulk_load(buf[b], in + (start - off), bytes, &s_bar[b]);
                how = off;
            }
        }
        s_tile[b] = t;
        s_off[b] = how;
    };
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        mbar_init_fence();
        stage(0);
    }
    uint32_t parity = 0;  // bit b: parity of buffer b's next phase
    int cur = 0;
    for (;;) {
        for (int i = tid; i < S_WARPS * BINS; i += S_BLOCK) (&sh.whist[0][0])[i] = 0;
        __syncthreads();  // the previous tile is done with every buffer and with sh; s_tile/s_off visible
        const uint32_t t = s_tile[cur], off = s_off[cur];
        if (t >= tiles) break;  // nothing was copied for a ticket past the last tile
        if (tid == 0) stage(cur ^ 1);  // buffer cur ^ 1 held the previous tile, now finished
        const uint64_t start = (uint64_t)t * TILE;
        const K *src = in + start;
        if (off != NO_BULK) {
            const bool ok = mbar_wait(&s_bar[cur], (parity >> cur) & 1u, BULK_WAIT_LIMIT);
            parity ^= 1u << cur;
            if (__syncthreads_or(!ok)) {  // a copy did not land in time: flag it, let the copies end, stop
                if (tid == 0) {
                    atomicOr(err, ERR_BULK_WAIT);
                    mbar_wait(&s_bar[cur], ((parity >> cur) & 1u) ^ 1u, BULK_WAIT_LIMIT);
                    if (s_off[cur ^ 1] != NO_BULK)  // the prefetch this thread started above
                        mbar_wait(&s_bar[cur ^ 1], (parity >> (cur ^ 1)) & 1u, BULK_WAIT_LIMIT);
                }
                return;
            }
            src = buf[cur] + off;
        }
        onesweep_tile<K, ITEMS, D, STABLE>(src, start, n, buf[cur], sdig, sh, out, shift, bin_base, lookback, t,
                                           epoch, err, digit);
        fence_proxy_async_smem();  // this thread's accesses of buf[cur] come before the copy that reuses it
        cur ^= 1;
    }
}

template <class K, int V, class D, bool STABLE>
static void onesweep_launch(const LaunchCfg &c, const K *src, K *dst, uint64_t n, int shift, const uint64_t *bin_base,
                            uint64_t *lookback, uint32_t *tile_ctr, uint32_t epoch, uint32_t *err, D digit) {
    if constexpr (V == BULK_VARIANT) {
        constexpr int ITEMS = SortCfg<K>::BULK_ITEMS, TILE = S_BLOCK * ITEMS;
        static_assert(TILE >= SortCfg<K>::MIN_TILE, "look-back array sized for larger tiles");
        const uint64_t tiles = (n + TILE - 1) / TILE;
        const size_t smem = 2 * sizeof(K) * (TILE + 2 * (16 / sizeof(K) - 1)) + TILE;
        auto kern = k_onesweep_bulk<K, ITEMS, D, STABLE>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, S_BLOCK, smem);
        if (per_sm < 1) per_sm = 1;
        const uint64_t cap = (uint64_t)c.sms * per_sm;
        kern<<<(int)(tiles < cap ? tiles : cap), S_BLOCK, smem, c.stream>>>(src, dst, n, shift, bin_base, lookback,
                                                                           tile_ctr, epoch, err, digit);
        return;
    }
    constexpr int VV = V < 3 ? V : 0;
    constexpr int ITEMS = SortCfg<K>::V_ITEMS[VV], MINB = SortCfg<K>::V_MINB[VV];
    static_assert(S_BLOCK * ITEMS >= SortCfg<K>::MIN_TILE, "look-back array sized for larger tiles");
    const uint64_t tiles = (n + S_BLOCK * ITEMS - 1) / (S_BLOCK * ITEMS);
    const size_t smem = sizeof(K) * S_BLOCK * ITEMS;
    auto kern = k_onesweep<K, ITEMS, MINB, D, STABLE>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<(int)tiles, S_BLOCK, smem, c.stream>>>(src, dst, n, shift, bin_base, lookback, tile_ctr, epoch, err, digit);
}

// One digit pass; stable = false for the first pass of a sort.
template <class K, int V, class D = RawDigit<K>>
static void onesweep_pass(const LaunchCfg &c, const K *src, K *dst, uint64_t n, int shift, const uint64_t *bin_base,
                          uint64_t *lookback, uint32_t *tile_ctr, uint32_t epoch, uint32_t *err, D digit = D{},
                          bool stable = true) {
    if (stable) onesweep_launch<K, V, D, true>(c, src, dst, n, shift, bin_base, lookback, tile_ctr, epoch, err, digit);
    else onesweep_launch<K, V, D, false>(c, src, dst, n, shift, bin_base, lookback, tile_ctr, epoch, err, digit);
}

template <class K>
K *launch_radix_sort(const LaunchCfg &c, K *keys, uint64_t n, int key_bits, const SortScratch &s, uint32_t *err,
                     bool hist_ready, uint32_t skip_mask, int *passes_run, int variant) {
    const int passes = sort_passes_for(key_bits);
    if (passes_run) *passes_run = 0;
    if (n <= 1 || passes == 0) return keys;
    if (variant < 0 || variant > BULK_VARIANT) variant = 0;
    const uint64_t TILE = (uint64_t)S_BLOCK * (variant == BULK_VARIANT ? SortCfg<K>::BULK_ITEMS
                                                                       : SortCfg<K>::V_ITEMS[variant]);
    const uint64_t tiles = (n + TILE - 1) / TILE;
    cudaMemsetAsync(s.tile_ctr, 0, sizeof(uint32_t) * (MAX_PASSES + 2), c.stream);
    cudaMemsetAsync(s.lookback, 0, sizeof(uint64_t) * tiles * BINS, c.stream);
    if (!hist_ready) {
        cudaMemsetAsync(s.hist, 0, sizeof(uint64_t) * passes * BINS, c.stream);
        uint64_t need = (n + S_BLOCK - 1) / S_BLOCK;
        const uint64_t cap = (uint64_t)c.sms * 4;
        k_hist<K><<<(int)(need < cap ? need : cap), S_BLOCK, 0, c.stream>>>(keys, n, passes, s.hist, RawDigit<K>{});
    }
    k_scan_bins<<<passes, BINS, 0, c.stream>>>(s.hist);
    K *src = keys, *dst = reinterpret_cast<K *>(s.alt);
    int done = 0;  // the first pass run needs no stability: the input order carries no information
    for (int p = 0; p < passes; p++) {
        if ((skip_mask >> p) & 1u) continue;  // every key has the same digit here: the pass would be a copy
        auto pass = variant == 0   ? onesweep_pass<K, 0>
                    : variant == 1 ? onesweep_pass<K, 1>
                    : variant == 2 ? onesweep_pass<K, 2>
                                   : onesweep_pass<K, BULK_VARIANT>;
        pass(c, src, dst, n, 8 * p, s.hist + (uint64_t)p * BINS, s.lookback, s.tile_ctr + p, (uint32_t)(p + 1), err,
             RawDigit<K>{}, done > 0);
        done++;
        if (passes_run) (*passes_run)++;
        K *t = src;
        src = dst;
        dst = t;
    }
    return src;
}

// Stable LSD sort by bucket index (bits bits, 8 per pass); keys keep their input order inside a
// bucket. Returns the buffer holding the result (keys or s.alt).
template <class K>
K *launch_bucket_sort(const LaunchCfg &c, K *keys, uint64_t n, const BucketGeom &g, int bits, const SortScratch &s,
                      uint32_t *err, int *passes_run, bool hist_ready, int variant) {
    const int passes = (bits + 7) / 8;
    if (passes_run) *passes_run = 0;
    if (n <= 1 || passes == 0) return keys;
    if (variant < 0 || variant > BULK_VARIANT) variant = 0;
    const BucketDigit<K> dig{g};
    const uint64_t TILE = (uint64_t)S_BLOCK * (variant == BULK_VARIANT ? SortCfg<K>::BULK_ITEMS
                                                                       : SortCfg<K>::V_ITEMS[variant]);
    const uint64_t tiles = (n + TILE - 1) / TILE;
    cudaMemsetAsync(s.tile_ctr, 0, sizeof(uint32_t) * (MAX_PASSES + 2), c.stream);
    cudaMemsetAsync(s.lookback, 0, sizeof(uint64_t) * tiles * BINS, c.stream);
    if (!hist_ready) {
        cudaMemsetAsync(s.hist, 0, sizeof(uint64_t) * passes * BINS, c.stream);
        const uint64_t need = (n + S_BLOCK - 1) / S_BLOCK, cap = (uint64_t)c.sms * 4;
        k_hist<K, BucketDigit<K>><<<(int)(need < cap ? need : cap), S_BLOCK, 0, c.stream>>>(keys, n, passes, s.hist,
                                                                                         dig);
    }
    k_scan_bins<<<passes, BINS, 0, c.stream>>>(s.hist);
    K *src = keys, *dst = reinterpret_cast<K *>(s.alt);
    for (int p = 0; p < passes; p++) {
        auto pass = variant == 0   ? onesweep_pass<K, 0, BucketDigit<K>>
                    : variant == 1 ? onesweep_pass<K, 1, BucketDigit<K>>
                    : variant == 2 ? onesweep_pass<K, 2, BucketDigit<K>>
                                   : onesweep_pass<K, BULK_VARIANT, BucketDigit<K>>;
        pass(c, src, dst, n, 8 * p, s.hist + (uint64_t)p * BINS, s.lookback, s.tile_ctr + p, (uint32_t)(p + 1), err,
             dig, p > 0);
        if (passes_run) (*passes_run)++;
        K *t = src;
        src = dst;
        dst = t;
    }
    return src;
}

// ---------------------------------------------------------------- run-length compaction
template <class K> struct RleCfg;
template <> struct RleCfg<uint64_t> { static constexpr int ITEMS = 16; };  // 4096 keys per tile
template <> struct RleCfg<Key128> { static constexpr int ITEMS = 8; };     // 2048 keys per tile

// Warp w of a tile owns a contiguous run of ITEMS rows of 32 keys (coalesced loads,
// no shared staging). A key starts a run iff it differs from its predecessor; the
// run starts of a row are ranked by ballot, rows are summed in order, warps by a
// block scan, tiles by decoupled look-back.
template <class K>
__global__ void __launch_bounds__(S_BLOCK, 4) k_rle(const K *__restrict__ sorted, uint64_t n, K *__restrict__ unique,
                                                 uint64_t *__restrict__ starts, unsigned long long *n_unique,
                                                 uint64_t *lookback, uint32_t *tile_ctr, uint32_t *err) {
    constexpr int R_ITEMS = RleCfg<K>::ITEMS;
    constexpr int R_TILE = S_BLOCK * R_ITEMS;
    __shared__ uint32_t s_warp[S_WARPS];
    __shared__ uint32_t s_scan[S_WARPS];
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_excl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const uint64_t tile = s_tile, start = tile * R_TILE;
    const uint64_t wstart = start + (uint64_t)warp * R_ITEMS * WARP;
    const uint32_t lt = lanemask_lt();
    K key[R_ITEMS];
    uint32_t ball[R_ITEMS];
    uint32_t wcount = 0;
    // all loads first (one memory latency per tile, not per row) ...
#pragma unroll
    for (int i = 0; i < R_ITEMS; i++) {
        const uint64_t idx = wstart + (uint64_t)i * WARP + lane;
        if (idx < n) key[i] = sorted[idx];
    }
    K before{};  // key just before this warp's run
    if (lane == 0 && wstart > 0 && wstart < n) before = sorted[wstart - 1];
    // ... then flags: the predecessor of lane l is lane l-1 of the same row, of lane 0 the last lane of the row before
#pragma unroll
    for (int i = 0; i < R_ITEMS; i++) {
        const uint64_t idx = wstart + (uint64_t)i * WARP + lane;
        K prev = shfl_up_key(key[i]);
        const K last_prev_row = shfl_key(i ? key[i - 1] : before, 31);
        if (lane == 0) prev = i ? last_prev_row : before;
        const bool f = idx < n && (idx == 0 || !KeyT<K>::eq(key[i], prev));
        ball[i] = __ballot_sync(FULL, f);
        wcount += __popc(ball[i]);
    }
    if (lane == 0) s_warp[warp] = wcount;
    __syncthreads();
    uint32_t total;
    const uint32_t wexcl = block_exclusive_scan<S_BLOCK>(tid < S_WARPS ? s_warp[tid] : 0u, s_scan, &total);
    __syncthreads();
    if (tid < S_WARPS) s_warp[tid] = wexcl;  // exclusive start of each warp inside the tile
    if (warp == 0) {
        const uint64_t e = lookback_prefix_warp(lookback, tile, total, 1, err);
        if (lane == 0) s_excl = e;
    }
    __syncthreads();
    uint64_t pos = s_excl + s_warp[warp];
#pragma unroll
    for (int i = 0; i < R_ITEMS; i++) {
        if ((ball[i] >> lane) & 1u) {
            const uint64_t o = pos + __popc(ball[i] & lt);
            unique[o] = key[i];
            if (starts) starts[o] = wstart + (uint64_t)i * WARP + lane;  // run starts only for run lengths
        }
        pos += __popc(ball[i]);
    }
    if (start + R_TILE >= n && tid == 0) *n_unique = s_excl + total;
}

__global__ void k_run_counts(const uint64_t *__restrict__ starts, const unsigned long long *n_unique, uint64_t n,
                             uint32_t *__restrict__ counts, uint32_t *err) {
    const uint64_t nu = *n_unique;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < nu; j += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t end = j + 1 < nu ? starts[j + 1] : n;
        const uint64_t c = end - starts[j];
        if (c > 0xfffffffeull) atomicOr(err, ERR_COUNT_OVERFLOW);
        counts[j] = (uint32_t)(c > 0xfffffffeull ? 0xfffffffeull : c);
    }
}

template <class K>
void launch_rle(const LaunchCfg &c, const K *sorted, uint64_t n, K *unique, uint64_t *starts,
                unsigned long long *n_unique, uint64_t *lookback, uint32_t *tile_ctr, uint32_t *err) {
    cudaMemsetAsync(n_unique, 0, sizeof(unsigned long long), c.stream);
    if (n == 0) return;
    constexpr int R_TILE = S_BLOCK * RleCfg<K>::ITEMS;
    const uint64_t tiles = (n + R_TILE - 1) / R_TILE;
    cudaMemsetAsync(tile_ctr, 0, sizeof(uint32_t), c.stream);
    cudaMemsetAsync(lookback, 0, sizeof(uint64_t) * tiles, c.stream);
    k_rle<K><<<(int)tiles, S_BLOCK, 0, c.stream>>>(sorted, n, unique, starts, n_unique, lookback, tile_ctr, err);
}

void launch_run_counts(const LaunchCfg &c, const uint64_t *starts, const unsigned long long *n_unique, uint64_t n,
                       uint64_t cap, uint32_t *counts, uint32_t *err) {
    uint64_t need = (cap + 255) / 256;
    const uint64_t lim = (uint64_t)c.sms * 8;
    k_run_counts<<<(int)(need < lim ? (need ? need : 1) : lim), 256, 0, c.stream>>>(starts, n_unique, n, counts, err);
}

template uint64_t *launch_radix_sort<uint64_t>(const LaunchCfg &, uint64_t *, uint64_t, int, const SortScratch &,
                                               uint32_t *, bool, uint32_t, int *, int);
template Key128 *launch_radix_sort<Key128>(const LaunchCfg &, Key128 *, uint64_t, int, const SortScratch &, uint32_t *,
                                           bool, uint32_t, int *, int);
template uint64_t *launch_bucket_sort<uint64_t>(const LaunchCfg &, uint64_t *, uint64_t, const BucketGeom &, int,
                                                const SortScratch &, uint32_t *, int *, bool, int);
template Key128 *launch_bucket_sort<Key128>(const LaunchCfg &, Key128 *, uint64_t, const BucketGeom &, int,
                                            const SortScratch &, uint32_t *, int *, bool, int);
template void launch_rle<uint64_t>(const LaunchCfg &, const uint64_t *, uint64_t, uint64_t *, uint64_t *,
                                   unsigned long long *, uint64_t *, uint32_t *, uint32_t *);
template void launch_rle<Key128>(const LaunchCfg &, const Key128 *, uint64_t, Key128 *, uint64_t *,
                                 unsigned long long *, uint64_t *, uint32_t *, uint32_t *);

}  // namespace turtle
