// Steps a5-a6: exact recount of every candidate and the min_count threshold.
//
// The paper adds 1 to each compacted count to make up for the first sighting
// that the filter swallowed (Sec. 2.1.4); that count is wrong whenever a key's
// first sighting was a filter false positive. Here the distinct candidates go
// into an open-addressing table (linear probing, key and count in one slot so a
// lookup touches one sector) and a second pass over every window adds 1 to the
// slot of its key, so each reported count is the exact number of occurrences,
// independent of atomic ordering and of false positives. Keys are then kept in
// their sorted order when count >= min_count (Sec. 2.1.1, Alg. 1).
#include "common.cuh"
#include "kernels.h"

namespace turtle {

template <> struct alignas(16) Slot<uint64_t> {
    uint64_t key;
    uint32_t count;  // EMPTY_COUNT until claimed
    uint32_t pad;
};
template <> struct alignas(32) Slot<Key128> {
    uint64_t hi, lo;
    uint32_t count;
    uint32_t pad[3];
};

__device__ __forceinline__ bool slot_has(const Slot<uint64_t> &s, uint64_t k) { return s.key == k; }
__device__ __forceinline__ bool slot_has(const Slot<Key128> &s, Key128 k) { return s.hi == k.hi && s.lo == k.lo; }
__device__ __forceinline__ void slot_put(Slot<uint64_t> *s, uint64_t k) { s->key = k; }
__device__ __forceinline__ void slot_put(Slot<Key128> *s, Key128 k) {
    s->hi = k.hi;
    s->lo = k.lo;
}
__device__ __forceinline__ Slot<uint64_t> slot_load(const Slot<uint64_t> *p) {
    const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2 *>(p));
    Slot<uint64_t> s;
    s.key = v.x;
    s.count = (uint32_t)v.y;
    return s;
}
__device__ __forceinline__ Slot<Key128> slot_load(const Slot<Key128> *p) {
    const ulonglong2 a = __ldcg(reinterpret_cast<const ulonglong2 *>(p));
    const uint32_t c = __ldcg(reinterpret_cast<const unsigned int *>(p) + 4);
    Slot<Key128> s;
    s.hi = a.x;
    s.lo = a.y;
    s.count = c;
    return s;
}
// Probe sequence of a key: start at slot p of line L (both from the hash), wrap inside the
// 128-byte line, then continue in the next lines. Insertion claims the first free slot of
// this sequence and slots are never freed, so a lookup that meets a free slot knows the key
// is absent. Most keys are decided within their first line: one DRAM line per probe.
template <class K> struct TableLine {
    static constexpr int S = 128 / (int)sizeof(Slot<K>);  // slots per 128-byte line (8 or 4)
};
template <class K>
__device__ __forceinline__ uint64_t probe_slot(uint64_t h, uint64_t j, uint64_t line_mask, uint64_t line_base = 0) {
    constexpr int S = TableLine<K>::S;
    const uint64_t g = h ^ (h >> 29);
    const uint64_t line = line_base + (((g >> 3) + j / S) & line_mask);
    return line * S + (uint64_t)((g + j) & (S - 1));
}

// The key's region: the whole table, or its library's lines (batched form).
struct Region {
    uint64_t base, mask;
};
template <class K>
__device__ __forceinline__ Region region_of(const K &key, const TableGeom &tg) {
    if (!tg.n_libs) return Region{0, tg.mask};
    const uint32_t l = tag_of(key, tg.tag_shift);
    return Region{__ldg(tg.lib_regions + 2 * l), __ldg(tg.lib_regions + 2 * l + 1)};
}

// Membership bitmap of the table's keys: two bits of one 64-bit word per key. It is
// small enough to stay in L2, so most probes of absent keys never reach the table.
__device__ __forceinline__ uint64_t member_word(uint64_t h, uint64_t word_mask) { return (h >> 24) & word_mask; }
__device__ __forceinline__ uint64_t member_bits(uint64_t h) { return (1ull << (h & 63)) | (1ull << ((h >> 6) & 63)); }

template <class K>
__global__ void k_table_insert(const K *__restrict__ unique, const uint32_t *__restrict__ counts,
                               const unsigned long long *n_unique, Slot<K> *table, TableGeom tg,
                               uint64_t *member, uint64_t member_mask, uint32_t *err) {
    const uint64_t nu = *n_unique;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < nu; j += (uint64_t)gridDim.x * blockDim.x) {
        const K key = unique[j];
        const uint32_t c0 = counts ? counts[j] : 0u;
        const uint64_t h = key_hash(key);
        const Region rg = region_of(key, tg);
        const uint64_t n_slots = (rg.mask + 1) * TableLine<K>::S;
        bool done = false;
        for (uint64_t probe = 0; probe < n_slots; probe++) {
            const uint64_t s = probe_slot<K>(h, probe, rg.mask, rg.base);
            if (atomicCAS(&table[s].count, EMPTY_COUNT, c0) == EMPTY_COUNT) {  // distinct keys: claim any free slot
                slot_put(&table[s], key);
                done = true;
                break;
            }
        }
        if (member) atomicOr((unsigned long long *)&member[member_word(h, member_mask)],
                             (unsigned long long)member_bits(h));
        if (!done) atomicOr(err, ERR_TABLE_FULL);
    }
}

constexpr int P2_BLOCK = 256;
constexpr int P2_WARPS = P2_BLOCK / WARP;
constexpr int P2_ILP = 4;
constexpr int P2_TILE = WARP * P2_ILP;

template <class K>
__global__ void __launch_bounds__(P2_BLOCK) k_pass2(const uint64_t *__restrict__ P, const uint64_t *__restrict__ V,
                                                    uint64_t n_pos, int k, Slot<K> *table, TableGeom tg,
                                                    int check_overflow, uint32_t *err) {
    const uint64_t mask = tg.mask;  // the windows form runs on one region
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t tiles = (n_pos + P2_TILE - 1) / P2_TILE;
    for (uint64_t t = (uint64_t)blockIdx.x * P2_WARPS + warp; t < tiles; t += (uint64_t)gridDim.x * P2_WARPS) {
        const uint64_t base = t * P2_TILE;
        const uint64_t v0 = V[2 * t], v1 = V[2 * t + 1];
        bool ok[P2_ILP];
        K key[P2_ILP];
        uint64_t h[P2_ILP];
        Slot<K> sl[P2_ILP];
#pragma unroll
        for (int i = 0; i < P2_ILP; i++) {
            const int r = lane + WARP * i;
            const uint64_t pos = base + r;
            ok[i] = pos < n_pos && (((r < 64 ? v0 : v1) >> (r & 63)) & 1);
            if (ok[i]) {
                key[i] = canonical<K>(P, pos, k);
                h[i] = key_hash(key[i]);
                sl[i] = slot_load(table + probe_slot<K>(h[i], 0, mask));
            }
        }
        const uint64_t n_slots = (mask + 1) * TableLine<K>::S;
#pragma unroll
        for (int i = 0; i < P2_ILP; i++) {
            if (!ok[i]) continue;
            for (uint64_t probe = 0; probe < n_slots;) {
                if (sl[i].count == EMPTY_COUNT) break;  // key absent: not a candidate
                if (slot_has(sl[i], key[i])) {
                    unsigned int *cnt = &table[probe_slot<K>(h[i], probe, mask)].count;
                    if (check_overflow) {
                        const uint32_t old = atomicAdd(cnt, 1u);
                        if (old >= 0xfffffffeu) atomicOr(err, ERR_COUNT_OVERFLOW);  // would pass 2^32-2
                    } else {
                        atomicAdd(cnt, 1u);
                    }
                    break;
                }
                if (++probe < n_slots) sl[i] = slot_load(table + probe_slot<K>(h[i], probe, mask));
            }
        }
    }
}

// First-sighting recount. In pass 1 each valid window went either to the
// candidates (filter said "seen") or to the firsts (its atomicOr completed the
// pattern), and at most one occurrence of a key can be a first. A candidate key's
// slot starts at its run length in the sorted candidates; adding 1 for its first
// sighting, if it has one, gives the exact number of occurrences. Keys absent from
// the table have all their occurrences among the firsts, so they occur once.
constexpr int F_ILP = 4;

template <class K>
__global__ void __launch_bounds__(256, 4) k_add_firsts(const K *__restrict__ firsts, uint64_t n, Slot<K> *table,
                                                    TableGeom tg, const uint64_t *__restrict__ member,
                                                    uint64_t member_mask, int check_overflow, uint32_t *err) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; base < n; base += stride * F_ILP) {
        K key[F_ILP];
        uint64_t h[F_ILP], mw[F_ILP];
        bool ok[F_ILP];
#pragma unroll
        for (int i = 0; i < F_ILP; i++) {
            const uint64_t j = base + i * stride;
            ok[i] = j < n;
            if (ok[i]) {
                key[i] = load_stream(firsts + j);
                h[i] = key_hash(key[i]);
                mw[i] = member ? __ldcg(member + member_word(h[i], member_mask)) : 0;
            }
        }
        Slot<K> sl[F_ILP];
#pragma unroll
        for (int i = 0; i < F_ILP; i++) {  // first probes of every possible member, issued together
            const uint64_t mb = member_bits(h[i]);
            ok[i] = ok[i] && (!member || (mw[i] & mb) == mb);  // else certainly not a candidate key
            if (ok[i]) {
                const Region rg = region_of(key[i], tg);
                sl[i] = slot_load(table + probe_slot<K>(h[i], 0, rg.mask, rg.base));
            }
        }
#pragma unroll
        for (int i = 0; i < F_ILP; i++) {
            if (!ok[i]) continue;
            const Region rg = region_of(key[i], tg);  // recomputed: cheaper than holding it in registers
            const uint64_t n_slots = (rg.mask + 1) * TableLine<K>::S;
            for (uint64_t probe = 0; probe < n_slots;) {
                if (sl[i].count == EMPTY_COUNT) break;
                if (slot_has(sl[i], key[i])) {
                    unsigned int *cnt = &table[probe_slot<K>(h[i], probe, rg.mask, rg.base)].count;
                    if (check_overflow) {
                        if (atomicAdd(cnt, 1u) >= 0xfffffffeu) atomicOr(err, ERR_COUNT_OVERFLOW);
                    } else {
                        atomicAdd(cnt, 1u);  // result unused: a fire-and-forget reduction
                    }
                    break;
                }
                if (++probe < n_slots) sl[i] = slot_load(table + probe_slot<K>(h[i], probe, rg.mask, rg.base));
            }
        }
    }
}

constexpr int T_ITEMS = 8;
constexpr int T_TILE = P2_BLOCK * T_ITEMS;

template <class K>
__device__ __forceinline__ uint32_t table_count(const Slot<K> *table, const TableGeom &tg, K key) {
    const uint64_t h = key_hash(key);
    const Region rg = region_of(key, tg);
    const uint64_t n_slots = (rg.mask + 1) * TableLine<K>::S;
    for (uint64_t probe = 0; probe < n_slots; probe++) {
        const Slot<K> sl = slot_load(table + probe_slot<K>(h, probe, rg.mask, rg.base));
        if (sl.count == EMPTY_COUNT) return EMPTY_COUNT;
        if (slot_has(sl, key)) return sl.count;
    }
    return EMPTY_COUNT;
}

template <class K>
__global__ void __launch_bounds__(P2_BLOCK) k_threshold(const K *__restrict__ unique, uint64_t n_unique,
                                                        const Slot<K> *table, TableGeom tg, uint32_t min_count,
                                                        K *__restrict__ out_keys, uint32_t *__restrict__ out_counts,
                                                        unsigned long long *n_out, uint64_t *lookback,
                                                        uint32_t *tile_ctr, uint32_t *err) {
    __shared__ uint32_t s_scan[P2_WARPS];
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_excl;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const uint64_t tile = s_tile, start = tile * T_TILE;
    K key[T_ITEMS];
    uint32_t cnt[T_ITEMS];
    uint32_t keep = 0, nkeep = 0;
#pragma unroll
    for (int j = 0; j < T_ITEMS; j++) {
        const uint64_t idx = start + (uint64_t)j * P2_BLOCK + tid;  // striped: coalesced key reads
        if (idx < n_unique) {
            key[j] = unique[idx];
            cnt[j] = table_count(table, tg, key[j]);
            if (cnt[j] == EMPTY_COUNT) atomicOr(err, ERR_NOT_FOUND);
            else if (cnt[j] >= min_count) {
                keep |= 1u << j;
                nkeep++;
            }
        }
    }
    // Order must follow idx; striped ownership means rank = (count kept before idx in this tile).
    // Scan row by row: row j holds idx = start + j*BLOCK + tid.
    uint64_t row_base = 0;
    __shared__ uint64_t s_rowtot[T_ITEMS];
    uint32_t rowpos[T_ITEMS];
#pragma unroll
    for (int j = 0; j < T_ITEMS; j++) {
        uint32_t tot;
        rowpos[j] = block_exclusive_scan<P2_BLOCK>((keep >> j) & 1u, s_scan, &tot);
        if (tid == 0) s_rowtot[j] = tot;
        __syncthreads();
    }
    uint32_t total = 0;
    for (int j = 0; j < T_ITEMS; j++) total += (uint32_t)s_rowtot[j];
    if (tid < WARP) {
        const uint64_t e = lookback_prefix_warp(lookback, tile, total, 1, err);
        if (tid == 0) s_excl = e;
    }
    __syncthreads();
    row_base = s_excl;
#pragma unroll
    for (int j = 0; j < T_ITEMS; j++) {
        if ((keep >> j) & 1u) {
            const uint64_t o = row_base + rowpos[j];
            store_key(out_keys + o, key[j]);
            out_counts[o] = cnt[j];
        }
        row_base += s_rowtot[j];
    }
    if (start + T_TILE >= n_unique && tid == 0) *n_out = s_excl + total;
    (void)nkeep;
}

template <class K>
void launch_table_clear(const LaunchCfg &c, void *table, uint64_t lines) {
    cudaMemsetAsync(table, 0xff, 128 * lines, c.stream);
}

template <class K>
void launch_table_insert(const LaunchCfg &c, const K *unique, const uint32_t *counts,
                         const unsigned long long *n_unique, uint64_t cap, void *table, const TableGeom &tg,
                         uint64_t *member, uint64_t member_words, uint32_t *err) {
    uint64_t need = (cap + 255) / 256;
    const uint64_t lim = (uint64_t)c.sms * 8;
    k_table_insert<K><<<(int)(need < lim ? (need ? need : 1) : lim), 256, 0, c.stream>>>(
        unique, counts, n_unique, reinterpret_cast<Slot<K> *>(table), tg, member,
        member_words ? member_words - 1 : 0, err);
}

template <class K>
void launch_add_firsts(const LaunchCfg &c, const K *firsts, uint64_t n, void *table, const TableGeom &tg,
                       const uint64_t *member, uint64_t member_words, bool check_overflow, uint32_t *err) {
    if (n == 0) return;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_add_firsts<K>, 256, 0);
    if (per_sm < 1) per_sm = 1;
    uint64_t need = (n + 256 * F_ILP - 1) / (256 * F_ILP);
    const uint64_t lim = (uint64_t)c.sms * per_sm;
    k_add_firsts<K><<<(int)(need < lim ? (need ? need : 1) : lim), 256, 0, c.stream>>>(
        firsts, n, reinterpret_cast<Slot<K> *>(table), tg, member, member_words ? member_words - 1 : 0,
        check_overflow ? 1 : 0, err);
}

template <class K>
void launch_pass2(const LaunchCfg &c, const PackLayout &L, int k, const uint64_t *P, const uint64_t *V, void *table,
                  const TableGeom &tg, bool check_overflow, uint32_t *err) {
    const uint64_t tiles = (L.n_bases + P2_TILE - 1) / P2_TILE;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pass2<K>, P2_BLOCK, 0);
    if (per_sm < 1) per_sm = 1;
    uint64_t need = (tiles + P2_WARPS - 1) / P2_WARPS;
    const uint64_t cap = (uint64_t)c.sms * per_sm;
    k_pass2<K><<<(int)(need < cap ? (need ? need : 1) : cap), P2_BLOCK, 0, c.stream>>>(
        P, V, L.n_bases, k, reinterpret_cast<Slot<K> *>(table), tg, check_overflow ? 1 : 0, err);
}

template <class K>
void launch_threshold(const LaunchCfg &c, const K *unique, uint64_t n_unique, const void *table, const TableGeom &tg,
                      uint32_t min_count, K *out_keys, uint32_t *out_counts, unsigned long long *n_out,
                      uint64_t *lookback, uint32_t *tile_ctr, uint32_t *err) {
    cudaMemsetAsync(n_out, 0, sizeof(unsigned long long), c.stream);
    if (n_unique == 0) return;
    const uint64_t tiles = (n_unique + T_TILE - 1) / T_TILE;
    cudaMemsetAsync(tile_ctr, 0, sizeof(uint32_t), c.stream);
    cudaMemsetAsync(lookback, 0, sizeof(uint64_t) * tiles, c.stream);
    k_threshold<K><<<(int)tiles, P2_BLOCK, 0, c.stream>>>(unique, n_unique, reinterpret_cast<const Slot<K> *>(table),
                                                          tg, min_count, out_keys, out_counts, n_out, lookback,
                                                          tile_ctr, err);
}

size_t slot_bytes(int key_words) { return key_words == 1 ? sizeof(Slot<uint64_t>) : sizeof(Slot<Key128>); }
int slots_per_line(int key_words) { return key_words == 1 ? TableLine<uint64_t>::S : TableLine<Key128>::S; }

#define INST(K)                                                                                                  \
    template void launch_table_clear<K>(const LaunchCfg &, void *, uint64_t);                                    \
    template void launch_table_insert<K>(const LaunchCfg &, const K *, const uint32_t *,                         \
                                         const unsigned long long *, uint64_t, void *, const TableGeom &,        \
                                         uint64_t *, uint64_t, uint32_t *);                                      \
    template void launch_add_firsts<K>(const LaunchCfg &, const K *, uint64_t, void *, const TableGeom &,        \
                                       const uint64_t *, uint64_t, bool, uint32_t *);                            \
    template void launch_pass2<K>(const LaunchCfg &, const PackLayout &, int, const uint64_t *, const uint64_t *, \
                                  void *, const TableGeom &, bool, uint32_t *);                                  \
    template void launch_threshold<K>(const LaunchCfg &, const K *, uint64_t, const void *, const TableGeom &,   \
                                      uint32_t,                                                                  \
                                      K *, uint32_t *, unsigned long long *, uint64_t *, uint32_t *, uint32_t *);
INST(uint64_t)
INST(Key128)

}  // namespace turtle
