// Hash-table form of steps a4-a6 (params.compact = 2): the counterpart of the paper's Table 1,
// which sets sort-and-compress against hash tables for counting items and their frequencies
// (Sec. 2.1.1). The candidates of pass 1 are counted in one open-addressing table in device
// memory instead of being sorted:
//   1. a HyperLogLog sketch of the candidates (Flajolet, Fusy, Gandouet & Meunier, AofA 2007)
//      estimates how many distinct keys they hold, which sizes the table;
//   2. each candidate takes its key's slot with a compare-and-swap on the key (a free slot or
//      one that already holds the key) and adds 1 to the slot's count; a key that finds no
//      such slot within its probe bound marks the table full, and the caller doubles the table
//      and counts again;
//   3. each first sighting adds 1 to its key's slot if the key is there (keys that are not
//      there occur once);
//   4. a scan of the table keeps the keys whose count reaches min_count, in slot order;
//   5. the kept keys are radix-sorted and their counts looked up in the table.
// Steps 2 and 3 give every candidate key its exact number of occurrences, as the sort-based
// forms do, so all forms return the same result.
#include "common.cuh"
#include "kernels.h"

namespace turtle {

namespace {

constexpr unsigned long long EMPTY_KEY = ~0ull;  // no canonical key, tagged or not, is all ones

template <class K> struct HSlot;
template <> struct alignas(16) HSlot<uint64_t> {
    unsigned long long key;
    uint32_t count, pad;
};
template <> struct alignas(32) HSlot<Key128> {
    unsigned long long hi, lo;  // hi at the lower address
    uint32_t count, pad[3];
};
template <class K> struct HLine {
    static constexpr int S = 128 / (int)sizeof(HSlot<K>);  // slots per 128-byte line: 8 or 4
};

// Probe j of a key: the line (h >> 3) + j / S (wrapping at the table's end), slot (h + j) mod S
// inside it. Slots are never freed, so a key's probes stop at the first free slot.
template <class K>
__device__ __forceinline__ uint64_t hslot(uint64_t h, uint32_t j, uint64_t line_mask) {
    constexpr int S = HLine<K>::S;
    return (((h >> 3) + j / S) & line_mask) * S + ((h + j) & (S - 1));
}

__device__ __forceinline__ bool is_empty(unsigned long long k) { return k == EMPTY_KEY; }
__device__ __forceinline__ bool is_empty(Key128 k) { return k.hi == EMPTY_KEY && k.lo == EMPTY_KEY; }
__device__ __forceinline__ bool same(unsigned long long a, uint64_t b) { return a == b; }
__device__ __forceinline__ bool same(Key128 a, Key128 b) { return a.hi == b.hi && a.lo == b.lo; }

// Compare-and-swap of a free slot's key to `key`; returns the key the slot held before.
__device__ __forceinline__ unsigned long long claim(HSlot<uint64_t> *s, uint64_t key) {
    return atomicCAS(&s->key, EMPTY_KEY, (unsigned long long)key);
}
__device__ __forceinline__ Key128 claim(HSlot<Key128> *s, Key128 key) {
    unsigned long long o0, o1;
    // 16-byte atomic (sm_90 and later); the low 64 bits of an operand are the word at the lower
    // address, which is the slot's hi.
    asm volatile(
        "{\n\t.reg .b128 d, c, v;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 v, {%4, %5};\n\t"
        "atom.global.cas.b128 d, [%6], c, v;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(o0), "=l"(o1)
        : "l"(EMPTY_KEY), "l"(EMPTY_KEY), "l"(key.hi), "l"(key.lo), "l"(__cvta_generic_to_global(s))
        : "memory");
    return Key128{o0, o1};
}

// First look at a slot during insertion. A 64-bit key is loaded (a single-copy atomic access):
// most candidates find their key already there and then need only a fire-and-forget add, and a
// free slot is taken with a compare-and-swap afterwards. A 128-bit key goes straight to the
// compare-and-swap, because a 16-byte load racing with another thread's swap is not guaranteed
// to see the slot whole.
template <class K> constexpr bool LOOK_FIRST = sizeof(K) == 8;
__device__ __forceinline__ unsigned long long first_look(HSlot<uint64_t> *s, uint64_t) {
    return __ldcg(&s->key);
}
__device__ __forceinline__ Key128 first_look(HSlot<Key128> *s, Key128 key) { return claim(s, key); }

// The key a slot holds, read when no thread writes keys any more.
__device__ __forceinline__ unsigned long long slot_key(const HSlot<uint64_t> *s) { return __ldcg(&s->key); }
__device__ __forceinline__ Key128 slot_key(const HSlot<Key128> *s) {
    const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2 *>(s));
    return Key128{v.x, v.y};
}
// Key and count of a slot in one access where the slot fits 16 bytes.
__device__ __forceinline__ void slot_read(const HSlot<uint64_t> *s, unsigned long long *key, uint32_t *count) {
    const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2 *>(s));
    *key = v.x;
    *count = (uint32_t)v.y;
}
__device__ __forceinline__ void slot_read(const HSlot<Key128> *s, Key128 *key, uint32_t *count) {
    const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2 *>(s));
    *key = Key128{v.x, v.y};
    *count = __ldcg(&s->count);
}
__device__ __forceinline__ uint64_t as_key(unsigned long long k, uint64_t) { return k; }
__device__ __forceinline__ Key128 as_key(Key128 k, Key128) { return k; }

template <class K> struct Held { using T = unsigned long long; };
template <> struct Held<Key128> { using T = Key128; };

__device__ __forceinline__ void add_one(uint32_t *count, int check_overflow, uint32_t *err) {
    if (check_overflow) {
        if (atomicAdd(count, 1u) >= 0xfffffffeu) atomicOr(err, ERR_COUNT_OVERFLOW);  // would pass 2^32 - 2
    } else {
        atomicAdd(count, 1u);  // result unused: a reduction
    }
}

constexpr int H_BLOCK = 256;
constexpr int H_ILP = 4;
constexpr int HLL_BITS = 12;

// HyperLogLog registers: register (h >> 52) keeps the largest rank seen, rank = 1 + the number of
// leading zeros of the hash's low 52 bits (at most 53).
template <class K>
__global__ void __launch_bounds__(1024) k_hll(const K *__restrict__ keys, uint64_t n, uint32_t *regs) {
    __shared__ uint32_t r[1 << HLL_BITS];
    for (int i = threadIdx.x; i < (1 << HLL_BITS); i += 1024) r[i] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * 1024;
    for (uint64_t j = blockIdx.x * 1024ull + threadIdx.x; j < n; j += stride) {
        const uint64_t h = key_hash(load_stream(keys + j));
        const uint32_t idx = (uint32_t)(h >> (64 - HLL_BITS));
        const uint32_t rank = (uint32_t)__clzll((long long)((h << HLL_BITS) | (1ull << (HLL_BITS - 1)))) + 1;
        if (rank > r[idx]) atomicMax(&r[idx], rank);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (1 << HLL_BITS); i += 1024)
        if (r[i]) atomicMax(&regs[i], r[i]);
}

template <class K>
__global__ void k_hash_clear(HSlot<K> *table, uint64_t n_slots) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n_slots; j += stride) {
        ulonglong2 *p = reinterpret_cast<ulonglong2 *>(table + j);
        if (sizeof(HSlot<K>) == 16) {
            p[0] = make_ulonglong2(EMPTY_KEY, 0ull);
        } else {
            p[0] = make_ulonglong2(EMPTY_KEY, EMPTY_KEY);
            p[1] = make_ulonglong2(0ull, 0ull);
        }
    }
}

// Step 2: every candidate adds 1 to its key's slot. n_distinct += the slots taken.
template <class K>
__global__ void __launch_bounds__(H_BLOCK) k_hash_insert(const K *__restrict__ keys, uint64_t n, HSlot<K> *table,
                                                         uint64_t line_mask, uint32_t bound, int check_overflow,
                                                         unsigned long long *n_distinct, uint32_t *full, uint32_t *err) {
    using H = typename Held<K>::T;
    __shared__ uint32_t s_new;
    if (threadIdx.x == 0) s_new = 0;
    __syncthreads();
    uint32_t fresh = 0;
    const uint64_t stride = (uint64_t)gridDim.x * H_BLOCK;
    for (uint64_t base = blockIdx.x * (uint64_t)H_BLOCK + threadIdx.x; base < n; base += stride * H_ILP) {
        K key[H_ILP];
        uint64_t h[H_ILP];
        H old[H_ILP];
        bool ok[H_ILP];
#pragma unroll
        for (int i = 0; i < H_ILP; i++) {
            const uint64_t j = base + i * stride;
            ok[i] = j < n;
            if (ok[i]) {
                key[i] = load_stream(keys + j);
                h[i] = key_hash(key[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < H_ILP; i++)  // the first probes of all keys in flight together
            if (ok[i]) old[i] = first_look(table + hslot<K>(h[i], 0, line_mask), key[i]);
#pragma unroll
        for (int i = 0; i < H_ILP; i++) {
            if (!ok[i]) continue;
            for (uint32_t j = 0;;) {
                HSlot<K> *sl = table + hslot<K>(h[i], j, line_mask);
                if (LOOK_FIRST<K> && is_empty(old[i])) old[i] = claim(sl, key[i]);  // free when loaded: take it
                if (is_empty(old[i]) || same(old[i], key[i])) {
                    fresh += is_empty(old[i]) ? 1u : 0u;
                    add_one(&sl->count, check_overflow, err);
                    break;
                }
                if (++j >= bound) {  // no room within the bound: the table is too small
                    atomicOr(full, 1u);
                    break;
                }
                old[i] = first_look(table + hslot<K>(h[i], j, line_mask), key[i]);
            }
        }
    }
    if (fresh) atomicAdd(&s_new, fresh);
    __syncthreads();
    if (threadIdx.x == 0 && s_new) atomicAdd(n_distinct, (unsigned long long)s_new);
}

// Step 3: every first sighting whose key is in the table adds 1 to it.
template <class K>
__global__ void __launch_bounds__(H_BLOCK) k_hash_firsts(const K *__restrict__ keys, uint64_t n, HSlot<K> *table,
                                                         uint64_t line_mask, uint32_t bound, int check_overflow,
                                                         uint32_t *err) {
    using H = typename Held<K>::T;
    const uint64_t stride = (uint64_t)gridDim.x * H_BLOCK;
    for (uint64_t base = blockIdx.x * (uint64_t)H_BLOCK + threadIdx.x; base < n; base += stride * H_ILP) {
        K key[H_ILP];
        uint64_t h[H_ILP];
        H cur[H_ILP];
        bool ok[H_ILP];
#pragma unroll
        for (int i = 0; i < H_ILP; i++) {
            const uint64_t j = base + i * stride;
            ok[i] = j < n;
            if (ok[i]) {
                key[i] = load_stream(keys + j);
                h[i] = key_hash(key[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < H_ILP; i++)
            if (ok[i]) cur[i] = slot_key(table + hslot<K>(h[i], 0, line_mask));
#pragma unroll
        for (int i = 0; i < H_ILP; i++) {
            if (!ok[i]) continue;
            for (uint32_t j = 0;;) {
                if (same(cur[i], key[i])) {
                    add_one(&table[hslot<K>(h[i], j, line_mask)].count, check_overflow, err);
                    break;
                }
                if (is_empty(cur[i]) || ++j >= bound) break;  // not a candidate key
                cur[i] = slot_key(table + hslot<K>(h[i], j, line_mask));
            }
        }
    }
}

// Step 4: keys of the slots whose count reaches min_count, appended to out in slot order per tile.
constexpr int X_ITEMS = 8;
constexpr int X_TILE = H_BLOCK * X_ITEMS;

template <class K>
__global__ void __launch_bounds__(H_BLOCK) k_hash_extract(const HSlot<K> *__restrict__ table, uint64_t n_slots,
                                                          uint32_t min_count, K *__restrict__ out, uint64_t cap,
                                                          unsigned long long *n_out, uint32_t *err) {
    using H = typename Held<K>::T;
    __shared__ uint32_t s_scan[H_BLOCK / WARP];
    __shared__ unsigned long long s_base;
    const uint64_t tiles = (n_slots + X_TILE - 1) / X_TILE;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        K key[X_ITEMS];
        uint32_t keep = 0, nk = 0;
#pragma unroll
        for (int j = 0; j < X_ITEMS; j++) {
            const uint64_t idx = t * X_TILE + (uint64_t)j * H_BLOCK + threadIdx.x;  // striped: coalesced
            if (idx < n_slots) {
                H kk;
                uint32_t c;
                slot_read(table + idx, &kk, &c);
                if (!is_empty(kk) && c >= min_count) {
                    key[j] = as_key(kk, K{});
                    keep |= 1u << j;
                    nk++;
                }
            }
        }
        uint32_t total;
        const uint32_t before = block_exclusive_scan<H_BLOCK>(nk, s_scan, &total);
        if (threadIdx.x == 0) s_base = total ? atomicAdd(n_out, (unsigned long long)total) : 0ull;
        __syncthreads();
        uint64_t o = s_base + before;
#pragma unroll
        for (int j = 0; j < X_ITEMS; j++) {
            if ((keep >> j) & 1u) {
                if (o < cap) store_key(out + o, key[j]);
                else atomicOr(err, ERR_CAND_OVERFLOW);
                o++;
            }
        }
        __syncthreads();  // s_scan and s_base are reused by the next tile
    }
}

// Step 5: counts[i] <- the count of keys[i] in the table.
template <class K>
__global__ void __launch_bounds__(H_BLOCK) k_hash_lookup(const K *__restrict__ keys, uint64_t n,
                                                         const HSlot<K> *__restrict__ table, uint64_t line_mask,
                                                         uint32_t bound, uint32_t *__restrict__ counts, uint32_t *err) {
    using H = typename Held<K>::T;
    const uint64_t stride = (uint64_t)gridDim.x * H_BLOCK;
    for (uint64_t base = blockIdx.x * (uint64_t)H_BLOCK + threadIdx.x; base < n; base += stride * H_ILP) {
        K key[H_ILP];
        uint64_t h[H_ILP];
        H cur[H_ILP];
        uint32_t c[H_ILP];
        bool ok[H_ILP];
#pragma unroll
        for (int i = 0; i < H_ILP; i++) {
            const uint64_t j = base + i * stride;
            ok[i] = j < n;
            if (ok[i]) {
                key[i] = load_stream(keys + j);
                h[i] = key_hash(key[i]);
                slot_read(table + hslot<K>(h[i], 0, line_mask), &cur[i], &c[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < H_ILP; i++) {
            if (!ok[i]) continue;
            for (uint32_t j = 0;;) {
                if (same(cur[i], key[i])) {
                    counts[base + i * stride] = c[i];
                    break;
                }
                if (is_empty(cur[i]) || ++j >= bound) {  // every kept key is in the table
                    atomicOr(err, ERR_NOT_FOUND);
                    break;
                }
                slot_read(table + hslot<K>(h[i], j, line_mask), &cur[i], &c[i]);
            }
        }
    }
}

// Probes per key before the table counts as full: 32 lines, or every slot of a smaller table.
template <class K>
uint32_t probe_bound(uint64_t lines) {
    return (uint32_t)((lines < 32 ? lines : 32) * HLine<K>::S);
}

// Grid of a grid-stride kernel: every CTA the device holds at once, no more than the items need.
template <class F>
int grid_for(const LaunchCfg &c, F kernel, int block, uint64_t items, uint64_t per_block) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const uint64_t need = (items + per_block - 1) / per_block;
    const uint64_t cap = (uint64_t)c.sms * per_sm;
    return (int)(need < cap ? (need ? need : 1) : cap);
}

}  // namespace

int hash_sketch_bits() { return HLL_BITS; }

template <class K>
void launch_hash_sketch(const LaunchCfg &c, const K *keys, uint64_t n, uint32_t *regs) {
    if (n == 0) return;
    k_hll<K><<<grid_for(c, k_hll<K>, 1024, n, 1024 * 16), 1024, 0, c.stream>>>(keys, n, regs);
}

template <class K>
void launch_hash_clear(const LaunchCfg &c, void *table, uint64_t lines) {
    const uint64_t n_slots = lines * HLine<K>::S;
    k_hash_clear<K><<<grid_for(c, k_hash_clear<K>, 256, n_slots, 256 * 8), 256, 0, c.stream>>>(reinterpret_cast<HSlot<K> *>(table),
                                                                           n_slots);
}

template <class K>
void launch_hash_insert(const LaunchCfg &c, const K *keys, uint64_t n, void *table, uint64_t lines,
                        bool check_overflow, unsigned long long *n_distinct, uint32_t *full, uint32_t *err) {
    if (n == 0) return;
    k_hash_insert<K><<<grid_for(c, k_hash_insert<K>, H_BLOCK, n, H_BLOCK * H_ILP), H_BLOCK, 0, c.stream>>>(
        keys, n, reinterpret_cast<HSlot<K> *>(table), lines - 1, probe_bound<K>(lines), check_overflow ? 1 : 0,
        n_distinct, full, err);
}

template <class K>
void launch_hash_firsts(const LaunchCfg &c, const K *keys, uint64_t n, void *table, uint64_t lines,
                        bool check_overflow, uint32_t *err) {
    if (n == 0) return;
    k_hash_firsts<K><<<grid_for(c, k_hash_firsts<K>, H_BLOCK, n, H_BLOCK * H_ILP), H_BLOCK, 0, c.stream>>>(
        keys, n, reinterpret_cast<HSlot<K> *>(table), lines - 1, probe_bound<K>(lines), check_overflow ? 1 : 0, err);
}

template <class K>
void launch_hash_extract(const LaunchCfg &c, const void *table, uint64_t lines, uint32_t min_count, K *out,
                         uint64_t cap, unsigned long long *n_out, uint32_t *err) {
    const uint64_t n_slots = lines * HLine<K>::S;
    k_hash_extract<K><<<grid_for(c, k_hash_extract<K>, H_BLOCK, n_slots, X_TILE), H_BLOCK, 0, c.stream>>>(
        reinterpret_cast<const HSlot<K> *>(table), n_slots, min_count, out, cap, n_out, err);
}

template <class K>
void launch_hash_lookup(const LaunchCfg &c, const K *keys, uint64_t n, const void *table, uint64_t lines,
                        uint32_t *counts, uint32_t *err) {
    if (n == 0) return;
    k_hash_lookup<K><<<grid_for(c, k_hash_lookup<K>, H_BLOCK, n, H_BLOCK * H_ILP), H_BLOCK, 0, c.stream>>>(
        keys, n, reinterpret_cast<const HSlot<K> *>(table), lines - 1, probe_bound<K>(lines), counts, err);
}

int hash_slots_per_line(int key_words) { return key_words == 1 ? HLine<uint64_t>::S : HLine<Key128>::S; }

#define INST(K)                                                                                                   \
    template void launch_hash_sketch<K>(const LaunchCfg &, const K *, uint64_t, uint32_t *);                      \
    template void launch_hash_clear<K>(const LaunchCfg &, void *, uint64_t);                                      \
    template void launch_hash_insert<K>(const LaunchCfg &, const K *, uint64_t, void *, uint64_t, bool,           \
                                        unsigned long long *, uint32_t *, uint32_t *);                            \
    template void launch_hash_firsts<K>(const LaunchCfg &, const K *, uint64_t, void *, uint64_t, bool,           \
                                        uint32_t *);                                                              \
    template void launch_hash_extract<K>(const LaunchCfg &, const void *, uint64_t, uint32_t, K *, uint64_t,      \
                                         unsigned long long *, uint32_t *);                                       \
    template void launch_hash_lookup<K>(const LaunchCfg &, const K *, uint64_t, const void *, uint64_t,          \
                                        uint32_t *, uint32_t *);
INST(uint64_t)
INST(Key128)

}  // namespace turtle
