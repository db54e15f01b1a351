// Bucketed sort-and-compact (Sec. 2.1.4), with the exact recount and the threshold folded in.
//
// The paper keeps each consumer's working array small enough for the cache and compacts it
// by sorting and merging duplicates. On the GPU the same idea is one MSD radix step followed
// by work that stays in shared memory:
//   1. every key (candidates and first sightings) gets a bucket: an order-preserving function
//      of its top bits, so bucket b holds a contiguous key range and buckets come in key order;
//   2. a stable LSD radix sort on the bucket index alone (onesweep, 8 bits per pass: two passes
//      for up to 65536 buckets) groups the candidates, and separately the first sightings, by
//      bucket; a binary search per bucket finds where each bucket starts;
//   3. one CTA per bucket merges the bucket's candidates into a shared-memory table (key ->
//      run length, i.e. sort-and-compact of the bucket), adds one for each key that has a
//      first sighting in the bucket, keeps count >= min_count, sorts those keys and writes
//      them out; a bucket whose distinct keys do not fit is split into key ranges and redone;
//   4. an exclusive scan of the per-bucket output counts and a gather give the final,
//      ascending output.
// The result equals the global sort-and-compact plus recount exactly (same keys, same counts).
#include <algorithm>

#include "bucket.cuh"

namespace turtle {

namespace {

// Bucket CTA shapes: threads, shared-memory table slots, CTAs per SM. A table attempt holds at most
// LIMIT distinct keys (load 0.75); every thread extracts ITEMS table entries.
template <uint32_t THREADS_, uint32_t LOG2_, int MINB_>
struct BtCfg {
    static constexpr uint32_t THREADS = THREADS_, LOG2 = LOG2_, SLOTS = 1u << LOG2_;
    static constexpr uint32_t LIMIT = SLOTS / 4 * 3, ITEMS = LIMIT / THREADS;
    static constexpr int MINB = MINB_;
    static_assert(LIMIT + THREADS < SLOTS, "an empty slot must always remain");
    static_assert(LIMIT % THREADS == 0, "extraction items per thread");
};
using BtSmall = BtCfg<512, 12, 2>;   // 4096 slots, two CTAs per SM
using BtLarge = BtCfg<1024, 13, 1>;  // 8192 slots, one CTA per SM
constexpr int BT_STACK = 136;        // pending key ranges (2 per split level, 128-bit ranges)
constexpr uint32_t BT_LOG2_NSUB = 10, BT_NSUB = 1u << BT_LOG2_NSUB;  // sub-buckets of the kept keys
constexpr uint32_t BT_SUB_SORT = 32;  // largest sub-bucket sorted by insertion

typedef unsigned __int128 u128;

__device__ __forceinline__ u128 as_u128(uint64_t k) { return (u128)k; }
__device__ __forceinline__ u128 as_u128(Key128 k) { return ((u128)k.hi << 64) | (u128)k.lo; }

template <class K> __device__ __forceinline__ K empty_key();
template <> __device__ __forceinline__ uint64_t empty_key<uint64_t>() { return ~0ull; }
template <> __device__ __forceinline__ Key128 empty_key<Key128>() { return Key128{~0ull, ~0ull}; }
// A canonical key is never all ones: min(x, rc(x)) of the all-T string is the all-A string.

template <uint32_t LOG2>
__device__ __forceinline__ uint32_t slot_hash(uint64_t k) {
    return (uint32_t)((k * 0x9e3779b97f4a7c15ull) >> (64 - LOG2));
}
template <uint32_t LOG2>
__device__ __forceinline__ uint32_t slot_hash(Key128 k) {
    return (uint32_t)(((k.hi * 0xc2b2ae3d27d4eb4full) ^ k.lo) * 0x9e3779b97f4a7c15ull >> (64 - LOG2));
}

// Shared-memory compare-and-swap of a whole key; returns the previous value.
__device__ __forceinline__ uint64_t cas_key(uint64_t *slot, uint64_t expect, uint64_t desired) {
    return atomicCAS(reinterpret_cast<unsigned long long *>(slot), expect, desired);
}
__device__ __forceinline__ Key128 cas_key(Key128 *slot, Key128 expect, Key128 desired) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(slot);
    uint64_t o0, o1;
    // 16-byte atomic (sm_90 and later); the low 64 bits of the operand are the word at the lower
    // address, which is Key128::hi.
    asm volatile(
        "{\n\t.reg .b128 d, c, v;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 v, {%4, %5};\n\t"
        "atom.shared.cas.b128 d, [%6], c, v;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(o0), "=l"(o1)
        : "l"(expect.hi), "l"(expect.lo), "l"(desired.hi), "l"(desired.lo), "r"(a)
        : "memory");
    return Key128{o0, o1};
}

// off[b] = first position of bucket b in keys sorted by bucket (b = 0 .. n_buckets), by binary
// search: the bucket index is non-decreasing along the sorted keys.
template <class K>
__global__ __launch_bounds__(256) void k_bucket_bounds(const K *__restrict__ keys, uint64_t n, BucketGeom g,
                                                       unsigned long long *__restrict__ off) {
    const uint64_t b = (uint64_t)blockIdx.x * 256 + threadIdx.x;
    if (b > g.n_buckets) return;
    uint64_t lo = 0, hi = n;  // first index whose bucket >= b
    if (b == g.n_buckets) lo = n;
    else if (b > 0)
        while (lo < hi) {
            const uint64_t mid = lo + (hi - lo) / 2;
            if (bucket_of(keys[mid], g) < b) lo = mid + 1;
            else hi = mid;
        }
    off[b] = lo;
}

// Exclusive scan of n counters by one CTA; out[n] = total.
constexpr int SCAN_THREADS = 1024, SCAN_ITEMS = 8;
__global__ __launch_bounds__(SCAN_THREADS) void k_scan_u64(const unsigned long long *__restrict__ in, uint64_t n,
                                                           unsigned long long *__restrict__ out) {
    __shared__ unsigned long long warp_sums[SCAN_THREADS / 32];
    __shared__ unsigned long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t base = 0; base < n; base += (uint64_t)SCAN_THREADS * SCAN_ITEMS) {
        unsigned long long v[SCAN_ITEMS], sum = 0;
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; j++) {
            const uint64_t i = base + (uint64_t)threadIdx.x * SCAN_ITEMS + j;
            v[j] = i < n ? in[i] : 0;
            sum += v[j];
        }
        unsigned long long x = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULL, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long s = warp_sums[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long y = __shfl_up_sync(FULL, s, d);
                if (lane >= d) s += y;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        unsigned long long run = s_carry + (warp ? warp_sums[warp - 1] : 0) + x - sum;
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; j++) {
            const uint64_t i = base + (uint64_t)threadIdx.x * SCAN_ITEMS + j;
            if (i < n) out[i] = run;
            run += v[j];
        }
        __syncthreads();
        if (threadIdx.x == 0) s_carry += warp_sums[SCAN_THREADS / 32 - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = s_carry;
}

template <class K, class C>
struct BucketSmem {
    K key[C::SLOTS];
    uint32_t count[C::SLOTS];
    uint16_t list[C::SLOTS];  // claimed slots in claim order
    u128 lo[BT_STACK], hi[BT_STACK];
    uint32_t warp_sums[C::THREADS / 32];
    K wmin[C::THREADS / 32], wmax[C::THREADS / 32];
    uint32_t distinct, overflow, top, bucket, n_rep, sub_max;
    unsigned long long out_at, n_distinct;
};

// +1 on a slot's count, checked against overflow when `check` (a bucket with fewer than 2^32 - 2
// keys cannot overflow a count).
__device__ __forceinline__ void bt_add(uint32_t *count, bool check, uint32_t *err) {
    if (check) {
        if (atomicAdd(count, 1u) >= 0xfffffffeu) atomicOr(err, ERR_COUNT_OVERFLOW);
    } else {
        atomicAdd(count, 1u);
    }
}

// Insert one candidate: claim its slot or add to the slot that holds it. Gives up (returns) once
// the table has been declared over its limit for this attempt. (Reading a 64-bit slot before the
// compare-and-swap, to skip the swap for keys already present, was slower; so was issuing the
// first swaps of a thread's four keys together before settling them.)
template <class K, class C>
__device__ __forceinline__ void bt_insert(BucketSmem<K, C> &sm, K key, bool check, uint32_t *err) {
    const K E = empty_key<K>();
    uint32_t h = slot_hash<C::LOG2>(key);
    for (uint32_t probe = 0; probe < C::SLOTS; probe++) {
        if (*(volatile uint32_t *)&sm.overflow) return;
        const K old = cas_key(&sm.key[h], E, key);
        if (KeyT<K>::eq(old, E)) {  // claimed a new slot
            const uint32_t d = atomicAdd(&sm.distinct, 1u);
            sm.list[d] = (uint16_t)h;  // d < C::LIMIT + C::THREADS < C::SLOTS
            if (d + 1 >= C::LIMIT) sm.overflow = 1;
            atomicAdd(&sm.count[h], 1u);
            return;
        }
        if (KeyT<K>::eq(old, key)) {
            bt_add(&sm.count[h], check, err);
            return;
        }
        h = (h + 1) & (C::SLOTS - 1);
    }
}

// One CTA at a time per bucket, taken in ticket order. Bucket b's candidates are
// cand[off_c[b] .. off_c[b+1]), its first sightings first[off_f[b] .. off_f[b+1]). Output: the
// bucket's kept keys, ascending, with counts, at tmp_* + off_c[b]; their number at n_rep[b].
template <class K, class C>
__global__ __launch_bounds__(C::THREADS, C::MINB) void k_bucket_count(const K *__restrict__ cand,
                                                                 const unsigned long long *__restrict__ off_c,
                                                                 const K *__restrict__ first,
                                                                 const unsigned long long *__restrict__ off_f,
                                                                 uint32_t B, uint32_t min_count,
                                                                 K *__restrict__ tmp_keys,
                                                                 uint32_t *__restrict__ tmp_counts,
                                                                 unsigned long long *__restrict__ n_rep,
                                                                 uint32_t *ticket, unsigned long long *n_distinct,
                                                                 uint32_t *err) {
    static_assert(BT_NSUB % C::THREADS == 0, "sub-bucket scan");
    static_assert(2 * BT_NSUB * 4 <= C::SLOTS * 2, "sub-bucket counters fit in the claim list");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BucketSmem<K, C> &sm = *reinterpret_cast<BucketSmem<K, C> *>(smem_raw);
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const K E = empty_key<K>();
    if (tid == 0) sm.n_distinct = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            sm.bucket = atomicAdd(ticket, 1u);
            sm.top = 1;
            sm.lo[0] = 0;
            sm.hi[0] = ~(u128)0;
            sm.out_at = 0;
        }
        __syncthreads();
        const uint32_t b = sm.bucket;
        if (b >= B) break;
        const uint64_t c0 = off_c[b], c1 = off_c[b + 1];
        const uint64_t f0 = first ? off_f[b] : 0, f1 = first ? off_f[b + 1] : 0;
        // Adds without a returned value where a count cannot reach 2^32 - 2. Measured on this GPU
        // they are faster with 128-bit keys and slower with 64-bit keys (which keep the checked add).
        const bool check = sizeof(K) == 8 || (c1 - c0) + (f1 - f0) >= 0xfffffffeull;
        bool narrowed = false;
        while (sm.top > 0) {  // uniform: every thread reads top after the same barrier
            const u128 lo = sm.lo[sm.top - 1], hi = sm.hi[sm.top - 1];
            __syncthreads();
            for (uint32_t i = tid; i < C::SLOTS; i += C::THREADS) {
                sm.key[i] = E;
                sm.count[i] = 0;
            }
            if (tid == 0) {
                sm.top--;
                sm.distinct = 0;
                sm.overflow = 0;
                sm.n_rep = 0;
            }
            __syncthreads();
            // candidates of this key range -> table
            for (uint64_t i = c0 + tid; i < c1; i += 4 * C::THREADS) {
                K kk[4];
#pragma unroll
                for (int j = 0; j < 4; j++) kk[j] = i + j * C::THREADS < c1 ? cand[i + j * C::THREADS] : E;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const u128 v = as_u128(kk[j]);
                    if (!KeyT<K>::eq(kk[j], E) && v >= lo && v <= hi) bt_insert(sm, kk[j], check, err);
                }
            }
            __syncthreads();
            if (sm.overflow) {
                // too many distinct keys: split the range in two and redo both halves (lower first)
                u128 nlo = lo, nhi = hi;
                if (!narrowed) {  // first split: shrink to the bucket's own key span
                    K mn = E, mx = K{};
                    bool any = false;
                    for (uint64_t i = c0 + tid; i < c1; i += C::THREADS) {
                        const K x = cand[i];
                        if (!any || KeyT<K>::lt(x, mn)) mn = x;
                        if (!any || KeyT<K>::lt(mx, x)) mx = x;
                        any = true;
                    }
                    if (!any) {
                        mn = E;
                        mx = K{};
                    }
                    for (int d = 16; d > 0; d >>= 1) {
                        const K a = shfl_down_key(mn, d), c = shfl_down_key(mx, d);
                        if (KeyT<K>::lt(a, mn)) mn = a;
                        if (KeyT<K>::lt(mx, c)) mx = c;
                    }
                    if (lane == 0) {
                        sm.wmin[warp] = mn;
                        sm.wmax[warp] = mx;
                    }
                    __syncthreads();
                    if (tid == 0) {
                        for (uint32_t w = 1; w < C::THREADS / 32; w++) {
                            if (KeyT<K>::lt(sm.wmin[w], sm.wmin[0])) sm.wmin[0] = sm.wmin[w];
                            if (KeyT<K>::lt(sm.wmax[0], sm.wmax[w])) sm.wmax[0] = sm.wmax[w];
                        }
                    }
                    __syncthreads();
                    const u128 a = as_u128(sm.wmin[0]), c = as_u128(sm.wmax[0]);
                    nlo = a > lo ? a : lo;
                    nhi = c < hi ? c : hi;
                    narrowed = true;
                }
                __syncthreads();
                if (tid == 0) {
                    if (nhi > nlo && sm.top + 2 <= (uint32_t)BT_STACK) {
                        const u128 mid = nlo + (nhi - nlo) / 2;
                        sm.lo[sm.top] = mid + 1;
                        sm.hi[sm.top] = nhi;
                        sm.lo[sm.top + 1] = nlo;
                        sm.hi[sm.top + 1] = mid;
                        sm.top += 2;
                    } else {
                        atomicOr(err, ERR_TABLE_FULL);  // cannot happen: one key is one slot
                    }
                }
                __syncthreads();
                continue;
            }
            // first sightings of this key range: +1 for keys that are candidates too
            for (uint64_t i = f0 + tid; i < f1; i += 4 * C::THREADS) {
                K xs[4];
#pragma unroll
                for (int j = 0; j < 4; j++) xs[j] = i + j * C::THREADS < f1 ? first[i + j * C::THREADS] : E;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const K x = xs[j];
                    const u128 v = as_u128(x);
                    if (KeyT<K>::eq(x, E) || v < lo || v > hi) continue;
                    uint32_t h = slot_hash<C::LOG2>(x);
                    for (uint32_t probe = 0; probe < C::SLOTS; probe++) {
                        const K y = sm.key[h];
                        if (KeyT<K>::eq(y, x)) {
                            bt_add(&sm.count[h], check, err);
                            break;
                        }
                        if (KeyT<K>::eq(y, E)) break;
                        h = (h + 1) & (C::SLOTS - 1);
                    }
                }
            }
            __syncthreads();
            // keep count >= min_count: gather to registers, then rewrite the arrays as a dense list
            const uint32_t nd = sm.distinct;
            K ik[C::ITEMS];
            uint32_t ic[C::ITEMS], kept = 0;
#pragma unroll
            for (uint32_t j = 0; j < C::ITEMS; j++) {
                const uint32_t e = tid + j * C::THREADS;
                ic[j] = 0;
                if (e < nd) {
                    const uint32_t h = sm.list[e];
                    ik[j] = sm.key[h];
                    ic[j] = sm.count[h];
                    if (ic[j] >= min_count) kept++;
                    else ic[j] = 0;
                }
            }
            uint32_t total;
            uint32_t pos = block_exclusive_scan<C::THREADS>(kept, sm.warp_sums, &total);
            // Sort the kept keys. Common case: sub-buckets by the leading bits of (key - min) (counting
            // sort), then an insertion sort inside each (a few keys). Skewed keys: bitonic sort.
            uint32_t *sub_cnt = reinterpret_cast<uint32_t *>(sm.list);  // the claim list is no longer needed
            uint32_t *sub_off = sub_cnt + BT_NSUB;
            {
                K mn = E, mx = K{};
#pragma unroll
                for (uint32_t j = 0; j < C::ITEMS; j++)
                    if (ic[j]) {
                        if (KeyT<K>::lt(ik[j], mn)) mn = ik[j];
                        if (KeyT<K>::lt(mx, ik[j])) mx = ik[j];
                    }
                for (int d = 16; d > 0; d >>= 1) {
                    const K a = shfl_down_key(mn, d), c = shfl_down_key(mx, d);
                    if (KeyT<K>::lt(a, mn)) mn = a;
                    if (KeyT<K>::lt(mx, c)) mx = c;
                }
                if (lane == 0) {
                    sm.wmin[warp] = mn;
                    sm.wmax[warp] = mx;
                }
                for (uint32_t d = tid; d < BT_NSUB; d += C::THREADS) sub_cnt[d] = 0;
                if (tid == 0) sm.sub_max = 0;
                __syncthreads();
                if (tid == 0) {
                    for (uint32_t w = 1; w < C::THREADS / 32; w++) {
                        if (KeyT<K>::lt(sm.wmin[w], sm.wmin[0])) sm.wmin[0] = sm.wmin[w];
                        if (KeyT<K>::lt(sm.wmax[0], sm.wmax[w])) sm.wmax[0] = sm.wmax[w];
                    }
                }
                __syncthreads();
            }
            const u128 kmin = as_u128(sm.wmin[0]);
            const u128 span = total ? as_u128(sm.wmax[0]) - kmin : 0;
            const int span_bits = (uint64_t)(span >> 64) ? 128 - __clzll((long long)(uint64_t)(span >> 64))
                                                          : 64 - __clzll((long long)(uint64_t)span);
            const int sub_shift = span_bits > BT_LOG2_NSUB ? span_bits - BT_LOG2_NSUB : 0;
            uint32_t packed[C::ITEMS];  // sub-bucket | rank inside it << BT_LOG2_NSUB
#pragma unroll
            for (uint32_t j = 0; j < C::ITEMS; j++)
                if (ic[j]) {
                    const uint32_t d = (uint32_t)((as_u128(ik[j]) - kmin) >> sub_shift);
                    const uint32_t r = atomicAdd(&sub_cnt[d], 1u);
                    if (r + 1 > BT_SUB_SORT) atomicMax(&sm.sub_max, r + 1);
                    packed[j] = d | (r << BT_LOG2_NSUB);
                }
            __syncthreads();
            if (sm.sub_max == 0) {
                constexpr uint32_t PER = BT_NSUB / C::THREADS;
                uint32_t v[PER], sum = 0;
#pragma unroll
                for (uint32_t q = 0; q < PER; q++) {
                    v[q] = sub_cnt[tid * PER + q];
                    sum += v[q];
                }
                uint32_t run = block_exclusive_scan<C::THREADS>(sum, sm.warp_sums, nullptr);
#pragma unroll
                for (uint32_t q = 0; q < PER; q++) {
                    sub_off[tid * PER + q] = run;
                    run += v[q];
                }
                __syncthreads();
#pragma unroll
                for (uint32_t j = 0; j < C::ITEMS; j++)
                    if (ic[j]) {
                        const uint32_t d = packed[j] & (BT_NSUB - 1), dst = sub_off[d] + (packed[j] >> BT_LOG2_NSUB);
                        sm.key[dst] = ik[j];
                        sm.count[dst] = ic[j];
                    }
                __syncthreads();
                for (uint32_t d = tid; d < BT_NSUB; d += C::THREADS) {
                    const uint32_t a = sub_off[d], m = sub_cnt[d];
                    for (uint32_t x = 1; x < m; x++) {
                        const K key = sm.key[a + x];
                        const uint32_t cnt = sm.count[a + x];
                        uint32_t y = x;
                        while (y > 0 && KeyT<K>::lt(key, sm.key[a + y - 1])) {
                            sm.key[a + y] = sm.key[a + y - 1];
                            sm.count[a + y] = sm.count[a + y - 1];
                            y--;
                        }
                        sm.key[a + y] = key;
                        sm.count[a + y] = cnt;
                    }
                }
                __syncthreads();
            } else {
                uint32_t N = 1;
                while (N < total) N <<= 1;
#pragma unroll
                for (uint32_t j = 0; j < C::ITEMS; j++)
                    if (ic[j]) {
                        sm.key[pos] = ik[j];
                        sm.count[pos] = ic[j];
                        pos++;
                    }
                for (uint32_t i = total + tid; i < N; i += C::THREADS) {
                    sm.key[i] = E;
                    sm.count[i] = 0;
                }
                __syncthreads();
                // bitonic sort of the kept keys (N <= C::SLOTS)
                for (uint32_t size = 2; size <= N; size <<= 1) {
                    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
                        for (uint32_t t = tid; t < N / 2; t += C::THREADS) {
                            const uint32_t i = 2 * t - (t & (stride - 1)), j = i + stride;
                            const bool up = (i & size) == 0;
                            const K a = sm.key[i], c = sm.key[j];
                            if (KeyT<K>::lt(c, a) == up) {
                                sm.key[i] = c;
                                sm.key[j] = a;
                                const uint32_t t0 = sm.count[i];
                                sm.count[i] = sm.count[j];
                                sm.count[j] = t0;
                            }
                        }
                        __syncthreads();
                    }
                }
            }
            const uint64_t at = c0 + sm.out_at;
            for (uint32_t i = tid; i < total; i += C::THREADS) {
                tmp_keys[at + i] = sm.key[i];
                tmp_counts[at + i] = sm.count[i];
            }
            __syncthreads();
            if (tid == 0) {
                sm.out_at += total;
                sm.n_distinct += nd;
            }
        }
        __syncthreads();
        if (tid == 0) n_rep[b] = sm.out_at;
    }
    if (tid == 0 && sm.n_distinct) atomicAdd(n_distinct, sm.n_distinct);
}

template <class K>
__global__ __launch_bounds__(256) void k_bucket_gather(const K *__restrict__ tmp_keys,
                                                       const uint32_t *__restrict__ tmp_counts,
                                                       const unsigned long long *__restrict__ off,
                                                       const unsigned long long *__restrict__ out_off, uint32_t B,
                                                       K *__restrict__ okeys, uint32_t *__restrict__ ocounts) {
    for (uint32_t b = blockIdx.x; b < B; b += gridDim.x) {
        const uint64_t src = off[b], dst = out_off[b], n = out_off[b + 1] - dst;
        for (uint64_t i = threadIdx.x; i < n; i += 256) {
            okeys[dst + i] = tmp_keys[src + i];
            ocounts[dst + i] = tmp_counts[src + i];
        }
    }
}

}  // namespace

template <class K>
void launch_bucket_bounds(const LaunchCfg &c, const K *keys, uint64_t n, const BucketGeom &g,
                          unsigned long long *off) {
    const unsigned grid = (unsigned)((g.n_buckets + 1 + 255) / 256);
    k_bucket_bounds<K><<<grid, 256, 0, c.stream>>>(keys, n, g, off);
}

void launch_scan_u64(const LaunchCfg &c, const unsigned long long *in, uint64_t n, unsigned long long *out) {
    k_scan_u64<<<1, SCAN_THREADS, 0, c.stream>>>(in, n, out);
}

template <class K, class C>
static void bucket_count_cfg(const LaunchCfg &c, const K *cand, const unsigned long long *off_c, const K *first,
                             const unsigned long long *off_f, uint32_t B, uint32_t min_count, K *tmp_keys,
                             uint32_t *tmp_counts, unsigned long long *n_rep, uint32_t *ticket,
                             unsigned long long *n_distinct, uint32_t *err) {
    const size_t smem = sizeof(BucketSmem<K, C>);  // above the 48 KB default: opt in (per device, cheap)
    cudaFuncSetAttribute(k_bucket_count<K, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const unsigned grid = (unsigned)std::min<uint64_t>(B, (uint64_t)c.sms * C::MINB);
    k_bucket_count<K, C><<<grid, C::THREADS, smem, c.stream>>>(cand, off_c, first, off_f, B, min_count, tmp_keys,
                                                                 tmp_counts, n_rep, ticket, n_distinct, err);
}

template <class K>
void launch_bucket_count(const LaunchCfg &c, const K *cand, const unsigned long long *off_c, const K *first,
                         const unsigned long long *off_f, uint32_t B, uint32_t min_count, K *tmp_keys,
                         uint32_t *tmp_counts, unsigned long long *n_rep, uint32_t *ticket,
                         unsigned long long *n_distinct, uint32_t *err, int large) {
    if (!B) return;
    if (large)
        bucket_count_cfg<K, BtLarge>(c, cand, off_c, first, off_f, B, min_count, tmp_keys, tmp_counts, n_rep, ticket,
                                     n_distinct, err);
    else
        bucket_count_cfg<K, BtSmall>(c, cand, off_c, first, off_f, B, min_count, tmp_keys, tmp_counts, n_rep, ticket,
                                     n_distinct, err);
}

template <class K>
void launch_bucket_gather(const LaunchCfg &c, const K *tmp_keys, const uint32_t *tmp_counts,
                          const unsigned long long *off, const unsigned long long *out_off, uint32_t B, K *okeys,
                          uint32_t *ocounts) {
    if (!B) return;
    const unsigned grid = (unsigned)std::min<uint64_t>(B, (uint64_t)c.sms * 8);
    k_bucket_gather<K><<<grid, 256, 0, c.stream>>>(tmp_keys, tmp_counts, off, out_off, B, okeys, ocounts);
}

#define INST(K)                                                                                                   \
    template void launch_bucket_bounds<K>(const LaunchCfg &, const K *, uint64_t, const BucketGeom &,             \
                                          unsigned long long *);                                                   \
    template void launch_bucket_count<K>(const LaunchCfg &, const K *, const unsigned long long *, const K *,      \
                                         const unsigned long long *, uint32_t, uint32_t, K *, uint32_t *,          \
                                         unsigned long long *, uint32_t *, unsigned long long *, uint32_t *, int); \
    template void launch_bucket_gather<K>(const LaunchCfg &, const K *, const uint32_t *,                          \
                                          const unsigned long long *, const unsigned long long *, uint32_t, K *,   \
                                          uint32_t *);
INST(uint64_t)
INST(Key128)
#undef INST

}  // namespace turtle
