// Device-side building blocks shared by the libturtle kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace turtle {

// ---------------------------------------------------------------- error word bits (device -> host)
enum : uint32_t {
    ERR_LOOKBACK = 1u,        // a decoupled look-back wait hit its iteration limit
    ERR_CAND_OVERFLOW = 2u,   // candidate buffer full (cannot happen with the planned capacity)
    ERR_TABLE_FULL = 4u,      // recount table had no free slot
    ERR_COUNT_OVERFLOW = 8u,  // a uint32 count reached 2^32-1
    ERR_BAD_OFFSETS = 16u,    // offsets not monotone or past n_bases
    ERR_NOT_FOUND = 32u,      // threshold lookup missed a key that was inserted
    ERR_PART_MISMATCH = 64u,  // a window's key-range test disagreed with its canonical key's range
    ERR_BULK_WAIT = 128u,     // a bulk copy into shared memory did not complete within its wait limit
};

constexpr int WARP = 32;
constexpr uint32_t FULL = 0xffffffffu;
constexpr uint32_t EMPTY_COUNT = 0xffffffffu;  // table slot marker

// ---------------------------------------------------------------- keys
// 64-bit keys for k <= 32, {hi, lo} pairs for 33 <= k <= 64 (Sec. 3 of the paper: 64- and 128-bit integers).
struct alignas(16) Key128 {
    uint64_t hi, lo;
};

template <class K> struct KeyT;

template <> struct KeyT<uint64_t> {
    static constexpr int WORDS = 1;
    __device__ __forceinline__ static bool lt(uint64_t a, uint64_t b) { return a < b; }
    __device__ __forceinline__ static bool eq(uint64_t a, uint64_t b) { return a == b; }
    __device__ __forceinline__ static uint32_t digit(uint64_t a, int shift) { return (uint32_t)(a >> shift) & 0xffu; }
};
template <> struct KeyT<Key128> {
    static constexpr int WORDS = 2;
    __device__ __forceinline__ static bool lt(Key128 a, Key128 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
    __device__ __forceinline__ static bool eq(Key128 a, Key128 b) { return a.hi == b.hi && a.lo == b.lo; }
    __device__ __forceinline__ static uint32_t digit(Key128 a, int shift) {
        return shift < 64 ? (uint32_t)(a.lo >> shift) & 0xffu : (uint32_t)(a.hi >> (shift - 64)) & 0xffu;
    }
};

// MurmurHash3 64-bit finaliser (Appleby, public domain).
__device__ __forceinline__ uint64_t fmix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}
__device__ __forceinline__ uint64_t key_hash(uint64_t k) { return fmix64(k); }
__device__ __forceinline__ uint64_t key_hash(Key128 k) { return fmix64(k.lo ^ fmix64(k.hi)); }

// Reverse the order of the 32 two-bit digits of x (digit 0 <-> digit 31).
__device__ __forceinline__ uint64_t rev2(uint64_t x) {
    uint64_t y = __brevll(x);  // bit-reverse, then restore the bit order inside each digit
    return ((y >> 1) & 0x5555555555555555ull) | ((y & 0x5555555555555555ull) << 1);
}

// Packed layout: word w holds bases 32w..32w+31, base 32w+j in bits (63-2j, 62-2j).
// The 64 bits starting at bit offset o (0..62, even) of the big-endian stream P[w], P[w+1].
__device__ __forceinline__ uint64_t stream_bits(uint64_t a, uint64_t b, int o) {
    return (a << o) | ((b >> 1) >> (63 - o));
}

// Canonical key of the window starting at position s (Sec. 2.1.2): fwd has the
// first base most significant; rc is the reverse complement; keep the smaller.
__device__ __forceinline__ uint64_t canonical_at(const uint64_t *__restrict__ P, uint64_t s, int k, uint64_t *fwd_out = nullptr) {
    const uint64_t w = s >> 5;
    const int o = (int)(s & 31) << 1;
    const uint64_t top = stream_bits(__ldg(P + w), __ldg(P + w + 1), o);
    const int drop = 64 - 2 * k;
    const uint64_t fwd = top >> drop;
    const uint64_t rc = (~rev2(fwd)) >> drop;
    if (fwd_out) *fwd_out = fwd;
    return fwd < rc ? fwd : rc;
}

__device__ __forceinline__ Key128 canonical_at128(const uint64_t *__restrict__ P, uint64_t s, int k) {
    const uint64_t w = s >> 5;
    const int o = (int)(s & 31) << 1;
    const uint64_t p0 = __ldg(P + w), p1 = __ldg(P + w + 1), p2 = __ldg(P + w + 2);
    unsigned __int128 top = ((unsigned __int128)stream_bits(p0, p1, o) << 64) | stream_bits(p1, p2, o);
    const int drop = 128 - 2 * k;  // 0..62 for k in 33..64
    unsigned __int128 fwd = top >> drop;
    unsigned __int128 r = ((unsigned __int128)rev2((uint64_t)fwd) << 64) | rev2((uint64_t)(fwd >> 64));
    unsigned __int128 rc = (~r) >> drop;
    unsigned __int128 m = fwd < rc ? fwd : rc;
    Key128 out;
    out.hi = (uint64_t)(m >> 64);
    out.lo = (uint64_t)m;
    return out;
}

template <class K> __device__ __forceinline__ K canonical(const uint64_t *__restrict__ P, uint64_t s, int k);
template <> __device__ __forceinline__ uint64_t canonical<uint64_t>(const uint64_t *__restrict__ P, uint64_t s, int k) {
    return canonical_at(P, s, k);
}
template <> __device__ __forceinline__ Key128 canonical<Key128>(const uint64_t *__restrict__ P, uint64_t s, int k) {
    return canonical_at128(P, s, k);
}

// ---------------------------------------------------------------- key-range parts
// Monotone map of a canonical key to [0, 2^62): v = top 31 bits of the 2k-bit key,
// f(v) = v * (2^32 - v), which is increasing on [0, 2^31). For random sequence the
// canonical key min(x, rc(x)) has density 2(1 - u) on u in [0, 1), whose CDF
// u(2 - u) equals f(v) / 2^62: equal slices of f hold about equal numbers of keys.
// Part p of 2^bits takes the keys with f(v) >> (62 - bits) == p; since f is
// monotone, parts are ordered key ranges.
// (Bits above the 2k key bits, i.e. a batch's library tag, are masked off.)
__device__ __forceinline__ uint64_t top31(uint64_t key, int k) {
    const int b = 2 * k;
    return (b >= 31 ? key >> (b - 31) : key << (31 - b)) & 0x7fffffffull;
}
__device__ __forceinline__ uint64_t top31(Key128 key, int k) {
    const int b = 2 * k;  // 2..128 bits (a mixed batch also keeps short keys in 128 bits)
    if (b < 31) return (key.lo << (31 - b)) & 0x7fffffffull;
    const int sh = b - 31;  // 1..97: the top 31 bits lie in lo, straddle hi/lo, or lie in hi
    if (sh >= 64) return (key.hi >> (sh - 64)) & 0x7fffffffull;
    return ((key.hi << (64 - sh)) | (key.lo >> sh)) & 0x7fffffffull;
}
template <class K>
__device__ __forceinline__ uint32_t key_part(K key, int k, int part_bits) {
    if (part_bits == 0) return 0;
    const uint64_t v = top31(key, k);
    return (uint32_t)((v * ((1ull << 32) - v)) >> (62 - part_bits));
}

// ---------------------------------------------------------------- library tags (batched form)
// A batch of libraries is one position range per library; a window's key carries its library
// index in the bits just above the 2k key bits, so libraries never mix in any later step.
__device__ __forceinline__ uint64_t add_tag(uint64_t key, uint32_t lib, int shift) {
    return key | ((uint64_t)lib << shift);
}
__device__ __forceinline__ Key128 add_tag(Key128 key, uint32_t lib, int shift) {
    if (shift >= 64) key.hi |= (uint64_t)lib << (shift - 64);
    else {
        key.lo |= (uint64_t)lib << shift;
        if (shift > 0) key.hi |= (uint64_t)lib >> (64 - shift);
    }
    return key;
}

template <class K>
__device__ __forceinline__ uint32_t tag_of(const K &key, int shift) {
    if constexpr (sizeof(K) == 8) return (uint32_t)(key >> shift);  // shift < 64 whenever a tag is present
    else return (uint32_t)(key.hi >> (shift - 64));                // tags of 128-bit runs sit in hi (2k >= 66)
}

// ---------------------------------------------------------------- key loads/stores
__device__ __forceinline__ uint64_t load_stream(const uint64_t *p) { return __ldcs(p); }  // read once
__device__ __forceinline__ Key128 load_stream(const Key128 *p) {
    const ulonglong2 v = __ldcs(reinterpret_cast<const ulonglong2 *>(p));
    Key128 k;
    k.hi = v.x;
    k.lo = v.y;
    return k;
}
__device__ __forceinline__ uint64_t shfl_key(uint64_t k, int src) { return __shfl_sync(FULL, k, src); }
__device__ __forceinline__ Key128 shfl_key(Key128 k, int src) {
    Key128 r;
    r.hi = __shfl_sync(FULL, k.hi, src);
    r.lo = __shfl_sync(FULL, k.lo, src);
    return r;
}
__device__ __forceinline__ uint64_t shfl_down_key(uint64_t k, int d) { return __shfl_down_sync(FULL, k, d); }
__device__ __forceinline__ Key128 shfl_down_key(Key128 k, int d) {
    Key128 r;
    r.hi = __shfl_down_sync(FULL, k.hi, d);
    r.lo = __shfl_down_sync(FULL, k.lo, d);
    return r;
}
__device__ __forceinline__ uint64_t shfl_up_key(uint64_t k) { return __shfl_up_sync(FULL, k, 1); }
__device__ __forceinline__ Key128 shfl_up_key(Key128 k) {
    Key128 r;
    r.hi = __shfl_up_sync(FULL, k.hi, 1);
    r.lo = __shfl_up_sync(FULL, k.lo, 1);
    return r;
}
__device__ __forceinline__ void store_key(uint64_t *p, uint64_t k) { *p = k; }
__device__ __forceinline__ void store_key(Key128 *p, Key128 k) { *p = k; }

// ---------------------------------------------------------------- relaxed GPU-scope accesses
__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------- decoupled look-back (single value)
// Status word: bits 63..62 state (1 = tile aggregate, 2 = inclusive prefix), bits 61..40 epoch,
// bits 39..0 value. The epoch separates uses of one zeroed array (e.g. sort passes).
constexpr uint64_t LB_AGG = 1ull << 62, LB_INC = 2ull << 62;
constexpr uint64_t LB_VALUE = (1ull << 40) - 1;
constexpr uint32_t LB_SPIN_LIMIT = 1u << 22;  // iterations with nanosleep back-off: well over a second

__device__ __forceinline__ uint64_t lb_pack(uint64_t state, uint32_t epoch, uint64_t v) {
    return state | ((uint64_t)(epoch & 0x3fffffu) << 40) | (v & LB_VALUE);
}

// Exclusive prefix of tile `tile` given its aggregate; publishes the inclusive prefix.
// Status of tile j lives at status[j * stride]. Waits on predecessors (bounded: on
// expiry sets ERR_LOOKBACK and continues with what it has, so the kernel always ends).
__device__ __forceinline__ uint64_t lookback_prefix(uint64_t *status, uint64_t stride, uint64_t tile,
                                                    uint64_t aggregate, uint32_t epoch, uint32_t *err) {
    if (tile == 0) {
        st_relaxed(status, lb_pack(LB_INC, epoch, aggregate));
        return 0;
    }
    st_relaxed(status + tile * stride, lb_pack(LB_AGG, epoch, aggregate));
    uint64_t excl = 0;
    int64_t j = (int64_t)tile - 1;
    uint32_t spins = 0;
    while (j >= 0) {
        const uint64_t v = ld_relaxed(status + (uint64_t)j * stride);
        const uint32_t ep = (uint32_t)(v >> 40) & 0x3fffffu;
        const uint64_t st = v & (3ull << 62);
        if (ep != (epoch & 0x3fffffu) || st == 0) {
            if (++spins > LB_SPIN_LIMIT) {
                atomicOr(err, ERR_LOOKBACK);
                break;
            }
            __nanosleep(32);
            continue;
        }
        excl += v & LB_VALUE;
        if (st == LB_INC) break;
        --j;
    }
    st_relaxed(status + tile * stride, lb_pack(LB_INC, epoch, excl + aggregate));
    return excl;
}

// Warp-wide decoupled look-back: all 32 lanes of ONE warp call this; lane l inspects
// predecessor tile-1-l, so one round trip covers 32 predecessors. Returns the exclusive
// prefix in every lane and publishes the inclusive one. Bounded like lookback_prefix.
__device__ __forceinline__ uint64_t lookback_prefix_warp(uint64_t *status, uint64_t tile, uint64_t aggregate,
                                                         uint32_t epoch, uint32_t *err,
                                                         uint32_t spin_limit = LB_SPIN_LIMIT) {
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) st_relaxed(status, lb_pack(LB_INC, epoch, aggregate));
        return 0;
    }
    if (lane == 0) st_relaxed(status + tile, lb_pack(LB_AGG, epoch, aggregate));
    uint64_t excl = 0;
    int64_t base = (int64_t)tile - 1;
    uint32_t spins = 0;
    while (base >= 0) {
        const int64_t j = base - lane;
        uint64_t v = 0;
        bool ready = true, inc = true;  // lanes before tile 0 act as an inclusive prefix of 0
        if (j >= 0) {
            v = ld_relaxed(status + j);
            const uint64_t st = v & (3ull << 62);
            ready = ((uint32_t)(v >> 40) & 0x3fffffu) == (epoch & 0x3fffffu) && st != 0;
            inc = ready && st == LB_INC;
        }
        const uint32_t inc_mask = __ballot_sync(FULL, inc);
        const uint32_t ready_mask = __ballot_sync(FULL, ready);
        const int first_inc = inc_mask ? __ffs(inc_mask) - 1 : 32;  // nearest predecessor with a prefix
        const uint32_t need = first_inc >= 31 ? FULL : ((2u << first_inc) - 1u);
        if ((ready_mask & need) != need) {
            if (++spins > spin_limit) {
                if (lane == 0) atomicOr(err, ERR_LOOKBACK);
                break;
            }
            __nanosleep(32);
            continue;
        }
        uint64_t c = (lane <= first_inc && j >= 0) ? (v & LB_VALUE) : 0;
#pragma unroll
        for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(FULL, c, d);
        excl += c;
        if (first_inc < 32) break;
        base -= 32;
    }
    if (lane == 0) st_relaxed(status + tile, lb_pack(LB_INC, epoch, excl + aggregate));
    return excl;
}

// Block-wide exclusive scan of one uint32 per thread (blockDim.x == BLOCK, a multiple of 32).
template <int BLOCK>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_sums /* BLOCK/32 */, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < BLOCK / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, s, d);
            if (lane >= d) s += y;
        }
        if (lane < BLOCK / 32) warp_sums[lane] = s;  // inclusive warp prefix
    }
    __syncthreads();
    uint32_t before = warp ? warp_sums[warp - 1] : 0;
    if (total) *total = warp_sums[BLOCK / 32 - 1];
    return before + x - v;
}

}  // namespace turtle
