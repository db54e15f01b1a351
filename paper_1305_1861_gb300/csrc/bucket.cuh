// Bucket index of a key for the bucketed sort-and-compact (device side).
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace turtle {

// ((f(v) - f_lo) >> shift) clamped to [0, n_buckets), v = top 31 bits of the 2k-bit key,
// f(v) = v (2^32 - v): monotone in the key, so buckets are consecutive key ranges, and about
// equally full for the canonical keys of random sequence. Tagged keys (batches) first select
// their library's range of buckets; tags are the most significant key bits, so the order holds.
template <class K>
__device__ __forceinline__ uint32_t bucket_of(K key, const BucketGeom &g) {
    if (g.lib) {
        const uint4 e = __ldg(g.lib + tag_of(key, g.tag_shift));
        const uint64_t v = top31(key, e.w ? (int)e.w : g.k);  // a mixed batch: the library's own k
        const uint64_t b = (v * ((1ull << 32) - v)) >> e.z;
        return e.x + (b < e.y ? (uint32_t)b : e.y - 1);
    }
    const uint64_t v = top31(key, g.k);
    const uint64_t f = v * ((1ull << 32) - v);
    const uint64_t b = f >= g.f_lo ? (f - g.f_lo) >> g.shift : 0;
    return b < g.n_buckets ? (uint32_t)b : g.n_buckets - 1;
}

// Radix digit policies for the onesweep passes: a byte of the key, or a byte of its bucket index.
// same_low(x, y, shift): x and y agree in every digit below `shift` (what earlier passes sorted by).
template <class K>
struct RawDigit {
    __device__ __forceinline__ uint32_t operator()(K key, int shift) const { return KeyT<K>::digit(key, shift); }
    __device__ __forceinline__ bool same_low(K x, K y, int shift) const {
        for (int s = 0; s < shift; s += 8)
            if (KeyT<K>::digit(x, s) != KeyT<K>::digit(y, s)) return false;
        return true;
    }
};
template <class K>
struct BucketDigit {
    BucketGeom g;
    __device__ __forceinline__ uint32_t operator()(K key, int shift) const {
        return (bucket_of(key, g) >> shift) & 0xffu;
    }
    __device__ __forceinline__ bool same_low(K x, K y, int shift) const {
        const uint32_t m = shift ? 0xffffffffu >> (32 - shift) : 0u;
        return ((bucket_of(x, g) ^ bucket_of(y, g)) & m) == 0;
    }
};

}  // namespace turtle
