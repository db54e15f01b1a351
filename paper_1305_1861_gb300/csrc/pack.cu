// Step a1/a2 support: ASCII reads -> 2-bit codes + bitmaps; valid-window bitmap; per-window keys.
//
// Sec. 2.1.2: k-mers are 2-bit encoded and taken from reads split at ambiguous
// calls. Here every base position of the concatenated library gets a 2-bit code
// (P), a "bad" bit (B: not A/C/G/T, or outside [offsets[0], offsets[n_reads])) and
// a read-start bit (S). A window [s, s+k) is valid iff no bad bit lies in
// [s, s+k) and no read starts in (s, s+k); V holds one bit per start s.
#include <cstdio>

#include "common.cuh"
#include "kernels.h"

namespace turtle {

// 4 ASCII bytes (first base in the low byte) -> 8-bit code group (first base most significant)
// and 4 bad bits (bit j for byte j).
__device__ __forceinline__ void decode4(uint32_t x, uint32_t &codes8, uint32_t &bad4) {
    const uint32_t u = x & 0xDFDFDFDFu;  // fold lower case onto upper case
    const uint32_t ok = __vcmpeq4(u, 0x41414141u) | __vcmpeq4(u, 0x43434343u) | __vcmpeq4(u, 0x47474747u) |
                        __vcmpeq4(u, 0x54545454u);
    const uint32_t t = (u >> 1) & 0x03030303u;          // A->0 C->1 G->3 T->2
    const uint32_t c = t ^ ((t >> 1) & 0x01010101u);   // A->0 C->1 G->2 T->3
    codes8 = ((c & 3u) << 6) | (((c >> 8) & 3u) << 4) | (((c >> 16) & 3u) << 2) | ((c >> 24) & 3u);
    const uint32_t nb = ~ok;
    bad4 = ((nb >> 7) & 1u) | ((nb >> 14) & 2u) | ((nb >> 21) & 4u) | ((nb >> 28) & 8u);
}

// One thread per group of 32 positions: P[g] (uint64) and 32 bad bits (half of a B word).
// `bases` is indexed by absolute position; for a streamed chunk it is the staging buffer
// shifted back by the chunk's first position, and only groups [g_begin, g_end) are touched.
__global__ void __launch_bounds__(256) k_pack(const uint8_t *__restrict__ bases, uint64_t n_bases,
                                              const uint64_t *__restrict__ offsets, uint64_t n_reads,
                                              uint64_t g_begin, uint64_t g_end, uint64_t *__restrict__ P,
                                              uint32_t *__restrict__ B32) {
    const uint64_t lo = offsets[0], hi = offsets[n_reads] < n_bases ? offsets[n_reads] : n_bases;
    const bool aligned = (((uintptr_t)bases) & 15u) == 0;
    for (uint64_t g = g_begin + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < g_end;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t p0 = g * 32;
        uint32_t w[8];
        if (aligned && p0 + 32 <= n_bases) {
            const uint4 a = __ldcs(reinterpret_cast<const uint4 *>(bases + p0));
            const uint4 b = __ldcs(reinterpret_cast<const uint4 *>(bases + p0 + 16));
            w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
            w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
        } else {
#pragma unroll
            for (int i = 0; i < 8; i++) {
                uint32_t v = 0;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const uint64_t p = p0 + 4 * i + j;
                    v |= (uint32_t)(p < n_bases ? bases[p] : (uint8_t)'N') << (8 * j);
                }
                w[i] = v;
            }
        }
        uint64_t packed = 0;
        uint32_t bad = 0;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            uint32_t c8, b4;
            decode4(w[i], c8, b4);
            packed |= (uint64_t)c8 << (56 - 8 * i);
            bad |= b4 << (4 * i);
        }
        // positions outside [lo, hi) belong to no read
        if (p0 < lo) bad |= (lo >= p0 + 32) ? 0xffffffffu : ((1u << (lo - p0)) - 1u);
        if (p0 + 32 > hi) bad |= (hi <= p0) ? 0xffffffffu : ~((1u << (hi - p0)) - 1u);
        P[g] = packed;
        B32[g] = bad;
    }
}

// Read-start bits and offsets validation. One thread per offsets entry.
__global__ void k_mark_starts(const uint64_t *__restrict__ offsets, uint64_t n_reads, uint64_t n_bases,
                              uint32_t *__restrict__ S32, uint32_t *err) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r <= n_reads;
         r += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t p = offsets[r];
        if (r < n_reads && offsets[r + 1] < p) atomicOr(err, ERR_BAD_OFFSETS);
        if (p > n_bases) atomicOr(err, ERR_BAD_OFFSETS);
        if (r > 0 && r < n_reads && p < n_bases) atomicOr(S32 + (p >> 5), 1u << (p & 31));
    }
}

// OR of x >> j for j in [0, len) (bit s of the result covers positions s .. s+len-1).
__device__ __forceinline__ unsigned __int128 smear(unsigned __int128 x, int len) {
    unsigned __int128 acc = 0, cur = x;
    int span = 1, off = 0;
    while (len) {
        if (len & 1) {
            acc |= cur >> off;
            off += span;
        }
        cur |= cur >> span;
        span <<= 1;
        len >>= 1;
    }
    return acc;
}

__global__ void __launch_bounds__(256) k_valid(const uint64_t *__restrict__ B, const uint64_t *__restrict__ S,
                                               uint64_t w_begin, uint64_t w_end, int k, uint64_t *__restrict__ V,
                                               unsigned long long *n_windows) {
    uint32_t mine = 0;
    for (uint64_t i = w_begin + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < w_end;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned __int128 b = ((unsigned __int128)B[i + 1] << 64) | B[i];
        const unsigned __int128 s = ((unsigned __int128)S[i + 1] << 64) | S[i];
        const uint64_t badspan = (uint64_t)smear(b, k);
        const uint64_t startspan = (uint64_t)smear(s >> 1, k - 1);
        const uint64_t v = ~(badspan | startspan);
        V[i] = v;
        mine += __popcll(v);
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) mine += __shfl_xor_sync(FULL, mine, d);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(n_windows, (unsigned long long)mine);
}

template <class K>
__global__ void __launch_bounds__(256) k_extract(const uint64_t *__restrict__ P, const uint64_t *__restrict__ V,
                                                 uint64_t n_pos, int k, K *__restrict__ keys) {
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n_pos;
         s += (uint64_t)gridDim.x * blockDim.x) {
        if ((V[s >> 6] >> (s & 63)) & 1) keys[s] = canonical<K>(P, s, k);
    }
}

// Per-library valid-window counts: each 64-position word is split among the libraries it touches.
__global__ void __launch_bounds__(256) k_lib_windows(const uint64_t *__restrict__ V, uint64_t n_words,
                                                     const uint64_t *__restrict__ lib_starts, int n_libs,
                                                     unsigned long long *counts) {
    // The library table and the counts stay in shared memory: one global add per block and library
    // (a global add per word would serialise on the few library counters).
    __shared__ uint64_t s_lib[65];
    __shared__ unsigned long long s_cnt[64];
    for (int i = threadIdx.x; i <= n_libs; i += blockDim.x) s_lib[i] = lib_starts[i];
    for (int i = threadIdx.x; i < n_libs; i += blockDim.x) s_cnt[i] = 0;
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_words;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = V[i];
        if (!v) continue;
        const uint64_t p0 = i * 64, p1 = p0 + 64;
        int lo = 0, hi = n_libs;  // library holding p0
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_lib[mid] <= p0) lo = mid;
            else hi = mid;
        }
        for (int l = lo; l < n_libs && s_lib[l] < p1; l++) {
            const uint64_t a = s_lib[l] > p0 ? s_lib[l] - p0 : 0;
            const uint64_t b = s_lib[l + 1] < p1 ? s_lib[l + 1] - p0 : 64;
            if (b <= a) continue;
            const uint64_t m = (b - a == 64) ? ~0ull : (((1ull << (b - a)) - 1) << a);
            const int c = __popcll(v & m);
            if (c) atomicAdd(&s_cnt[l], (unsigned long long)c);
        }
    }
    __syncthreads();
    for (int l = threadIdx.x; l < n_libs; l += blockDim.x)
        if (s_cnt[l]) atomicAdd(&counts[l], s_cnt[l]);
}

// Concatenated per-library offsets -> offsets into the concatenated bases (one thread per output entry).
__global__ void k_batch_offsets(const uint64_t *__restrict__ src, const uint64_t *__restrict__ entry_starts,
                                const uint64_t *__restrict__ lib_starts, int n_libs, uint64_t *__restrict__ dst,
                                uint64_t n_entries) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n_entries;
         j += (uint64_t)gridDim.x * blockDim.x) {
        if (j + 1 == n_entries) {  // the end of the last read
            dst[j] = lib_starts[n_libs];
            continue;
        }
        int lo = 0, hi = n_libs;  // library whose reads contain output entry j
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (entry_starts[mid] <= j) lo = mid;
            else hi = mid;
        }
        const uint64_t r = j - entry_starts[lo];
        const uint64_t *o = src + entry_starts[lo] + lo;  // library lo's own offsets
        dst[j] = o[r] - o[0] + lib_starts[lo];
    }
}

// Batched output sorted by library tag. First pass: the first index of each library's run
// (starts[] holds UINT64_MAX on entry). Second pass (a separate launch, so no thread reads a
// neighbour whose tag is already cleared): clear the tag bits in place.
template <class K>
__global__ void k_tag_starts(const K *keys, uint64_t n, int shift, uint64_t *starts) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t t = tag_of(keys[i], shift);
        if (i == 0 || tag_of(keys[i - 1], shift) != t) starts[t] = i;
    }
}

template <class K>
__global__ void k_clear_tags(K *keys, uint64_t n, int shift) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        if constexpr (sizeof(K) == 8) keys[i] &= (1ull << shift) - 1;
        else keys[i].hi &= (1ull << (shift - 64)) - 1;
    }
}

static int grid_for(uint64_t items, int block, int sms, int per_sm) {
    uint64_t need = (items + block - 1) / block;
    uint64_t cap = (uint64_t)sms * per_sm;
    if (need < 1) need = 1;
    return (int)(need < cap ? need : cap);
}

void launch_pack_groups(const LaunchCfg &c, const uint8_t *bases, const uint64_t *offsets, uint64_t n_reads,
                        const PackLayout &L, uint64_t g_begin, uint64_t g_end, uint64_t *P, uint64_t *B) {
    if (g_end <= g_begin) return;
    k_pack<<<grid_for(g_end - g_begin, 256, c.sms, 16), 256, 0, c.stream>>>(
        bases, L.n_bases, offsets, n_reads, g_begin, g_end, P, reinterpret_cast<uint32_t *>(B));
}

void launch_mark_starts(const LaunchCfg &c, const uint64_t *offsets, uint64_t n_reads, const PackLayout &L,
                        uint64_t *S, uint32_t *err) {
    k_mark_starts<<<grid_for(n_reads + 1, 256, c.sms, 8), 256, 0, c.stream>>>(offsets, n_reads, L.n_bases,
                                                                            reinterpret_cast<uint32_t *>(S), err);
}

void launch_pack(const LaunchCfg &c, const uint8_t *bases, const uint64_t *offsets, uint64_t n_reads,
                 const PackLayout &L, uint64_t *P, uint64_t *B, uint64_t *S, uint32_t *err) {
    // every B word, including the padding (all bad)
    launch_pack_groups(c, bases, offsets, n_reads, L, 0, L.pack_groups(), P, B);
    launch_mark_starts(c, offsets, n_reads, L, S, err);
}

void launch_valid(const LaunchCfg &c, const PackLayout &L, int k, const uint64_t *B, const uint64_t *S, uint64_t *V,
                  unsigned long long *n_windows, uint64_t w_begin, uint64_t w_end) {
    const uint64_t n_words = L.v_words - 2;
    if (w_end > n_words) w_end = n_words;
    if (w_begin >= w_end) return;
    k_valid<<<grid_for(w_end - w_begin, 256, c.sms, 8), 256, 0, c.stream>>>(B, S, w_begin, w_end, k, V, n_windows);
}

void launch_lib_windows(const LaunchCfg &c, const PackLayout &L, const uint64_t *V, const uint64_t *lib_starts,
                        int n_libs, unsigned long long *counts) {
    const uint64_t n_words = L.v_words - 2;
    k_lib_windows<<<grid_for(n_words, 256, c.sms, 8), 256, 0, c.stream>>>(V, n_words, lib_starts, n_libs, counts);
}

template <class K>
void launch_tag_starts(const LaunchCfg &c, const K *keys, uint64_t n, int shift, uint64_t *starts) {
    if (!n) return;
    k_tag_starts<K><<<grid_for(n, 256, c.sms, 8), 256, 0, c.stream>>>(keys, n, shift, starts);
}
template void launch_tag_starts<uint64_t>(const LaunchCfg &, const uint64_t *, uint64_t, int, uint64_t *);
template void launch_tag_starts<Key128>(const LaunchCfg &, const Key128 *, uint64_t, int, uint64_t *);

template <class K>
void launch_split_tags(const LaunchCfg &c, K *keys, uint64_t n, int shift, uint64_t *starts) {
    if (!n) return;
    k_tag_starts<K><<<grid_for(n, 256, c.sms, 8), 256, 0, c.stream>>>(keys, n, shift, starts);
    k_clear_tags<K><<<grid_for(n, 256, c.sms, 8), 256, 0, c.stream>>>(keys, n, shift);
}
template void launch_split_tags<uint64_t>(const LaunchCfg &, uint64_t *, uint64_t, int, uint64_t *);
template void launch_split_tags<Key128>(const LaunchCfg &, Key128 *, uint64_t, int, uint64_t *);

void launch_batch_offsets(const LaunchCfg &c, const uint64_t *src, const uint64_t *entry_starts,
                          const uint64_t *lib_starts, int n_libs, uint64_t *dst, uint64_t n_entries) {
    k_batch_offsets<<<grid_for(n_entries, 256, c.sms, 8), 256, 0, c.stream>>>(src, entry_starts, lib_starts, n_libs,
                                                                            dst, n_entries);
}

__global__ void k_narrow_keys(const Key128 *__restrict__ in, uint64_t n, uint64_t *__restrict__ out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = in[i].lo;
}

void launch_narrow_keys(const LaunchCfg &c, const Key128 *in, uint64_t n, uint64_t *out) {
    if (n) k_narrow_keys<<<grid_for(n, 256, c.sms, 8), 256, 0, c.stream>>>(in, n, out);
}

void launch_extract(const LaunchCfg &c, const PackLayout &L, int k, const uint64_t *P, const uint64_t *V,
                    uint64_t *keys) {
    if (k <= 32)
        k_extract<uint64_t><<<grid_for(L.n_bases, 256, c.sms, 8), 256, 0, c.stream>>>(P, V, L.n_bases, k, keys);
    else
        k_extract<Key128><<<grid_for(L.n_bases, 256, c.sms, 8), 256, 0, c.stream>>>(
            P, V, L.n_bases, k, reinterpret_cast<Key128 *>(keys));
}

}  // namespace turtle
