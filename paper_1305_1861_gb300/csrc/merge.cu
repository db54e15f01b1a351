// Lazy sort-and-compact phases (Sec. 2.1.4, Alg. 1): the running array of counted k-mers is
// kept sorted and compacted; a new batch of k-mers is sorted and compacted on its own and then
// merged with it in one linear pass, instead of sorting everything again.
//
// Here both inputs are ascending runs of distinct keys with uint32 counts (the running set and
// one chunk's compacted candidates). The merge follows the merge-path partition (Green, McColl &
// Bader, "GPU merge path", 2012): the merged sequence is cut into tiles of equal length, the
// split of every tile boundary between the two inputs is found by a binary search along its
// cross diagonal, and each CTA merges its tile in shared memory. On equal keys the element of A
// comes first; since each input holds a key at most once, a key present in both inputs forms an
// adjacent pair, which is compacted into its first element with the two counts added. Output
// positions come from a scan of the kept elements across tiles (decoupled look-back).
#include "common.cuh"
#include "kernels.h"

namespace turtle {

constexpr int M_BLOCK = 256;
constexpr int M_ITEMS = 8;
constexpr int M_TILE = M_BLOCK * M_ITEMS;

template <class K>
__device__ __forceinline__ bool key_le(const K &a, const K &b) {
    return !KeyT<K>::lt(b, a);
}

// Number of A elements among the first d elements of the merged order (A first on ties).
template <class K>
__device__ __forceinline__ uint64_t merge_split(const K *A, uint64_t na, const K *B, uint64_t nb, uint64_t d) {
    uint64_t lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (key_le(A[mid], B[d - mid - 1])) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// split[t] for t = 0 .. n_tiles: A's share of the first min(t * M_TILE, na + nb) merged elements.
template <class K>
__global__ void k_merge_splits(const K *__restrict__ A, uint64_t na, const K *__restrict__ B, uint64_t nb,
                               uint64_t n_tiles, uint64_t *split) {
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (t > n_tiles) return;
    const uint64_t d = t * (uint64_t)M_TILE < na + nb ? t * (uint64_t)M_TILE : na + nb;
    split[t] = merge_split(A, na, B, nb, d);
}

template <class K>
__global__ void __launch_bounds__(M_BLOCK) k_merge_counts(const K *__restrict__ A, const uint32_t *__restrict__ ca,
                                                          uint64_t na, const K *__restrict__ B,
                                                          const uint32_t *__restrict__ cb, uint64_t nb,
                                                          const uint64_t *__restrict__ split, K *__restrict__ out,
                                                          uint32_t *__restrict__ cout, unsigned long long *n_out,
                                                          uint64_t *lookback, uint32_t *tile_ctr, uint64_t n_tiles,
                                                          uint32_t spin_limit, uint32_t *err) {
    __shared__ K s_key[M_TILE];          // the tile's A part, then its B part; later the merged tile
    __shared__ uint32_t s_cnt[M_TILE];
    __shared__ uint32_t s_scan[M_BLOCK / WARP];
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_excl;
    __shared__ K s_pred, s_succ;
    __shared__ uint32_t s_succ_cnt;
    __shared__ int s_has_pred, s_has_succ;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);  // tiles in ticket order: look-back never waits on a later one
    __syncthreads();
    if (s_tile >= n_tiles) return;  // a ticket past the last tile (only when the counter did not start at 0)
    const uint64_t tile = s_tile, n = na + nb;
    const uint64_t d0 = tile * (uint64_t)M_TILE, d1 = d0 + M_TILE < n ? d0 + M_TILE : n;
    const uint64_t i0 = split[tile], i1 = split[tile + 1];
    const uint64_t j0 = d0 - i0, j1 = d1 - i1;
    const int la = (int)(i1 - i0), lb = (int)(j1 - j0), len = la + lb;
    for (int x = tid; x < la; x += M_BLOCK) {
        s_key[x] = A[i0 + x];
        s_cnt[x] = ca[i0 + x];
    }
    for (int x = tid; x < lb; x += M_BLOCK) {
        s_key[la + x] = B[j0 + x];
        s_cnt[la + x] = cb[j0 + x];
    }
    if (tid == 0) {
        // merged element d0 - 1: the later (in merged order) of A[i0 - 1] and B[j0 - 1]
        s_has_pred = d0 > 0;
        if (d0 > 0) {
            if (i0 == 0) s_pred = B[j0 - 1];
            else if (j0 == 0) s_pred = A[i0 - 1];
            else s_pred = key_le(A[i0 - 1], B[j0 - 1]) ? B[j0 - 1] : A[i0 - 1];
        }
        // merged element d1: the earlier of A[i1] and B[j1]
        s_has_succ = d1 < n;
        if (d1 < n) {
            const bool take_a = i1 < na && (j1 >= nb || key_le(A[i1], B[j1]));
            s_succ = take_a ? A[i1] : B[j1];
            s_succ_cnt = take_a ? ca[i1] : cb[j1];
        }
    }
    __syncthreads();
    // each thread merges positions [M_ITEMS * tid, M_ITEMS * tid + M_ITEMS) of the tile
    K key[M_ITEMS];
    uint32_t cnt[M_ITEMS];
    const int dl = M_ITEMS * tid < len ? M_ITEMS * tid : len;
    int lo = dl > lb ? dl - lb : 0, hi = dl < la ? dl : la;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (key_le(s_key[mid], s_key[la + dl - mid - 1])) lo = mid + 1;
        else hi = mid;
    }
    int ia = lo, ib = dl - lo;
    const int mine = len - dl < M_ITEMS ? len - dl : M_ITEMS;
#pragma unroll
    for (int p = 0; p < M_ITEMS; p++) {
        if (p < mine) {
            const bool take_a = ia < la && (ib >= lb || key_le(s_key[ia], s_key[la + ib]));
            const int src = take_a ? ia++ : la + ib++;
            key[p] = s_key[src];
            cnt[p] = s_cnt[src];
        }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < M_ITEMS; p++)
        if (p < mine) {
            s_key[dl + p] = key[p];
            s_cnt[dl + p] = cnt[p];
        }
    __syncthreads();
    // compact: keep the first element of each run of equal keys, with the next element's count
    // added when it holds the same key (the pair's B copy)
    uint32_t keep = 0, nkeep = 0;
#pragma unroll
    for (int p = 0; p < M_ITEMS; p++) {
        if (p >= mine) continue;
        const int x = dl + p;
        const bool dup = x > 0 ? KeyT<K>::eq(s_key[x - 1], key[p]) : (s_has_pred && KeyT<K>::eq(s_pred, key[p]));
        if (dup) continue;
        uint64_t c = cnt[p];
        if (x + 1 < len) {
            if (KeyT<K>::eq(s_key[x + 1], key[p])) c += s_cnt[x + 1];
        } else if (s_has_succ && KeyT<K>::eq(s_succ, key[p])) {
            c += s_succ_cnt;
        }
        if (c > 0xfffffffeull) {
            atomicOr(err, ERR_COUNT_OVERFLOW);
            c = 0xfffffffeull;
        }
        cnt[p] = (uint32_t)c;
        keep |= 1u << p;
        nkeep++;
    }
    uint32_t total;
    const uint32_t before = block_exclusive_scan<M_BLOCK>(nkeep, s_scan, &total);
    if (tid < WARP) {
        const uint64_t e = lookback_prefix_warp(lookback, tile, total, 1, err, spin_limit);
        if (tid == 0) s_excl = e;
    }
    __syncthreads();
    uint64_t o = s_excl + before;
#pragma unroll
    for (int p = 0; p < M_ITEMS; p++)
        if ((keep >> p) & 1u) {
            store_key(out + o, key[p]);
            cout[o] = cnt[p];
            o++;
        }
    if (d1 == n && tid == 0) *n_out = s_excl + total;
}

template <class K>
void launch_merge_counts(const LaunchCfg &c, const K *A, const uint32_t *ca, uint64_t na, const K *B,
                         const uint32_t *cb, uint64_t nb, K *out, uint32_t *cout, unsigned long long *n_out,
                         uint64_t *split, uint64_t *lookback, uint32_t *tile_ctr, uint32_t *err, bool skip_tile0,
                         uint32_t spin_limit) {
    cudaMemsetAsync(n_out, 0, sizeof(unsigned long long), c.stream);
    const uint64_t n = na + nb;
    if (n == 0) return;
    const uint64_t tiles = (n + M_TILE - 1) / M_TILE;
    k_merge_splits<K><<<(int)((tiles + 1 + 255) / 256), 256, 0, c.stream>>>(A, na, B, nb, tiles, split);
    cudaMemsetAsync(tile_ctr, 0, sizeof(uint32_t), c.stream);
    // failure injection: tickets start at 1, so tile 0 never runs and its successors' look-back waits
    // run out (the ticket past the last tile returns at once)
    if (skip_tile0) cudaMemsetAsync(tile_ctr, 1, 1, c.stream);
    cudaMemsetAsync(lookback, 0, sizeof(uint64_t) * tiles, c.stream);
    k_merge_counts<K><<<(int)tiles, M_BLOCK, 0, c.stream>>>(A, ca, na, B, cb, nb, split, out, cout, n_out, lookback,
                                                             tile_ctr, tiles, spin_limit ? spin_limit : LB_SPIN_LIMIT,
                                                             err);
}

uint64_t merge_tiles(uint64_t n) { return (n + M_TILE - 1) / M_TILE; }

template void launch_merge_counts<uint64_t>(const LaunchCfg &, const uint64_t *, const uint32_t *, uint64_t,
                                            const uint64_t *, const uint32_t *, uint64_t, uint64_t *, uint32_t *,
                                            unsigned long long *, uint64_t *, uint64_t *, uint32_t *, uint32_t *, bool,
                                            uint32_t);
template void launch_merge_counts<Key128>(const LaunchCfg &, const Key128 *, const uint32_t *, uint64_t,
                                          const Key128 *, const uint32_t *, uint64_t, Key128 *, uint32_t *,
                                          unsigned long long *, uint64_t *, uint64_t *, uint32_t *, uint32_t *, bool,
                                          uint32_t);

}  // namespace turtle
