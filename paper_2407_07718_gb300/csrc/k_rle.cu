// k_rle.cu -- stage S5: the linear scan of Sec. 3.1 over sorted keys: run
// lengths (counts), the histogram of counts over all distinct k-mers, and the
// frequency-range filter lo <= count <= hi (Sec. 4 uses [2, 50]).
//
// Runs may cross tile boundaries (a repeat k-mer can occur thousands of
// times), so no thread ever scans forward to a run's end.  Two kernels:
//   k_rle_heads -- head flag (key differs from its predecessor) for every key;
//                  the heads' indices are compacted, in order, with a
//                  decoupled look-back across tiles;
//   k_rle_emit  -- count of run j = heads[j+1] - heads[j]; histogram bins in
//                  shared memory; kept (key, count) pairs compacted in order.
#include "hsk_device.cuh"

namespace hsk {

constexpr int RLE_ITEMS = 16;
constexpr int RLE_TILE = 256 * RLE_ITEMS;
constexpr int RLE_SBINS = 2048;  // histogram bins kept in shared memory

uint64_t rle_tiles(uint64_t n, int /*key_words*/) { return (n + RLE_TILE - 1) / RLE_TILE; }
uint64_t rle_status_words(uint64_t n) { return ((n + RLE_TILE - 1) / RLE_TILE + 1) * LB_PAD; }

// Order-preserving compaction of one tile: flags[i] for item (i, thread) in
// index order i * 256 + threadIdx.x.  Returns each thread's per-item output
// slots via `slot` (valid where flagged) relative to the tile, and the tile
// total.  Uses s_wc (RLE_ITEMS * 8 words) and s_scr.
__device__ __forceinline__ uint32_t tile_compact(const bool (&flag)[RLE_ITEMS], uint32_t (&slot)[RLE_ITEMS],
                                                 uint32_t* s_wc, uint32_t* s_scr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t ballots[RLE_ITEMS];
#pragma unroll
    for (int i = 0; i < RLE_ITEMS; ++i) {
        ballots[i] = __ballot_sync(0xffffffffu, flag[i]);
        if (lane == 0) s_wc[i * 8 + warp] = __popc(ballots[i]);
    }
    __syncthreads();
    // exclusive scan over (item, warp) in index order: RLE_ITEMS * 8 = 128 entries
    uint32_t v = threadIdx.x < RLE_ITEMS * 8 ? s_wc[threadIdx.x] : 0u;
    uint32_t total;
    uint32_t e = block_excl_sum<256, uint32_t>(v, s_scr, total);
    if (threadIdx.x < RLE_ITEMS * 8) s_wc[threadIdx.x] = e;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RLE_ITEMS; ++i) slot[i] = s_wc[i * 8 + warp] + __popc(ballots[i] & lt);
    return total;
}

template <typename K>
__global__ void __launch_bounds__(256) k_rle_heads(const K* __restrict__ keys, u64 n,
                                                   uint32_t* __restrict__ heads, u64* n_heads,
                                                   u64* status, uint32_t* tile_ctr, uint32_t epoch,
                                                   int* err) {
    __shared__ uint32_t s_wc[RLE_ITEMS * 8];
    __shared__ uint32_t s_scr[9];
    __shared__ u64 s_prefix;
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const u64 tile = s_tile;
    const u64 base = tile * RLE_TILE;
    const u64 n_tiles = (n + RLE_TILE - 1) / RLE_TILE;
    bool flag[RLE_ITEMS];
    uint32_t slot[RLE_ITEMS];
#pragma unroll
    for (int i = 0; i < RLE_ITEMS; ++i) {
        u64 idx = base + (u64)i * 256 + threadIdx.x;
        flag[i] = idx < n && (idx == 0 || !key_eq(keys[idx], keys[idx - 1]));
    }
    uint32_t total = tile_compact(flag, slot, s_wc, s_scr);
    if (threadIdx.x == 0) {
        u64 pre = 0;
        if (tile == 0) {
            st_relaxed(status, lb_word(LB_PREFIX, epoch, total));
        } else {
            st_relaxed(status + tile * LB_PAD, lb_word(LB_AGG, epoch, total));
            pre = lookback_exclusive_win<16>(status, LB_PAD, tile, epoch, err);
            st_relaxed(status + tile * LB_PAD, lb_word(LB_PREFIX, epoch, pre + total));
        }
        s_prefix = pre;
        if (tile == n_tiles - 1) {
            if (pre + total > n) {
                raise_error(err, HSK_DERR_BOUNDS);
            } else {
                *n_heads = pre + total;
                heads[pre + total] = (uint32_t)n;
            }
        }
    }
    __syncthreads();
    const u64 pre = s_prefix;
#pragma unroll
    for (int i = 0; i < RLE_ITEMS; ++i) {
        if (!flag[i]) continue;
        if (pre + slot[i] >= n) {  // only after a failed look-back
            raise_error(err, HSK_DERR_BOUNDS);
            continue;
        }
        heads[pre + slot[i]] = (uint32_t)(base + (u64)i * 256 + threadIdx.x);
    }
}

template <typename K>
__global__ void __launch_bounds__(256) k_rle_emit(const K* __restrict__ keys, const uint32_t* __restrict__ heads,
                                                  const u64* __restrict__ n_heads, uint32_t lo, uint32_t hi,
                                                  u64* __restrict__ hist, uint32_t hist_len,
                                                  uint32_t* max_count, K* __restrict__ out_keys,
                                                  uint32_t* __restrict__ out_counts, u64* n_out,
                                                  u64* status, uint32_t* tile_ctr, uint32_t epoch, int* err) {
    __shared__ uint32_t s_hist[RLE_SBINS];
    __shared__ uint32_t s_wc[RLE_ITEMS * 8];
    __shared__ uint32_t s_scr[9];
    __shared__ u64 s_prefix;
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_max;
    const u64 D = *n_heads;
    const u64 n_tiles = (D + RLE_TILE - 1) / RLE_TILE;
    if (threadIdx.x == 0) {
        s_tile = atomicAdd(tile_ctr, 1u);
        s_max = 0;
    }
    const uint32_t sb = hist_len < RLE_SBINS ? hist_len : RLE_SBINS;
    for (uint32_t b = threadIdx.x; b < sb; b += 256) s_hist[b] = 0;
    __syncthreads();
    const u64 tile = s_tile;
    if (tile >= n_tiles) return;  // uniform: the launch may be sized for more runs
    const u64 base = tile * RLE_TILE;
    bool flag[RLE_ITEMS];
    uint32_t slot[RLE_ITEMS], cnt[RLE_ITEMS];
    uint32_t mx = 0;
#pragma unroll
    for (int i = 0; i < RLE_ITEMS; ++i) {
        u64 j = base + (u64)i * 256 + threadIdx.x;
        cnt[i] = 0;
        flag[i] = false;
        if (j < D) {
            uint32_t c = heads[j + 1] - heads[j];
            cnt[i] = c;
            uint32_t bin = c >= hist_len - 1 ? hist_len - 1 : c;
            if (bin < sb) atomicAdd(&s_hist[bin], 1u);
            else atomicAdd(reinterpret_cast<unsigned long long*>(hist + bin), 1ULL);
            mx = c > mx ? c : mx;
            flag[i] = c >= lo && c <= hi;
        }
    }
    uint32_t total = tile_compact(flag, slot, s_wc, s_scr);
    if (threadIdx.x == 0) {
        u64 pre = 0;
        if (tile == 0) {
            st_relaxed(status, lb_word(LB_PREFIX, epoch, total));
        } else {
            st_relaxed(status + tile * LB_PAD, lb_word(LB_AGG, epoch, total));
            pre = lookback_exclusive_win<16>(status, LB_PAD, tile, epoch, err);
            st_relaxed(status + tile * LB_PAD, lb_word(LB_PREFIX, epoch, pre + total));
        }
        s_prefix = pre;
        if (tile == n_tiles - 1) *n_out = pre + total;
    }
    // warp max -> block max
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        uint32_t o = __shfl_xor_sync(0xffffffffu, mx, d);
        mx = o > mx ? o : mx;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&s_max, mx);
    __syncthreads();
    const u64 pre = s_prefix;
#pragma unroll
    for (int i = 0; i < RLE_ITEMS; ++i) {
        if (flag[i]) {
            u64 j = base + (u64)i * 256 + threadIdx.x;
            if (pre + slot[i] >= D) {  // only after a failed look-back
                raise_error(err, HSK_DERR_BOUNDS);
                continue;
            }
            out_keys[pre + slot[i]] = keys[heads[j]];
            out_counts[pre + slot[i]] = cnt[i];
        }
    }
    for (uint32_t b = threadIdx.x; b < sb; b += 256)
        if (s_hist[b]) atomicAdd(reinterpret_cast<unsigned long long*>(hist + b), (unsigned long long)s_hist[b]);
    if (threadIdx.x == 0 && s_max) atomicMax(max_count, s_max);
}

void launch_rle_heads(const void* keys, uint64_t n, int key_words, uint32_t* heads,
                      uint64_t* n_heads, uint64_t* status, uint32_t* tile_ctr, uint32_t epoch,
                      int* err, cudaStream_t st) {
    if (n == 0) {
        cudaMemsetAsync(n_heads, 0, sizeof(uint64_t), st);
        cudaMemsetAsync(heads, 0, sizeof(uint32_t), st);
        return;
    }
    unsigned tiles = (unsigned)((n + RLE_TILE - 1) / RLE_TILE);
    count_launch();
    if (key_words == 1)
        k_rle_heads<u64><<<tiles, 256, 0, st>>>((const u64*)keys, n, heads, (u64*)n_heads, (u64*)status,
                                                tile_ctr, epoch, err);
    else
        k_rle_heads<key128><<<tiles, 256, 0, st>>>((const key128*)keys, n, heads, (u64*)n_heads,
                                                   (u64*)status, tile_ctr, epoch, err);
}

void launch_rle_emit(const void* keys, const uint32_t* heads, const uint64_t* n_heads,
                     uint64_t n_heads_host, int key_words, uint32_t lo, uint32_t hi,
                     uint64_t* hist, uint32_t hist_len, uint32_t* max_count, void* out_keys,
                     uint32_t* out_counts, uint64_t* n_out, uint64_t* status, uint32_t* tile_ctr,
                     uint32_t epoch, int* err, cudaStream_t st) {
    if (n_heads_host == 0) {
        cudaMemsetAsync(n_out, 0, sizeof(uint64_t), st);
        return;
    }
    unsigned tiles = (unsigned)((n_heads_host + RLE_TILE - 1) / RLE_TILE);
    count_launch();
    if (key_words == 1)
        k_rle_emit<u64><<<tiles, 256, 0, st>>>((const u64*)keys, heads, (const u64*)n_heads, lo, hi,
                                               (u64*)hist, hist_len, max_count, (u64*)out_keys, out_counts,
                                               (u64*)n_out, (u64*)status, tile_ctr, epoch, err);
    else
        k_rle_emit<key128><<<tiles, 256, 0, st>>>((const key128*)keys, heads, (const u64*)n_heads, lo, hi,
                                                  (u64*)hist, hist_len, max_count, (key128*)out_keys,
                                                  out_counts, (u64*)n_out, (u64*)status, tile_ctr, epoch, err);
}

}  // namespace hsk
