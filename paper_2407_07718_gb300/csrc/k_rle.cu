// k_rle.cu -- stage S5: the linear scan of Sec. 3.1 over sorted keys: run
// lengths (counts), the histogram of counts over all distinct k-mers, and the
// frequency-range filter lo <= count <= hi (Sec. 4 uses [2, 50]).
//
// Runs may cross tiles (a repeat k-mer can occur thousands of times), so no
// thread scans forward to a run's end, and no tile waits on another:
//   k_rle_mark   -- reads every key once: run-head bitmask (one ballot per 32
//                   keys), and per tile its first and last head, the number
//                   of heads, the runs that end inside the tile (histogram,
//                   max, kept count);
//   k_rle_next_* -- for each tile the first head after it (a suffix minimum
//                   over tiles), which closes the tile's last run;
//   k_rle_write  -- reads the bitmask, gathers the keys of kept runs and
//                   writes (key, count) pairs at scanned offsets.
// Tiles are 4096 keys; thread t of a tile owns keys 16t .. 16t+15.
#include "hsk_device.cuh"

namespace hsk {

constexpr int RLE_ITEMS = 16;
constexpr int RLE_TILE = 256 * RLE_ITEMS;   // 4096 keys, 128 bitmask words
constexpr int RLE_SBINS = 2048;             // histogram bins kept in shared memory
constexpr uint32_t NO_HEAD = 0xFFFFFFFFu;

uint64_t rle_tiles(uint64_t n, int /*key_words*/) { return (n + RLE_TILE - 1) / RLE_TILE; }
uint64_t rle_bits_words(uint64_t n) { return (n + 31) / 32 + 1; }

// Heads among this thread's 16 keys: bit b is key 16*threadIdx.x + b.
__device__ __forceinline__ uint32_t rle_thread_bits(const uint32_t* s_bits) {
    const int t = threadIdx.x;
    return (s_bits[t >> 1] >> (16 * (t & 1))) & 0xFFFFu;
}

// Exclusive suffix minimum over the threads after this one (256 threads).
__device__ __forceinline__ uint32_t block_excl_suffix_min(uint32_t v, uint32_t* s_w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t o = __shfl_down_sync(0xffffffffu, inc, d);
        if (lane + d < 32) inc = min(inc, o);
    }
    if (lane == 0) s_w[warp] = inc;  // minimum of the whole warp
    __syncthreads();
    uint32_t after_warp = NO_HEAD;
    for (int w = warp + 1; w < 8; ++w) after_warp = min(after_warp, s_w[w]);
    uint32_t nxt = __shfl_down_sync(0xffffffffu, inc, 1);
    if (lane == 31) nxt = NO_HEAD;
    __syncthreads();
    return min(nxt, after_warp);
}

// Visit the runs whose head lies in this thread's keys, in order: f(head
// position in the tile, count).  The next head of the thread's last head is
// next_local (in the tile) or, when the tile has no later head, the position
// after_tile (tile-relative) if known; otherwise that run is skipped (it is
// the tile's last run, closed by k_rle_close).
template <typename F>
__device__ __forceinline__ void rle_visit(uint32_t bits16, uint32_t next_local, u64 after_tile, bool known,
                                          F&& f) {
    const uint32_t t0 = 16 * threadIdx.x;
    while (bits16) {
        const int b = __ffs(bits16) - 1;
        bits16 &= bits16 - 1;
        const uint32_t pos = t0 + b;
        u64 nxt;
        if (bits16) nxt = t0 + __ffs(bits16) - 1;
        else if (next_local != NO_HEAD) nxt = next_local;
        else if (known) nxt = after_tile;
        else break;
        f(pos, (uint32_t)(nxt - pos));
    }
}

template <typename K>
__device__ __forceinline__ K shfl_up1(K v);
template <>
__device__ __forceinline__ u64 shfl_up1<u64>(u64 v) { return __shfl_up_sync(0xffffffffu, v, 1); }
template <>
__device__ __forceinline__ key128 shfl_up1<key128>(key128 v) {
    return key128{__shfl_up_sync(0xffffffffu, v.lo, 1), __shfl_up_sync(0xffffffffu, v.hi, 1)};
}

template <typename K>
__global__ void __launch_bounds__(256) k_rle_mark(const K* __restrict__ keys, u64 n, uint32_t* __restrict__ bits,
                                                  u64* __restrict__ tile_first, u64* __restrict__ tile_last,
                                                  uint32_t* __restrict__ tile_keep, uint32_t lo, uint32_t hi,
                                                  u64* __restrict__ hist, uint32_t hist_len, uint32_t* max_count,
                                                  u64* n_heads) {
    __shared__ uint32_t s_bits[RLE_TILE / 32];
    __shared__ uint32_t s_hist[RLE_SBINS];
    __shared__ uint32_t s_w[8];
    __shared__ uint32_t s_keep[8];
    __shared__ uint32_t s_fl[2];
    __shared__ K s_edge[1 + RLE_ITEMS * 8];  // key before each run of 32 keys
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t sb = hist_len < RLE_SBINS ? hist_len : RLE_SBINS;
    for (uint32_t b = threadIdx.x; b < sb; b += 256) s_hist[b] = 0;
    uint32_t mx = 0;
    u64 heads = 0;
    const u64 n_tiles = (n + RLE_TILE - 1) / RLE_TILE;
    const u64 n_words = (n + 31) / 32;
    for (u64 t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const u64 base = t * RLE_TILE;
        if (threadIdx.x == 0) {
            s_fl[0] = NO_HEAD;
            s_fl[1] = 0;
        }
        // ---- head flags, one ballot per 32 consecutive keys; all loads first.
        // The left neighbour of a warp's lane 0 is the last key of the previous
        // 32, passed through shared memory (the tile's first key reads the key
        // before the tile).
        K cur[RLE_ITEMS];
#pragma unroll
        for (int i = 0; i < RLE_ITEMS; ++i) {
            const u64 idx = base + (u64)i * 256 + warp * 32 + lane;
            cur[i] = idx < n ? keys[idx] : K{};
        }
        if (threadIdx.x == 0) s_edge[0] = base > 0 ? keys[base - 1] : K{};
        if (lane == 31) {
#pragma unroll
            for (int i = 0; i < RLE_ITEMS; ++i) s_edge[1 + i * 8 + warp] = cur[i];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < RLE_ITEMS; ++i) {
            const u64 idx = base + (u64)i * 256 + warp * 32 + lane;
            const bool in = idx < n;
            K prv = shfl_up1(cur[i]);
            if (lane == 0) prv = s_edge[i * 8 + warp];  // key idx - 1
            const bool head = in && (idx == 0 || !key_eq(cur[i], prv));
            const uint32_t word = __ballot_sync(0xffffffffu, head);
            if (lane == 0) {
                s_bits[i * 8 + warp] = word;
                const u64 wi = base / 32 + i * 8 + warp;
                if (wi < n_words) bits[wi] = word;
            }
        }
        __syncthreads();
        // ---- runs that close inside the tile
        const uint32_t b16 = rle_thread_bits(s_bits);
        const uint32_t first_here = b16 ? 16 * threadIdx.x + __ffs(b16) - 1 : NO_HEAD;
        const uint32_t next_local = block_excl_suffix_min(first_here, s_w);
        heads += __popc(b16);
        if (b16) {
            atomicMin(&s_fl[0], first_here);
            atomicMax(&s_fl[1], 16 * threadIdx.x + (31 - __clz(b16)) + 1);  // last head + 1
        }
        uint32_t keep = 0;
        rle_visit(b16, next_local, 0, false, [&](uint32_t, uint32_t c) {
            const uint32_t bin = c >= hist_len - 1 ? hist_len - 1 : c;
            if (bin < sb) atomicAdd(&s_hist[bin], 1u);
            else atomicAdd(reinterpret_cast<unsigned long long*>(hist + bin), 1ULL);
            mx = c > mx ? c : mx;
            keep += (c >= lo && c <= hi);
        });
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, d);
        if (lane == 0) s_keep[warp] = keep;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tk = 0;
            for (int w = 0; w < 8; ++w) tk += s_keep[w];
            tile_keep[t] = tk;
            tile_first[t] = s_fl[0] == NO_HEAD ? ~0ULL : base + s_fl[0];
            tile_last[t] = s_fl[1] == 0 ? ~0ULL : base + s_fl[1] - 1;
        }
        __syncthreads();
    }
    // ---- flush this CTA's histogram, max and head count
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, d));
        heads += __shfl_xor_sync(0xffffffffu, heads, d);
    }
    if (lane == 0) {
        if (mx) atomicMax(max_count, mx);
        if (heads) atomicAdd(reinterpret_cast<unsigned long long*>(n_heads), (unsigned long long)heads);
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < sb; b += 256)
        if (s_hist[b]) atomicAdd(reinterpret_cast<unsigned long long*>(hist + b), (unsigned long long)s_hist[b]);
}

// next[t] = first head after tile t within its block of 1024 tiles (or ~0);
// block_min[blk] = first head of the block (or ~0).
__global__ void __launch_bounds__(1024) k_rle_next_local(const u64* __restrict__ tile_first, u64 n_tiles,
                                                         u64* __restrict__ next, u64* __restrict__ block_min) {
    __shared__ u64 s_w[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const u64 t = (u64)blockIdx.x * 1024 + threadIdx.x;
    u64 inc = t < n_tiles ? tile_first[t] : ~0ULL;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        u64 o = __shfl_down_sync(0xffffffffu, inc, d);
        if (lane + d < 32) inc = inc < o ? inc : o;
    }
    if (lane == 0) s_w[warp] = inc;
    __syncthreads();
    u64 after = ~0ULL;
    for (int w = warp + 1; w < 32; ++w) after = after < s_w[w] ? after : s_w[w];
    u64 nx = __shfl_down_sync(0xffffffffu, inc, 1);
    if (lane == 31) nx = ~0ULL;
    nx = nx < after ? nx : after;
    if (t < n_tiles) next[t] = nx;
    if (threadIdx.x == 0) {
        u64 m = ~0ULL;
        for (int w = 0; w < 32; ++w) m = m < s_w[w] ? m : s_w[w];
        block_min[blockIdx.x] = m;
    }
}

// In place: block_min[b] becomes the first head after block b (~0 if none).
// One CTA walking 1024 blocks at a time from the end.
__global__ void __launch_bounds__(1024) k_rle_next_blocks(u64* block_min, u64 n_blocks) {
    __shared__ u64 s_w[32];
    __shared__ u64 s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = ~0ULL;
    __syncthreads();
    for (long long c0 = (long long)((n_blocks + 1023) / 1024 - 1) * 1024; c0 >= 0; c0 -= 1024) {
        const u64 b = (u64)c0 + threadIdx.x;
        u64 inc = b < n_blocks ? block_min[b] : ~0ULL;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            u64 o = __shfl_down_sync(0xffffffffu, inc, d);
            if (lane + d < 32) inc = inc < o ? inc : o;
        }
        if (lane == 0) s_w[warp] = inc;
        __syncthreads();
        u64 after = s_carry;
        for (int w = warp + 1; w < 32; ++w) after = after < s_w[w] ? after : s_w[w];
        u64 nx = __shfl_down_sync(0xffffffffu, inc, 1);
        if (lane == 31) nx = ~0ULL;
        nx = nx < after ? nx : after;
        __syncthreads();
        if (b < n_blocks) block_min[b] = nx;
        if (threadIdx.x == 0) {
            u64 m = s_carry;
            for (int w = 0; w < 32; ++w) m = m < s_w[w] ? m : s_w[w];
            s_carry = m;
        }
        __syncthreads();
    }
}

// Close every tile's last run: count = (first head after the tile, or n) - last head.
__global__ void __launch_bounds__(256) k_rle_close(const u64* __restrict__ tile_last, u64* __restrict__ next,
                                                   const u64* __restrict__ block_next, u64 n_tiles, u64 n,
                                                   uint32_t* __restrict__ tile_keep, uint32_t lo, uint32_t hi,
                                                   u64* __restrict__ hist, uint32_t hist_len, uint32_t* max_count) {
    const u64 t = (u64)blockIdx.x * 256 + threadIdx.x;
    uint32_t mx = 0;
    if (t < n_tiles) {
        u64 nx = next[t], bn = block_next[t / 1024];
        nx = nx < bn ? nx : bn;
        if (nx == ~0ULL) nx = n;
        next[t] = nx;
        const u64 last = tile_last[t];
        if (last != ~0ULL) {
            const uint32_t c = (uint32_t)(nx - last);  // a chunk holds < 2^32 keys
            const uint32_t bin = c >= hist_len - 1 ? hist_len - 1 : c;
            atomicAdd(reinterpret_cast<unsigned long long*>(hist + bin), 1ULL);
            mx = c;
            if (c >= lo && c <= hi) tile_keep[t] += 1;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, d));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(max_count, mx);
}

template <typename K>
__global__ void __launch_bounds__(256) k_rle_write(const K* __restrict__ keys, u64 n, const uint32_t* __restrict__ bits,
                                                   const u64* __restrict__ next, const u64* __restrict__ out_off,
                                                   uint32_t lo, uint32_t hi, K* __restrict__ out_keys,
                                                   uint32_t* __restrict__ out_counts, u64 out_cap, int* err) {
    __shared__ uint32_t s_bits[RLE_TILE / 32];
    __shared__ uint32_t s_w[8];
    __shared__ uint32_t s_scr[9];
    const u64 n_tiles = (n + RLE_TILE - 1) / RLE_TILE;
    const u64 n_words = (n + 31) / 32;
    for (u64 t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const u64 base = t * RLE_TILE;
        if (threadIdx.x < RLE_TILE / 32) {
            const u64 wi = base / 32 + threadIdx.x;
            s_bits[threadIdx.x] = wi < n_words ? bits[wi] : 0u;
        }
        __syncthreads();
        const uint32_t b16 = rle_thread_bits(s_bits);
        const uint32_t first_here = b16 ? 16 * threadIdx.x + __ffs(b16) - 1 : NO_HEAD;
        const uint32_t next_local = block_excl_suffix_min(first_here, s_w);
        const u64 after = next[t] - base;
        uint32_t my_keep = 0;
        rle_visit(b16, next_local, after, true, [&](uint32_t, uint32_t c) { my_keep += (c >= lo && c <= hi); });
        uint32_t tot;
        const uint32_t slot = block_excl_sum<256, uint32_t>(my_keep, s_scr, tot);
        u64 o = out_off[t] + slot;
        rle_visit(b16, next_local, after, true, [&](uint32_t pos, uint32_t c) {
            if (c >= lo && c <= hi) {
                if (o < out_cap) {
                    out_keys[o] = keys[base + pos];
                    out_counts[o] = c;
                } else {
                    raise_error(err, HSK_DERR_BOUNDS);
                }
                ++o;
            }
        });
        __syncthreads();
    }
}

void launch_rle_mark(const void* keys, uint64_t n, int key_words, uint32_t* bits, uint64_t* tile_first,
                     uint64_t* tile_last, uint32_t* tile_keep, uint32_t lo, uint32_t hi, uint64_t* hist,
                     uint32_t hist_len, uint32_t* max_count, uint64_t* n_heads, int grid, cudaStream_t st) {
    if (n == 0) return;
    count_launch();
    uint64_t tiles = rle_tiles(n, key_words);
    unsigned g = (unsigned)(tiles < (uint64_t)grid ? tiles : (uint64_t)grid);
    if (key_words == 1)
        k_rle_mark<u64><<<g, 256, 0, st>>>((const u64*)keys, n, bits, (u64*)tile_first, (u64*)tile_last, tile_keep,
                                           lo, hi, (u64*)hist, hist_len, max_count, (u64*)n_heads);
    else
        k_rle_mark<key128><<<g, 256, 0, st>>>((const key128*)keys, n, bits, (u64*)tile_first, (u64*)tile_last,
                                              tile_keep, lo, hi, (u64*)hist, hist_len, max_count, (u64*)n_heads);
}

void launch_rle_close(const uint64_t* tile_first, const uint64_t* tile_last, uint64_t* next, uint64_t* block_min,
                      uint64_t n_tiles, uint64_t n, uint32_t* tile_keep, uint32_t lo, uint32_t hi, uint64_t* hist,
                      uint32_t hist_len, uint32_t* max_count, cudaStream_t st) {
    if (n_tiles == 0) return;
    const uint64_t n_blocks = (n_tiles + 1023) / 1024;
    count_launch(3);
    k_rle_next_local<<<(unsigned)n_blocks, 1024, 0, st>>>((const u64*)tile_first, n_tiles, (u64*)next,
                                                         (u64*)block_min);
    k_rle_next_blocks<<<1, 1024, 0, st>>>((u64*)block_min, n_blocks);
    k_rle_close<<<(unsigned)((n_tiles + 255) / 256), 256, 0, st>>>((const u64*)tile_last, (u64*)next,
                                                                   (const u64*)block_min, n_tiles, n, tile_keep, lo,
                                                                   hi, (u64*)hist, hist_len, max_count);
}

void launch_rle_write(const void* keys, uint64_t n, int key_words, const uint32_t* bits, const uint64_t* next,
                      const uint64_t* out_off, uint32_t lo, uint32_t hi, void* out_keys, uint32_t* out_counts,
                      uint64_t out_cap, int* err, int grid, cudaStream_t st) {
    if (n == 0) return;
    count_launch();
    uint64_t tiles = rle_tiles(n, key_words);
    unsigned g = (unsigned)(tiles < (uint64_t)grid ? tiles : (uint64_t)grid);
    if (key_words == 1)
        k_rle_write<u64><<<g, 256, 0, st>>>((const u64*)keys, n, bits, (const u64*)next, (const u64*)out_off, lo,
                                            hi, (u64*)out_keys, out_counts, out_cap, err);
    else
        k_rle_write<key128><<<g, 256, 0, st>>>((const key128*)keys, n, bits, (const u64*)next, (const u64*)out_off,
                                               lo, hi, (key128*)out_keys, out_counts, out_cap, err);
}

}  // namespace hsk
