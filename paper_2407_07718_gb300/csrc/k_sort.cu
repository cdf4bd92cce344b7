// k_sort.cu -- stage S4: LSD radix sort of packed k-mer keys (Sec. 3.1: sort
// the k-mers so equal values become adjacent, then count them with one linear
// scan).  The paper sorts each task on the CPU with RADULS (out of place) or
// PARADIS (in place); on the GPU the sort is a onesweep-style LSD radix sort
// (Adinets & Merrill, 2022): one up-front pass builds the digit histograms of
// every pass, then each pass ranks a tile of keys in shared memory, obtains
// the tile's global digit offsets by decoupled look-back over earlier tiles
// and scatters the tile, digit by digit, with contiguous writes.
//
// This is the global path: it sorts the sub-segments that do not fit the
// on-chip sort (k_local.cu), the whole job when local_sort is off, the keys
// of hsk_stage_sort / hsk_sort_keys_noalloc, and the output pairs (S6).
//
// Segments.  The keys of a job are split into C segments, each a group of
// minimizer buckets -- the paper's tasks (Sec. 3.4), which never share a
// k-mer value -- and every segment is sorted on its own, as the paper's
// workers sort their tasks.  All segments go through one launch per pass
// with their tiles interleaved (global tile g is tile g / C of segment
// g % C), so each segment's look-back chain holds only ~1/C of the tiles in
// flight and a tile seldom waits for a predecessor that is itself still
// looking back.  A plain sort is the case C = 1.
//
//   k_expand_seg  -- supermer records -> canonical keys of each segment, plus
//                    the segment's up-front digit histograms (fused).
//   k_digit_hist  -- up-front histograms of plain keys (stage sort, S6).
//   k_digit_offsets_seg -- per (pass, segment) exclusive digit offsets.
//   k_onesweep_seg -- one 8-bit LSD pass over all segments; u64 keys
//                    (k <= 32) or 128-bit keys (k <= 64), optional uint32 value.
#include "hsk_device.cuh"

namespace hsk {

constexpr int RADIX = 256;
constexpr int MAX_PASS = 16;

// ---------------------------------------------------------------------------
// supermer records -> keys (+ digit histograms), per segment
// ---------------------------------------------------------------------------

uint64_t expand_tiles(uint64_t n_rec) { return (n_rec + EXP_TILE - 1) / EXP_TILE; }
int expand_grid(int num_sms) { return num_sms * 4; }

// Each CTA starts on segment blockIdx.x % C and takes that segment's record
// tiles from its counter; when they run out it flushes the segment's
// histogram and moves on to the next segment, so CTAs finish together.
// Segment c: records [rec_base[c], rec_base[c+1]), keys written from
// key_base[c]; look-back status of its tiles at status + c * st_stride.
// A tile's records are staged in shared memory with their k-mer counts'
// prefix; thread j of the CTA then takes keys j, j+256, ... of the tile and
// finds each key's record by binary search, so all threads expand the same
// number of keys and the key writes are contiguous.
template <bool WIDE>
__global__ void __launch_bounds__(256) k_expand_seg(const u64* __restrict__ rec, const u64* __restrict__ rec_base,
                                                    const u64* __restrict__ key_base, uint32_t C, int k,
                                                    void* __restrict__ keys_out, u64* status, u64 st_stride,
                                                    uint32_t* tile_ctr, uint32_t epoch, u64* __restrict__ hist,
                                                    int n_pass, int* err) {
    constexpr int RW = WIDE ? 4 : 2;
    __shared__ uint32_t s_hist[MAX_PASS * RADIX];
    extern __shared__ __align__(16) u64 s_rec[];  // EXP_TILE * RW words (dynamic)
    __shared__ uint32_t s_pre[EXP_TILE + 1];
    __shared__ u64 s_scr[9];
    __shared__ u64 s_prefix;
    __shared__ uint32_t s_tile;
    for (int i = threadIdx.x; i < n_pass * RADIX; i += 256) s_hist[i] = 0;
    uint32_t c = blockIdx.x % C, visited = 0;
    bool dirty = false;
    while (visited < C) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr + c, 1u);
        __syncthreads();
        const u64 tile = s_tile;
        const u64 rb = rec_base[c], n_rec = rec_base[c + 1] - rb;
        const u64 n_tiles = (n_rec + EXP_TILE - 1) / EXP_TILE;
        if (tile >= n_tiles) {  // segment done: flush its histogram, move on
            if (dirty) {
                u64* h = hist + (u64)c * n_pass * RADIX;
                for (int i = threadIdx.x; i < n_pass * RADIX; i += 256) {
                    uint32_t v = s_hist[i];
                    if (v) atomicAdd(reinterpret_cast<unsigned long long*>(h + i), (unsigned long long)v);
                    s_hist[i] = 0;
                }
                dirty = false;
            }
            c = c + 1 == C ? 0 : c + 1;
            ++visited;
            continue;
        }
        dirty = true;
        u64* seg_status = status + (u64)c * st_stride;
        const u64 r0 = tile * EXP_TILE;
        const uint32_t nr = (uint32_t)(n_rec - r0 < (u64)EXP_TILE ? n_rec - r0 : (u64)EXP_TILE);
        // ---- stage the tile's records (contiguous, 128-bit loads)
        const ulonglong2* src = reinterpret_cast<const ulonglong2*>(rec + (rb + r0) * RW);
        ulonglong2* dst = reinterpret_cast<ulonglong2*>(s_rec);
        for (uint32_t i = threadIdx.x; i < nr * (RW / 2); i += 256) dst[i] = src[i];
        __syncthreads();
        // ---- k-mer counts of records 4t .. 4t+3, block scan
        uint32_t nk[EXP_RPT], sum = 0;
#pragma unroll
        for (int i = 0; i < EXP_RPT; ++i) {
            const uint32_t r = threadIdx.x * EXP_RPT + i;
            nk[i] = r < nr ? (uint32_t)(s_rec[r * RW + RW - 1] & 0xFF) : 0u;
            sum += nk[i];
        }
        u64 total;
        u64 excl = block_excl_sum<256, u64>((u64)sum, s_scr, total);
        {
            uint32_t run = (uint32_t)excl;
#pragma unroll
            for (int i = 0; i < EXP_RPT; ++i) {
                s_pre[threadIdx.x * EXP_RPT + i] = run;
                run += nk[i];
            }
            if (threadIdx.x == 255) s_pre[EXP_TILE] = run;
        }
        if (threadIdx.x == 0) {
            u64 pre = 0;
            if (tile == 0) {
                st_relaxed(seg_status, lb_word(LB_PREFIX, epoch, total));
            } else {
                st_relaxed(seg_status + tile * LB_PAD, lb_word(LB_AGG, epoch, total));
                pre = lookback_exclusive_win<16>(seg_status, LB_PAD, tile, epoch, err);
                st_relaxed(seg_status + tile * LB_PAD, lb_word(LB_PREFIX, epoch, pre + total));
            }
            s_prefix = pre;
        }
        __syncthreads();
        const u64 o = key_base[c] + s_prefix;
        const uint32_t T = (uint32_t)total;
        if (o + T > key_base[c + 1]) {
            raise_error(err, HSK_DERR_BOUNDS);
            continue;
        }
        // ---- expand: key j of the tile belongs to the last record with s_pre[r] <= j
        for (uint32_t j = threadIdx.x; j < T; j += 256) {
            uint32_t lo = 0, hi = nr;  // s_pre[lo] <= j < s_pre[hi]
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (s_pre[mid] <= j) lo = mid;
                else hi = mid;
            }
            const uint32_t jj = j - s_pre[lo];
            u64 W[4];
            W[0] = s_rec[lo * RW];
            W[1] = s_rec[lo * RW + 1];
            W[2] = WIDE ? s_rec[lo * RW + 2] : 0ULL;
            W[3] = WIDE ? s_rec[lo * RW + 3] : 0ULL;
            if (!WIDE) {
                u64 key = canonical64(record_kmer64(W, jj, k), k);
                reinterpret_cast<u64*>(keys_out)[o + j] = key;
                for (int p = 0; p < n_pass; ++p) atomicAdd(&s_hist[p * RADIX + key_digit(key, 8 * p, 0xFF)], 1u);
            } else {
                key128 key = canonical128(record_kmer128(W, jj, k), k);
                reinterpret_cast<ulonglong2*>(keys_out)[o + j] = make_ulonglong2(key.lo, key.hi);
                for (int p = 0; p < n_pass; ++p) atomicAdd(&s_hist[p * RADIX + key_digit(key, 8 * p, 0xFF)], 1u);
            }
        }
    }
}

void launch_expand_seg(const uint64_t* records, const uint64_t* rec_base, const uint64_t* key_base,
                       uint32_t C, uint64_t max_tiles, int k, void* keys, uint64_t* status,
                       uint32_t* tile_ctrs, uint32_t epoch, uint64_t* hist, int n_pass, int* err,
                       int grid, cudaStream_t st) {
    if (C == 0 || max_tiles == 0) return;
    count_launch();
    uint64_t want = (uint64_t)C * max_tiles;
    unsigned g = (unsigned)(want < (uint64_t)grid ? want : (uint64_t)grid);
    if (g < C) g = C;  // every segment gets a starting CTA
    const u64 stride = (max_tiles + 1) * LB_PAD;
    const size_t dyn = (size_t)EXP_TILE * (k <= 32 ? 2 : 4) * sizeof(u64);
    if (k <= 32) {
        cudaFuncSetAttribute(k_expand_seg<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        k_expand_seg<false><<<g, 256, dyn, st>>>((const u64*)records, (const u64*)rec_base, (const u64*)key_base, C,
                                               k, keys, (u64*)status, stride, tile_ctrs, epoch, (u64*)hist,
                                               n_pass, err);
    } else {
        cudaFuncSetAttribute(k_expand_seg<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        k_expand_seg<true><<<g, 256, dyn, st>>>((const u64*)records, (const u64*)rec_base, (const u64*)key_base, C,
                                                k, keys, (u64*)status, stride, tile_ctrs, epoch, (u64*)hist,
                                                n_pass, err);
    }
}

// ---------------------------------------------------------------------------
// up-front digit histograms of plain keys (one segment)
// ---------------------------------------------------------------------------
template <typename K>
__global__ void __launch_bounds__(256) k_digit_hist(const K* __restrict__ keys, u64 n,
                                                    u64* __restrict__ hist, int n_pass) {
    __shared__ uint32_t s_hist[MAX_PASS * RADIX];
    for (int i = threadIdx.x; i < n_pass * RADIX; i += 256) s_hist[i] = 0;
    __syncthreads();
    for (u64 i = (u64)blockIdx.x * 256 + threadIdx.x; i < n; i += (u64)gridDim.x * 256) {
        K key = keys[i];
        for (int p = 0; p < n_pass; ++p) atomicAdd(&s_hist[p * RADIX + key_digit(key, 8 * p, 0xFF)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_pass * RADIX; i += 256)
        if (s_hist[i]) atomicAdd(reinterpret_cast<unsigned long long*>(hist + i), (unsigned long long)s_hist[i]);
}

void launch_digit_hist(const void* keys, int key_words, uint64_t n, uint64_t* hist, int n_pass,
                       int grid, cudaStream_t st) {
    if (n == 0) return;
    count_launch();
    uint64_t need = (n + 255) / 256;
    unsigned g = (unsigned)(need < (uint64_t)grid ? need : (uint64_t)grid);
    if (key_words == 1)
        k_digit_hist<u64><<<g, 256, 0, st>>>((const u64*)keys, n, (u64*)hist, n_pass);
    else
        k_digit_hist<key128><<<g, 256, 0, st>>>((const key128*)keys, n, (u64*)hist, n_pass);
}

// Digit histograms of C consecutive segments of plain keys: hist[c][p][256]
// for keys [key_base[c], key_base[c + 1]).  Block b takes keys [b * chunk,
// (b + 1) * chunk) and counts the segments that range meets one after the
// other, flushing each segment's counts before starting the next.
template <typename K>
__global__ void __launch_bounds__(256) k_digit_hist_seg(const K* __restrict__ keys, const u64* __restrict__ key_base,
                                                        uint32_t C, u64 n, u64 chunk, u64* __restrict__ hist,
                                                        int n_pass, int shift0) {
    __shared__ uint32_t s_hist[MAX_PASS * RADIX];
    const u64 r0 = (u64)blockIdx.x * chunk;
    const u64 r1 = r0 + chunk < n ? r0 + chunk : n;
    if (r0 >= r1) return;
    uint32_t c = 0, hi = C;  // key_base[c] <= r0 < key_base[hi]
    while (hi - c > 1) {
        const uint32_t mid = (c + hi) >> 1;
        if (key_base[mid] <= r0) c = mid;
        else hi = mid;
    }
    for (; c < C && key_base[c] < r1; ++c) {
        const u64 a = key_base[c] > r0 ? key_base[c] : r0;
        const u64 b = key_base[c + 1] < r1 ? key_base[c + 1] : r1;
        if (a >= b) continue;  // empty segment (uniform)
        for (int i = threadIdx.x; i < n_pass * RADIX; i += 256) s_hist[i] = 0;
        __syncthreads();
        for (u64 i = a + threadIdx.x; i < b; i += 256) {
            const K key = keys[i];
            for (int p = 0; p < n_pass; ++p) atomicAdd(&s_hist[p * RADIX + key_digit(key, shift0 + 8 * p, 0xFF)], 1u);
        }
        __syncthreads();
        u64* h = hist + (u64)c * n_pass * RADIX;
        for (int i = threadIdx.x; i < n_pass * RADIX; i += 256)
            if (s_hist[i]) atomicAdd(reinterpret_cast<unsigned long long*>(h + i), (unsigned long long)s_hist[i]);
        __syncthreads();
    }
}

void launch_digit_hist_seg(const void* keys, int key_words, const uint64_t* key_base, uint32_t C, uint64_t n,
                           uint64_t* hist, int n_pass, cudaStream_t st, int shift0) {
    if (n == 0 || C == 0) return;
    count_launch();
    const u64 chunk = 32768;
    const unsigned g = (unsigned)((n + chunk - 1) / chunk);
    if (key_words == 1)
        k_digit_hist_seg<u64><<<g, 256, 0, st>>>((const u64*)keys, (const u64*)key_base, C, n, chunk, (u64*)hist,
                                                 n_pass, shift0);
    else
        k_digit_hist_seg<key128><<<g, 256, 0, st>>>((const key128*)keys, (const u64*)key_base, C, n, chunk,
                                                    (u64*)hist, n_pass, shift0);
}

// dst[i] = src[idx[i]], i < n
__global__ void k_gather_u64(const u64* __restrict__ src, const u64* __restrict__ idx, uint32_t n,
                             u64* __restrict__ dst) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[idx[i]];
}

void launch_gather_u64(const uint64_t* src, const uint64_t* idx, uint32_t n, uint64_t* dst, cudaStream_t st) {
    if (n == 0) return;
    count_launch();
    const unsigned g = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
    k_gather_u64<<<g, 256, 0, st>>>((const u64*)src, (const u64*)idx, n, (u64*)dst);
}

// doff[(p * C + c) * 256 + d] = key_base[c] + sum over d' < d of hist[(c * P + p) * 256 + d']
__global__ void __launch_bounds__(256) k_digit_offsets_seg(const u64* __restrict__ hist, const u64* __restrict__ key_base,
                                                           u64* __restrict__ doff, int n_pass, uint32_t C) {
    __shared__ u64 s_scr[9];
    const int p = blockIdx.x;
    const uint32_t c = blockIdx.y;
    u64 v = hist[((u64)c * n_pass + p) * RADIX + threadIdx.x], total;
    u64 e = block_excl_sum<256, u64>(v, s_scr, total);
    doff[((u64)p * C + c) * RADIX + threadIdx.x] = key_base[c] + e;
}

void launch_digit_offsets_seg(const uint64_t* hist, const uint64_t* key_base, uint64_t* doff, int n_pass,
                              uint32_t C, cudaStream_t st) {
    if (n_pass <= 0 || C == 0) return;
    count_launch();
    k_digit_offsets_seg<<<dim3(n_pass, C), 256, 0, st>>>((const u64*)hist, (const u64*)key_base, (u64*)doff,
                                                         n_pass, C);
}

// ---------------------------------------------------------------------------
// one onesweep LSD pass over all segments
// ---------------------------------------------------------------------------
template <typename K>
struct PassCfg;
#ifndef HSK_OS_ITEMS_U64
#define HSK_OS_ITEMS_U64 8
#endif
template <>
struct PassCfg<u64> {
    static constexpr int ITEMS = HSK_OS_ITEMS_U64;  // 8: 2048 keys, 16 KB per tile
};
template <>
struct PassCfg<key128> {
    static constexpr int ITEMS = 8;   // 2048 keys, 32 KB per tile
};

uint64_t onesweep_tile_keys(int key_words) {
    return 256ull * (key_words == 1 ? PassCfg<u64>::ITEMS : PassCfg<key128>::ITEMS);
}

// Segment c and its tile j of global tile g, and the first status tile of
// the segment.  Interleaved (tile_start == nullptr): segment g % C, tile
// g / C, status tiles [c * tmax, (c + 1) * tmax).  Listed: segment c owns
// the consecutive global tiles [tile_start[c], tile_start[c + 1]) (C + 1
// entries, empty segments repeat an entry) and their status tiles.
__device__ __forceinline__ void seg_tile(uint32_t g, uint32_t C, uint32_t tmax, const uint32_t* tile_start,
                                         uint32_t& c, uint32_t& j, u64& st0) {
    if (tile_start) {
        uint32_t lo = 0, hi = C;  // tile_start[lo] <= g < tile_start[hi]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (tile_start[mid] <= g) lo = mid;
            else hi = mid;
        }
        c = lo;
        j = g - tile_start[lo];
        st0 = tile_start[lo];
    } else {
        c = g % C;
        j = g / C;
        st0 = (u64)c * tmax;
    }
}

__device__ __forceinline__ u64 load_stream(const u64* p) { return __ldcs(reinterpret_cast<const unsigned long long*>(p)); }
__device__ __forceinline__ key128 load_stream(const key128* p) {
    ulonglong2 v = __ldcs(reinterpret_cast<const ulonglong2*>(p));
    return key128{v.x, v.y};
}

// Registers per thread are capped so that 4 CTAs of 256 threads fit an SM
// (64 registers); ranks are kept as 16-bit halves (a tile holds < 65536 keys).
// Segment c holds keys [key_base[c], key_base[c+1]) in both buffers; the
// look-back word of digit d of tile j of segment c is status[(c*tmax + j)*256 + d].
template <typename K, bool HAS_VAL>
__global__ void __launch_bounds__(256, HAS_VAL ? 3 : 4)
    k_onesweep_seg(const K* __restrict__ kin, K* __restrict__ kout, const uint32_t* __restrict__ vin,
                   uint32_t* __restrict__ vout, const u64* __restrict__ key_base, uint32_t C, uint32_t tmax,
                   const uint32_t* __restrict__ tile_start, int shift, const u64* __restrict__ doff, u64* status,
                   uint32_t* tile_ctr, uint32_t epoch, int* err) {
    constexpr int ITEMS = PassCfg<K>::ITEMS;
    constexpr int TILE = 256 * ITEMS;
    constexpr int WARPS = 8;
    extern __shared__ __align__(16) unsigned char smem[];
    K* s_keys = reinterpret_cast<K*>(smem);                                   // TILE keys
    uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + TILE);            // TILE values
    __shared__ uint32_t s_whist[WARPS][RADIX];   // per-warp digit counts, then offsets
    __shared__ uint32_t s_tstart[RADIX];         // tile-local start of each digit
    __shared__ u64 s_gbase[RADIX];               // global position of tile-local index 0
    __shared__ uint32_t s_scr[9];
    __shared__ uint32_t s_tile;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
    for (int i = threadIdx.x; i < WARPS * RADIX; i += 256) (&s_whist[0][0])[i] = 0;
    __syncthreads();
    const uint32_t g = s_tile;
    uint32_t c, tile;
    u64 st0;
    seg_tile(g, C, tmax, tile_start, c, tile, st0);
    const u64 sb = key_base[c], sn = key_base[c + 1] - sb;
    if ((u64)tile * TILE >= sn) return;  // this segment has fewer tiles (uniform exit)
    const u64 base = sb + (u64)tile * TILE;
    const u64 seg_end = sb + sn;
    const u64 wbase = base + (u64)warp * (ITEMS * 32);

    K key[ITEMS];
    uint32_t val[HAS_VAL ? ITEMS : 1];
    uint32_t rank2[ITEMS / 2];  // two 16-bit in-warp ranks per register
    // keys of this warp that exist (the last tile of a segment is partial)
    const int wvalid = seg_end > wbase ? (int)(seg_end - wbase < (u64)(ITEMS * 32) ? seg_end - wbase : (u64)(ITEMS * 32)) : 0;
    const K* wk = kin + wbase;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (i * 32 + lane < wvalid) {
            key[i] = load_stream(wk + i * 32 + lane);
            if (HAS_VAL) val[i] = __ldcs(vin + wbase + i * 32 + lane);
        } else {
            key[i] = K{};
            if (HAS_VAL) val[i] = 0;
        }
    }
    // ---- rank within the warp, in index order (stable) ----
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const bool ok = i * 32 + lane < wvalid;
        uint32_t d = ok ? key_digit(key[i], shift, 0xFF) : RADIX;  // RADIX: padding
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t below = __popc(peers & lt);
        uint32_t cnt = __popc(peers);
        uint32_t b = ok ? s_whist[warp][d] : 0u;
        __syncwarp();
        if (ok && below == 0) s_whist[warp][d] = b + cnt;
        __syncwarp();
        uint32_t r = b + below;
        if (i & 1) rank2[i / 2] |= r << 16;
        else rank2[i / 2] = r;
    }
    __syncthreads();
    // ---- per digit: exclusive offsets across warps, tile count ----
    const uint32_t d = threadIdx.x;  // 256 threads == 256 digits
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
        uint32_t cc = s_whist[w][d];
        s_whist[w][d] = cnt;
        cnt += cc;
    }
    // publish this tile's count of digit d (its look-back comes after the keys
    // have left the registers).  Status words are laid out [segment][tile]
    // [digit]: a tile publishes its 256 words into 2 KB of its own, so tiles
    // never contend for the same L2 sectors.
    u64* seg_status = status + st0 * RADIX;
    u64* my = seg_status + (u64)tile * RADIX + d;
    if (tile == 0) st_relaxed(my, lb_word(LB_PREFIX, epoch, cnt));
    else st_relaxed(my, lb_word(LB_AGG, epoch, cnt));
    uint32_t tot;
    uint32_t tstart = block_excl_sum<256, uint32_t>(cnt, s_scr, tot);
    s_tstart[d] = tstart;
    __syncthreads();
    // ---- place keys in shared memory in tile-sorted order ----
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (i * 32 + lane < wvalid) {
            uint32_t dd = key_digit(key[i], shift, 0xFF);
            uint32_t rr = (i & 1) ? (rank2[i / 2] >> 16) : (rank2[i / 2] & 0xFFFFu);
            uint32_t r = s_tstart[dd] + s_whist[warp][dd] + rr;
            s_keys[r] = key[i];
            if (HAS_VAL) s_vals[r] = val[i];
        }
    }
    // ---- look back for the tile's offset of digit d within its segment ----
    u64 excl = 0;
    if (tile > 0) {
        excl = lookback_exclusive_win<8>(seg_status + d, RADIX, tile, epoch, err);
        st_relaxed(my, lb_word(LB_PREFIX, epoch, excl + cnt));
    }
    s_gbase[d] = doff[(u64)c * RADIX + d] + excl - tstart;
    __syncthreads();
    // ---- scatter: consecutive threads write consecutive slots of a digit ----
    const uint32_t tile_n = (uint32_t)(seg_end - base < (u64)TILE ? seg_end - base : (u64)TILE);
    for (uint32_t j = threadIdx.x; j < tile_n; j += 256) {
        K kk = s_keys[j];
        u64 pos = s_gbase[key_digit(kk, shift, 0xFF)] + j;
        if (pos < sb || pos >= seg_end) {  // only after a failed look-back: never write out of bounds
            raise_error(err, HSK_DERR_BOUNDS);
            continue;
        }
        kout[pos] = kk;
        if (HAS_VAL) vout[pos] = s_vals[j];
    }
}

template <typename K, bool HV>
static void launch_pass_t(const void* kin, void* kout, const uint32_t* vin, uint32_t* vout, const uint64_t* key_base,
                          uint32_t C, uint32_t tmax, const uint32_t* tile_start, int shift, const uint64_t* doff,
                          uint64_t* status, uint32_t* tile_ctr, uint32_t epoch, int* err, cudaStream_t st) {
    constexpr int TILE = 256 * PassCfg<K>::ITEMS;
    size_t smem = (size_t)TILE * sizeof(K) + (HV ? (size_t)TILE * sizeof(uint32_t) : 0);
    auto fn = k_onesweep_seg<K, HV>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    count_launch();
    const uint64_t blocks = tile_start ? (uint64_t)tmax : (uint64_t)C * tmax;
    fn<<<(unsigned)blocks, 256, smem, st>>>((const K*)kin, (K*)kout, vin, vout, (const u64*)key_base, C, tmax,
                                            tile_start, shift, (const u64*)doff, (u64*)status, tile_ctr, epoch, err);
}

// ---------------------------------------------------------------------------
// the same pass, persistent, with TMA-staged tiles (keys only)
// ---------------------------------------------------------------------------
// Each CTA takes tiles from the counter in order.  While it ranks, looks back
// and scatters one tile, the keys of the next tile it has claimed are already
// being copied into its other shared-memory buffer by a TMA bulk copy, so the
// SM always has a tile load in flight.  A copy starts at the 16-byte boundary
// at or below the tile (so `pre` keys of the previous tile lead the buffer)
// and covers whole 16-byte units inside the segment; a key left over at the
// end is loaded by one thread.  For the first tile of a u64 key array that
// starts 8 bytes past a 16-byte boundary the copy begins 8 bytes before the
// array: device allocations are at least 256-byte aligned, so those bytes lie
// in the same allocation; they are staged but never used or written.
// Threads per CTA and keys per thread of the TMA pass (compile-time knobs);
// CTAs per SM follow from the registers and the two staging buffers.
#ifndef HSK_TMA_NT
#define HSK_TMA_NT 256
#endif
#ifndef HSK_TMA_CTAS
#define HSK_TMA_CTAS 4
#endif
template <typename K>
struct TmaCfg;
template <>
struct TmaCfg<u64> {
    static constexpr int NT = HSK_TMA_NT, ITEMS = 256 * HSK_OS_ITEMS_U64 / HSK_TMA_NT;
};
template <>
struct TmaCfg<key128> {
    static constexpr int NT = HSK_TMA_NT, ITEMS = 256 * 8 / HSK_TMA_NT;
};
template <typename K>
constexpr int tma_buf_bytes() {
    return ((TmaCfg<K>::NT * TmaCfg<K>::ITEMS * (int)sizeof(K) + 16) + 127) & ~127;
}
// the host sizes segments' tile counts with the PassCfg tile: keep them equal
static_assert(TmaCfg<u64>::NT * TmaCfg<u64>::ITEMS == 256 * PassCfg<u64>::ITEMS, "tile sizes differ");
static_assert(TmaCfg<key128>::NT * TmaCfg<key128>::ITEMS == 256 * PassCfg<key128>::ITEMS, "tile sizes differ");

template <typename K>
__global__ void __launch_bounds__(TmaCfg<K>::NT, HSK_TMA_CTAS)
    k_onesweep_tma(const K* __restrict__ kin, K* __restrict__ kout, const u64* __restrict__ key_base, uint32_t C,
                   uint32_t tmax, const uint32_t* __restrict__ tile_start, int shift, const u64* __restrict__ doff,
                   u64* status, uint32_t* tile_ctr, uint32_t epoch, int* err) {
    constexpr int NT = TmaCfg<K>::NT;
    constexpr int ITEMS = TmaCfg<K>::ITEMS;
    constexpr int TILE = NT * ITEMS;
    constexpr int WARPS = NT / 32;
    constexpr int BUF = tma_buf_bytes<K>();
    extern __shared__ __align__(128) unsigned char smem_tma[];  // two staging buffers of BUF bytes
    __shared__ uint32_t s_whist[WARPS][RADIX];
    __shared__ uint32_t s_tstart[RADIX];
    __shared__ u64 s_gbase[RADIX];
    __shared__ uint32_t s_scr[NT / 32 + 1];
    __shared__ __align__(8) u64 s_bar[2];
    __shared__ uint32_t s_next;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t total = tile_start ? tmax : C * tmax;

    // geometry of global tile g (seg_tile)
    auto geom = [&](uint32_t g, u64& sb, u64& seg_end, u64& base, uint32_t& n_t) -> bool {
        uint32_t c, j;
        u64 st0;
        seg_tile(g, C, tmax, tile_start, c, j, st0);
        sb = key_base[c];
        seg_end = key_base[c + 1];
        base = sb + (u64)j * TILE;
        if (base >= seg_end) return false;
        n_t = (uint32_t)(seg_end - base < (u64)TILE ? seg_end - base : (u64)TILE);
        return true;
    };
    auto lead = [&](u64 base) -> uint32_t {
        return (uint32_t)((reinterpret_cast<uintptr_t>(kin + base) & 15) / sizeof(K));
    };
    // thread 0: start the copy of tile g into buffer b (returns whether one started)
    int outstanding[2] = {0, 0};  // thread 0: a copy into buffer b not yet waited for
    auto issue = [&](uint32_t g, int b) -> bool {
        u64 sb, se, base;
        uint32_t n_t;
        if (!geom(g, sb, se, base, n_t)) return false;
        outstanding[b] = 1;
        const uint32_t pre = lead(base);
        const uint32_t bulk = ((n_t + pre) * (uint32_t)sizeof(K)) & ~15u;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&s_bar[b], bulk);
        if (bulk)
            tma_load_1d(smem_tma + b * BUF, reinterpret_cast<const unsigned char*>(kin + base) - pre * sizeof(K), bulk,
                        &s_bar[b]);
        return true;
    };

    if (threadIdx.x == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        mbar_init_fence();
        const uint32_t g0 = atomicAdd(tile_ctr, 1u);
        s_next = g0;
        if (g0 < total) issue(g0, 0);
    }
    __syncthreads();
    uint32_t g = s_next;
    uint32_t ph0 = 0, ph1 = 0;
    int b = 0;
    bool failed = false;
    while (g < total) {
        __syncthreads();  // s_next consumed; buffer b ^ 1 idle since the last iteration
        if (threadIdx.x == 0) {
            const uint32_t gn = atomicAdd(tile_ctr, 1u);
            s_next = gn;
            if (gn < total) issue(gn, b ^ 1);
        }
        for (int i = threadIdx.x; i < WARPS * RADIX; i += NT) (&s_whist[0][0])[i] = 0;
        u64 sb, seg_end, base;
        uint32_t tile_n;
        if (geom(g, sb, seg_end, base, tile_n)) {
            const uint32_t parity = b ? ph1 : ph0;
            if (mbar_wait(&s_bar[b], parity, err)) {  // phase done: the next use waits on the other parity
                if (b) ph1 ^= 1u;
                else ph0 ^= 1u;
                outstanding[b] = 0;
            } else {
                failed = true;
            }
            K* stage = reinterpret_cast<K*>(smem_tma + b * BUF);
            const uint32_t pre = lead(base);
            const uint32_t bulk_keys = (((tile_n + pre) * (uint32_t)sizeof(K)) & ~15u) / (uint32_t)sizeof(K);
            if (threadIdx.x == 0 && bulk_keys < tile_n + pre) stage[tile_n + pre - 1] = kin[base + tile_n - 1];
            __syncthreads();
            if (__syncthreads_or(failed)) break;  // a copy never arrived: stop (the error word is set)

            const int wvalid = (int)tile_n - warp * (ITEMS * 32) > 0
                                   ? ((int)tile_n - warp * (ITEMS * 32) < ITEMS * 32 ? (int)tile_n - warp * (ITEMS * 32)
                                                                                      : ITEMS * 32)
                                   : 0;
            const K* wk = stage + pre + warp * (ITEMS * 32);
            K key[ITEMS];
            uint32_t rank2[ITEMS / 2];
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) key[i] = i * 32 + lane < wvalid ? wk[i * 32 + lane] : K{};
            // ---- rank within the warp, in index order (stable)
            const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const bool ok = i * 32 + lane < wvalid;
                uint32_t d = ok ? key_digit(key[i], shift, 0xFF) : RADIX;
                uint32_t peers = __match_any_sync(0xffffffffu, d);
                uint32_t below = __popc(peers & lt);
                uint32_t cnt = __popc(peers);
                uint32_t bb = ok ? s_whist[warp][d] : 0u;
                __syncwarp();
                if (ok && below == 0) s_whist[warp][d] = bb + cnt;
                __syncwarp();
                uint32_t r = bb + below;
                if (i & 1) rank2[i / 2] |= r << 16;
                else rank2[i / 2] = r;
            }
            __syncthreads();  // every key is in registers: the buffer may be overwritten
            const uint32_t d = threadIdx.x;  // threads 0..255: one digit each
            const bool dig = d < RADIX;
            uint32_t cnt = 0;
            if (dig) {
#pragma unroll
                for (int w = 0; w < WARPS; ++w) {
                    uint32_t cc = s_whist[w][d];
                    s_whist[w][d] = cnt;
                    cnt += cc;
                }
            }
            uint32_t c, tile;
            u64 st0;
            seg_tile(g, C, tmax, tile_start, c, tile, st0);
            u64* seg_status = status + st0 * RADIX;
            u64* my = seg_status + (u64)tile * RADIX + d;
            if (dig) {
                if (tile == 0) st_relaxed(my, lb_word(LB_PREFIX, epoch, cnt));
                else st_relaxed(my, lb_word(LB_AGG, epoch, cnt));
            }
            uint32_t tot;
            const uint32_t tstart = block_excl_sum<NT, uint32_t>(cnt, s_scr, tot);
            if (dig) s_tstart[d] = tstart;
            __syncthreads();
            // ---- place keys in the buffer in tile-sorted order (from index 0)
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                if (i * 32 + lane < wvalid) {
                    uint32_t dd = key_digit(key[i], shift, 0xFF);
                    uint32_t rr = (i & 1) ? (rank2[i / 2] >> 16) : (rank2[i / 2] & 0xFFFFu);
                    stage[s_tstart[dd] + s_whist[warp][dd] + rr] = key[i];
                }
            }
            // ---- look back for the tile's offset of digit d within its segment
            if (dig) {
                u64 excl = 0;
                if (tile > 0) {
                    excl = lookback_exclusive_win<8>(seg_status + d, RADIX, tile, epoch, err);
                    st_relaxed(my, lb_word(LB_PREFIX, epoch, excl + cnt));
                }
                s_gbase[d] = doff[(u64)c * RADIX + d] + excl - tstart;
            }
            __syncthreads();
            // ---- scatter: consecutive threads write consecutive slots of a digit
            for (uint32_t j = threadIdx.x; j < tile_n; j += NT) {
                K kk = stage[j];
                u64 pos = s_gbase[key_digit(kk, shift, 0xFF)] + j;
                if (pos < sb || pos >= seg_end) {
                    raise_error(err, HSK_DERR_BOUNDS);
                    continue;
                }
                kout[pos] = kk;
            }
        }
        __syncthreads();  // buffer b free again; s_next visible
        g = s_next;
        b ^= 1;
    }
    if (failed && threadIdx.x == 0) {
        // a copy did not arrive in time: give the copies still in flight a
        // bounded chance to land before the CTA's shared memory is released
        if (outstanding[0]) mbar_wait(&s_bar[0], ph0, nullptr);
        if (outstanding[1]) mbar_wait(&s_bar[1], ph1, nullptr);
    }
}

void launch_onesweep_seg(const void* kin, void* kout, const uint32_t* vin, uint32_t* vout,
                         const uint64_t* key_base, uint32_t C, uint32_t tmax, const uint32_t* tile_start,
                         int key_words, int shift, const uint64_t* doff, uint64_t* status, uint32_t* tile_ctr,
                         uint32_t epoch, int* err, cudaStream_t st) {
    if (C == 0 || tmax == 0) return;
    bool hv = vin != nullptr;
    if (!hv && key_words == 2) {
        // 128-bit keys alone: the tile-per-CTA pass (the persistent TMA pass
        // below measured slower for them: 1.5 against 2.7 TB/s)
        launch_pass_t<key128, false>(kin, kout, nullptr, nullptr, key_base, C, tmax, tile_start, shift, doff, status,
                                     tile_ctr, epoch, err, st);
        return;
    }
    if (!hv) {  // persistent, TMA-staged pass
        static int num_sms = 0;
        if (!num_sms) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
            if (num_sms <= 0) num_sms = 1;
        }
        const uint64_t tiles = tile_start ? (uint64_t)tmax : (uint64_t)C * tmax;
        const unsigned grid = (unsigned)(tiles < (uint64_t)num_sms * HSK_TMA_CTAS ? tiles : (uint64_t)num_sms * HSK_TMA_CTAS);
        count_launch();
        if (key_words == 1) {
            const size_t smem = 2 * (size_t)tma_buf_bytes<u64>();
            cudaFuncSetAttribute(k_onesweep_tma<u64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_onesweep_tma<u64><<<grid, TmaCfg<u64>::NT, smem, st>>>((const u64*)kin, (u64*)kout, (const u64*)key_base, C, tmax,
                                                         tile_start, shift, (const u64*)doff, (u64*)status, tile_ctr,
                                                         epoch, err);
        } else {
            const size_t smem = 2 * (size_t)tma_buf_bytes<key128>();
            cudaFuncSetAttribute(k_onesweep_tma<key128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_onesweep_tma<key128><<<grid, TmaCfg<key128>::NT, smem, st>>>((const key128*)kin, (key128*)kout, (const u64*)key_base,
                                                            C, tmax, tile_start, shift, (const u64*)doff, (u64*)status,
                                                            tile_ctr, epoch, err);
        }
        return;
    }
    if (key_words == 1)
        launch_pass_t<u64, true>(kin, kout, vin, vout, key_base, C, tmax, tile_start, shift, doff, status, tile_ctr,
                                 epoch, err, st);
    else
        launch_pass_t<key128, true>(kin, kout, vin, vout, key_base, C, tmax, tile_start, shift, doff, status,
                                    tile_ctr, epoch, err, st);
}

// ---------------------------------------------------------------------------
// S6 on chip: sort sub-ranges that already share their top digits
// ---------------------------------------------------------------------------
// After the kept pairs are laid out by their top digit and one segmented pass
// has grouped each top-digit range by the second digit, every sub-range
// holds pairs whose keys agree above bit `shift + 8`.  One CTA takes a
// sub-range: it counts the keys' digit at `shift` (256 bins), places the
// pairs bin by bin in shared memory, and writes each key to its sorted place:
// the start of its bin plus the number of smaller keys in the bin (the keys
// are distinct, so the places are too).
constexpr int RS_NT = 512;
template <typename K>
struct RangeCfg;
template <>
struct RangeCfg<u64> {
    static constexpr int CAP = 8192;  // 96 KB: two CTAs per SM
};
template <>
struct RangeCfg<key128> {
    static constexpr int CAP = 8192;  // 160 KB
};
uint32_t range_sort_cap(int key_words) { return key_words == 1 ? RangeCfg<u64>::CAP : RangeCfg<key128>::CAP; }

template <typename K>
__global__ void __launch_bounds__(RS_NT) k_range_sort(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                      K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                      const u64* __restrict__ bounds, uint32_t n_ranges, int shift,
                                                      int* too_big, uint32_t* claim) {
    constexpr int CAP = RangeCfg<K>::CAP;
    extern __shared__ __align__(16) unsigned char smem_rs[];
    K* sk = reinterpret_cast<K*>(smem_rs);
    uint32_t* sv = reinterpret_cast<uint32_t*>(sk + CAP);
    __shared__ uint32_t s_cnt[RADIX], s_start[RADIX], s_fill[RADIX];
    __shared__ uint32_t s_scr[RS_NT / 32 + 1];
    __shared__ uint32_t s_next;
    const int tid = threadIdx.x;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_next = atomicAdd(claim, 1u);
        if (tid < RADIX) s_cnt[tid] = 0;
        __syncthreads();
        const uint32_t r = s_next;
        if (r >= n_ranges) break;
        const u64 b = bounds[r], e = bounds[r + 1];
        if (e <= b) continue;
        const uint32_t n = (uint32_t)(e - b);
        if (e - b > (u64)CAP) {
            if (tid == 0) atomicExch(too_big, 1);
            continue;
        }
        if (n == 1) {
            if (tid == 0) {
                kout[b] = kin[b];
                vout[b] = vin[b];
            }
            continue;
        }
        for (uint32_t i = tid; i < n; i += RS_NT) atomicAdd(&s_cnt[key_digit(kin[b + i], shift, 0xFF)], 1u);
        __syncthreads();
        uint32_t tot;
        const uint32_t c = tid < RADIX ? s_cnt[tid] : 0u;
        const uint32_t ex = block_excl_sum<RS_NT, uint32_t>(c, s_scr, tot);
        if (tid < RADIX) {
            s_start[tid] = ex;
            s_fill[tid] = ex;
        }
        __syncthreads();
        for (uint32_t i = tid; i < n; i += RS_NT) {
            const K key = kin[b + i];
            const uint32_t at = atomicAdd(&s_fill[key_digit(key, shift, 0xFF)], 1u);
            sk[at] = key;
            sv[at] = vin[b + i];
        }
        __syncthreads();
        for (uint32_t i = tid; i < n; i += RS_NT) {
            const K key = sk[i];
            const uint32_t d = key_digit(key, shift, 0xFF);
            const uint32_t bs = s_start[d], be = bs + s_cnt[d];
            uint32_t rank = 0;
            for (uint32_t j = bs; j < be; ++j) rank += key_lt(sk[j], key) ? 1u : 0u;
            kout[b + bs + rank] = key;
            vout[b + bs + rank] = sv[i];
        }
    }
}

void launch_range_sort(const void* kin, const uint32_t* vin, void* kout, uint32_t* vout, const uint64_t* bounds,
                       uint32_t n_ranges, int key_words, int shift, int* too_big, uint32_t* claim, int num_sms,
                       cudaStream_t st) {
    if (n_ranges == 0) return;
    count_launch();
    if (key_words == 1) {
        const size_t dyn = (size_t)RangeCfg<u64>::CAP * 12;
        cudaFuncSetAttribute(k_range_sort<u64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_range_sort<u64>, RS_NT, dyn);
        if (occ < 1) occ = 1;
        const uint64_t want = (uint64_t)num_sms * occ;
        const unsigned g = (unsigned)(n_ranges < want ? n_ranges : want);
        k_range_sort<u64><<<g, RS_NT, dyn, st>>>((const u64*)kin, vin, (u64*)kout, vout, (const u64*)bounds,
                                                 n_ranges, shift, too_big, claim);
    } else {
        const size_t dyn = (size_t)RangeCfg<key128>::CAP * 20;
        cudaFuncSetAttribute(k_range_sort<key128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_range_sort<key128>, RS_NT, dyn);
        if (occ < 1) occ = 1;
        const uint64_t want = (uint64_t)num_sms * occ;
        const unsigned g = (unsigned)(n_ranges < want ? n_ranges : want);
        k_range_sort<key128><<<g, RS_NT, dyn, st>>>((const key128*)kin, vin, (key128*)kout, vout,
                                                    (const u64*)bounds, n_ranges, shift, too_big, claim);
    }
}

// ---------------------------------------------------------------------------
// S6 with the counts carried in the keys' spare bits
// ---------------------------------------------------------------------------
// A key of 2k bits sorted on its ceil(2k/8) 8-bit digits leaves the bits from
// cshift = 8 * ceil(2k/8) up unexamined by every pass; when the counts fit
// there, the pairs are sorted as keys alone (key-only passes move 8 * words
// bytes per element instead of 8 * words + 4).
template <typename K>
__global__ void __launch_bounds__(256) k_pack_pairs(K* keys, const uint32_t* __restrict__ counts, u64 n, int cshift) {
    for (u64 i = (u64)blockIdx.x * 256 + threadIdx.x; i < n; i += (u64)gridDim.x * 256) {
        if constexpr (std::is_same<K, u64>::value) keys[i] |= (u64)counts[i] << cshift;
        else keys[i].hi |= (u64)counts[i] << (cshift - 64);
    }
}

template <typename K>
__global__ void __launch_bounds__(256) k_unpack_pairs(K* keys, uint32_t* __restrict__ counts, u64 n, int cshift) {
    for (u64 i = (u64)blockIdx.x * 256 + threadIdx.x; i < n; i += (u64)gridDim.x * 256) {
        if constexpr (std::is_same<K, u64>::value) {
            const u64 v = keys[i];
            counts[i] = (uint32_t)(v >> cshift);
            keys[i] = v & ((1ULL << cshift) - 1);
        } else {
            const u64 h = keys[i].hi;
            const int s = cshift - 64;
            counts[i] = (uint32_t)(h >> s);
            keys[i].hi = s == 0 ? 0ULL : (h & ((1ULL << s) - 1));
        }
    }
}

void launch_pack_pairs(void* keys, uint32_t* counts, uint64_t n, int key_words, int cshift, bool unpack, int grid,
                       cudaStream_t st) {
    if (n == 0) return;
    count_launch();
    const uint64_t need = (n + 255) / 256;
    const unsigned g = (unsigned)(need < (uint64_t)grid ? need : (uint64_t)grid);
    if (key_words == 1) {
        if (unpack) k_unpack_pairs<u64><<<g, 256, 0, st>>>((u64*)keys, counts, n, cshift);
        else k_pack_pairs<u64><<<g, 256, 0, st>>>((u64*)keys, counts, n, cshift);
    } else {
        if (unpack) k_unpack_pairs<key128><<<g, 256, 0, st>>>((key128*)keys, counts, n, cshift);
        else k_pack_pairs<key128><<<g, 256, 0, st>>>((key128*)keys, counts, n, cshift);
    }
}

// ---------------------------------------------------------------------------
// failure detection: the look-back wait on a word nothing publishes
// ---------------------------------------------------------------------------
// Tile 1 waits for tile 0's status word, which stays zero: the wait gives up
// after spin_limit polls, records HSK_DERR_TIMEOUT and the kernel returns.
__global__ void k_debug_wait(u64* status, uint32_t spin_limit, int* err) {
    if (threadIdx.x == 0) (void)lookback_exclusive(status, LB_PAD, 1, 1, err, spin_limit);
}

void launch_debug_wait(uint64_t* status, uint32_t spin_limit, int* err, cudaStream_t st) {
    count_launch();
    k_debug_wait<<<1, 32, 0, st>>>((u64*)status, spin_limit, err);
}

}  // namespace hsk
