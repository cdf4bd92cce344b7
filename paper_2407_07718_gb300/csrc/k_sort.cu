// k_sort.cu -- stage S4: LSD radix sort of packed k-mer keys (Sec. 3.1: sort
// the k-mers so equal values become adjacent, then count them with one linear
// scan).  The paper sorts each task on the CPU with RADULS (out of place) or
// PARADIS (in place); on the GPU the sort is a onesweep-style LSD radix sort
// (Adinets & Merrill, 2022): one up-front pass builds the digit histograms of
// every pass, then each pass ranks a tile of keys in shared memory, obtains
// the tile's global digit offsets by decoupled look-back over earlier tiles
// and scatters the tile, digit by digit, with contiguous writes.
//
//   k_expand      -- supermer records -> canonical keys, plus the up-front
//                    digit histograms of all passes (fused: no extra read).
//   k_digit_hist  -- up-front histograms of plain keys (stage sort, S6).
//   k_onesweep    -- one 8-bit LSD pass; u64 keys (k <= 32) or 128-bit keys
//                    (k <= 64), optionally carrying a uint32 value.
#include "hsk_device.cuh"

namespace hsk {

constexpr int RADIX = 256;
constexpr int MAX_PASS = 16;

// ---------------------------------------------------------------------------
// supermer records -> keys (+ digit histograms)
// ---------------------------------------------------------------------------
constexpr int EXP_RPT = 4;                 // records per thread
constexpr int EXP_TILE = 256 * EXP_RPT;    // records per tile

uint64_t expand_status_words(uint64_t n_rec) { return (n_rec + EXP_TILE - 1) / EXP_TILE + 1; }
int expand_grid(int num_sms) { return num_sms * 4; }

__device__ __forceinline__ u64 sel4(const u64 (&W)[4], uint32_t i) {
    return i == 0 ? W[0] : i == 1 ? W[1] : i == 2 ? W[2] : i == 3 ? W[3] : 0ULL;
}

// k-mer j (k <= 32) of a record held in registers (no local-memory indexing).
__device__ __forceinline__ u64 record_kmer64(const u64 (&W)[4], uint32_t j, int k) {
    uint32_t i = j >> 5, off = (j & 31) * 2;
    return funnel64(sel4(W, i), sel4(W, i + 1), off) >> (64 - 2 * k);
}

// k-mer j (33 <= k <= 64) of a record held in registers.
__device__ __forceinline__ key128 record_kmer128(const u64 (&W)[4], uint32_t j, int k) {
    uint32_t i = j >> 5, off = (j & 31) * 2;
    u64 a = funnel64(sel4(W, i), sel4(W, i + 1), off);
    u64 b = funnel64(sel4(W, i + 1), sel4(W, i + 2), off);
    int s = 128 - 2 * k;
    key128 r;
    if (s == 0) {
        r.hi = a;
        r.lo = b;
    } else {
        r.hi = a >> s;
        r.lo = (b >> s) | (a << (64 - s));
    }
    return r;
}

template <bool WIDE>
__global__ void __launch_bounds__(256) k_expand(const u64* __restrict__ rec, u64 n_rec, int rec_words,
                                                int k, void* __restrict__ keys_out, u64 n_keys,
                                                u64* status, uint32_t* tile_ctr, uint32_t epoch,
                                                u64* __restrict__ hist, int n_pass, int* err) {
    __shared__ uint32_t s_hist[MAX_PASS * RADIX];
    __shared__ u64 s_scr[9];
    __shared__ u64 s_prefix;
    __shared__ uint32_t s_tile;
    for (int i = threadIdx.x; i < n_pass * RADIX; i += 256) s_hist[i] = 0;
    const u64 n_tiles = (n_rec + EXP_TILE - 1) / EXP_TILE;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
        __syncthreads();
        const u64 tile = s_tile;
        if (tile >= n_tiles) break;
        const u64 r0 = tile * EXP_TILE + (u64)threadIdx.x * EXP_RPT;
        u64 W[EXP_RPT][4];
        uint32_t nk[EXP_RPT];
        u64 sum = 0;
#pragma unroll
        for (int i = 0; i < EXP_RPT; ++i) {
            nk[i] = 0;
            W[i][0] = W[i][1] = W[i][2] = W[i][3] = 0;
            if (r0 + i < n_rec) {
                const u64* r = rec + (r0 + i) * (u64)rec_words;
                ulonglong2 a = *reinterpret_cast<const ulonglong2*>(r);
                W[i][0] = a.x;
                W[i][1] = a.y;
                if (WIDE) {
                    ulonglong2 b = *reinterpret_cast<const ulonglong2*>(r + 2);
                    W[i][2] = b.x;
                    W[i][3] = b.y;
                }
                nk[i] = (uint32_t)((WIDE ? W[i][3] : W[i][1]) & 0xFF);
            }
            sum += nk[i];
        }
        u64 total;
        u64 excl = block_excl_sum<256, u64>(sum, s_scr, total);
        if (threadIdx.x == 0) {
            u64 pre = 0;
            if (tile == 0) {
                st_relaxed(status, lb_word(LB_PREFIX, epoch, total));
            } else {
                st_relaxed(status + tile, lb_word(LB_AGG, epoch, total));
                pre = lookback_exclusive(status, 1, tile, epoch, err);
                st_relaxed(status + tile, lb_word(LB_PREFIX, epoch, pre + total));
            }
            s_prefix = pre;
        }
        __syncthreads();
        u64 o = s_prefix + excl;
        if (o + sum > n_keys) {
            raise_error(err, HSK_DERR_BOUNDS);
            continue;
        }
#pragma unroll
        for (int i = 0; i < EXP_RPT; ++i) {
            // the record's low 8 bits of its last word hold n; they never fall
            // inside a k-mer (n + k - 1 <= 32 * rec_words - 4 bases)
            for (uint32_t j = 0; j < nk[i]; ++j, ++o) {
                if (!WIDE) {
                    u64 key = canonical64(record_kmer64(W[i], j, k), k);
                    reinterpret_cast<u64*>(keys_out)[o] = key;
                    for (int p = 0; p < n_pass; ++p)
                        atomicAdd(&s_hist[p * RADIX + key_digit(key, 8 * p, 0xFF)], 1u);
                } else {
                    key128 key = canonical128(record_kmer128(W[i], j, k), k);
                    reinterpret_cast<ulonglong2*>(keys_out)[o] = make_ulonglong2(key.lo, key.hi);
                    for (int p = 0; p < n_pass; ++p)
                        atomicAdd(&s_hist[p * RADIX + key_digit(key, 8 * p, 0xFF)], 1u);
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_pass * RADIX; i += 256)
        if (s_hist[i]) atomicAdd(reinterpret_cast<unsigned long long*>(hist + i), (unsigned long long)s_hist[i]);
}

void launch_expand(const uint64_t* records, uint64_t n_rec, int rec_words, int k, void* keys,
                   uint64_t n_keys, uint64_t* status, uint32_t* tile_ctr, uint32_t epoch,
                   uint64_t* hist, int n_pass, int* err, int grid, cudaStream_t st) {
    if (n_rec == 0) return;
    count_launch();
    uint64_t tiles = (n_rec + EXP_TILE - 1) / EXP_TILE;
    unsigned g = (unsigned)(tiles < (uint64_t)grid ? tiles : (uint64_t)grid);
    if (k <= 32)
        k_expand<false><<<g, 256, 0, st>>>((const u64*)records, n_rec, rec_words, k, keys, n_keys,
                                           (u64*)status, tile_ctr, epoch, (u64*)hist, n_pass, err);
    else
        k_expand<true><<<g, 256, 0, st>>>((const u64*)records, n_rec, rec_words, k, keys, n_keys,
                                          (u64*)status, tile_ctr, epoch, (u64*)hist, n_pass, err);
}

// ---------------------------------------------------------------------------
// up-front digit histograms of plain keys
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

__global__ void __launch_bounds__(256) k_digit_offsets(const u64* __restrict__ hist, u64* __restrict__ off) {
    __shared__ u64 s_scr[9];
    const int p = blockIdx.x;
    u64 v = hist[p * RADIX + threadIdx.x], total;
    u64 e = block_excl_sum<256, u64>(v, s_scr, total);
    off[p * RADIX + threadIdx.x] = e;
}

void launch_digit_offsets(const uint64_t* hist, uint64_t* digit_off, int n_pass, cudaStream_t st) {
    if (n_pass <= 0) return;
    count_launch();
    k_digit_offsets<<<n_pass, 256, 0, st>>>((const u64*)hist, (u64*)digit_off);
}

// ---------------------------------------------------------------------------
// one onesweep LSD pass
// ---------------------------------------------------------------------------
template <typename K>
struct PassCfg;
template <>
struct PassCfg<u64> {
    static constexpr int ITEMS = 16;  // 4096 keys, 32 KB per tile
};
template <>
struct PassCfg<key128> {
    static constexpr int ITEMS = 8;   // 2048 keys, 32 KB per tile
};

uint64_t onesweep_tiles(uint64_t n, int key_words) {
    uint64_t tile = 256ull * (key_words == 1 ? PassCfg<u64>::ITEMS : PassCfg<key128>::ITEMS);
    return (n + tile - 1) / tile;
}

template <typename K>
__device__ __forceinline__ K load_key(const K* p) { return *p; }

template <typename K, bool HAS_VAL>
__global__ void __launch_bounds__(256) k_onesweep(const K* __restrict__ kin, K* __restrict__ kout,
                                                  const uint32_t* __restrict__ vin,
                                                  uint32_t* __restrict__ vout, u64 n, int shift,
                                                  const u64* __restrict__ digit_off, u64* status,
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
    const u64 tile = s_tile;
    const u64 base = tile * TILE;
    const u64 wbase = base + (u64)warp * (ITEMS * 32);

    K key[ITEMS];
    uint32_t val[ITEMS];
    uint32_t rank[ITEMS];
    uint32_t dig[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        u64 idx = wbase + i * 32 + lane;
        bool ok = idx < n;
        if (ok) {
            key[i] = kin[idx];
            if (HAS_VAL) val[i] = vin[idx];
        } else {
            key[i] = K{};
            val[i] = 0;
        }
        dig[i] = ok ? key_digit(key[i], shift, 0xFF) : RADIX;  // RADIX: padding
    }
    // ---- rank within the warp, in index order (stable) ----
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint32_t d = dig[i];
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t below = __popc(peers & lt);
        uint32_t cnt = __popc(peers);
        uint32_t b = d < RADIX ? s_whist[warp][d] : 0u;
        __syncwarp();
        if (d < RADIX && below == 0) s_whist[warp][d] = b + cnt;
        __syncwarp();
        rank[i] = b + below;
    }
    __syncthreads();
    // ---- per digit: exclusive offsets across warps, tile count ----
    const uint32_t d = threadIdx.x;  // 256 threads == 256 digits
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
        uint32_t c = s_whist[w][d];
        s_whist[w][d] = cnt;
        cnt += c;
    }
    // publish this tile's count of digit d, then look back for its prefix
    u64* my = status + tile * RADIX + d;
    if (tile == 0) st_relaxed(my, lb_word(LB_PREFIX, epoch, cnt));
    else st_relaxed(my, lb_word(LB_AGG, epoch, cnt));
    uint32_t tot;
    uint32_t tstart = block_excl_sum<256, uint32_t>(cnt, s_scr, tot);
    s_tstart[d] = tstart;
    u64 excl = 0;
    if (tile > 0) {
        excl = lookback_exclusive(status + d, RADIX, tile, epoch, err);
        st_relaxed(my, lb_word(LB_PREFIX, epoch, excl + cnt));
    }
    s_gbase[d] = digit_off[d] + excl - tstart;
    __syncthreads();
    // ---- place keys in shared memory in tile-sorted order ----
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint32_t dd = dig[i];
        if (dd < RADIX) {
            uint32_t r = s_tstart[dd] + s_whist[warp][dd] + rank[i];
            s_keys[r] = key[i];
            if (HAS_VAL) s_vals[r] = val[i];
        }
    }
    __syncthreads();
    // ---- scatter: consecutive threads write consecutive slots of a digit ----
    const uint32_t tile_n = (uint32_t)(n - base < (u64)TILE ? n - base : (u64)TILE);
    for (uint32_t j = threadIdx.x; j < tile_n; j += 256) {
        K kk = s_keys[j];
        u64 pos = s_gbase[key_digit(kk, shift, 0xFF)] + j;
        if (pos >= n) {  // only after a failed look-back: never write out of bounds
            raise_error(err, HSK_DERR_BOUNDS);
            continue;
        }
        kout[pos] = kk;
        if (HAS_VAL) vout[pos] = s_vals[j];
    }
}

template <typename K, bool HV>
static void launch_pass_t(const void* kin, void* kout, const uint32_t* vin, uint32_t* vout, uint64_t n,
                          int shift, const uint64_t* digit_off, uint64_t* status, uint32_t* tile_ctr,
                          uint32_t epoch, int* err, cudaStream_t st) {
    constexpr int TILE = 256 * PassCfg<K>::ITEMS;
    size_t smem = (size_t)TILE * sizeof(K) + (HV ? (size_t)TILE * sizeof(uint32_t) : 0);
    auto fn = k_onesweep<K, HV>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    uint64_t tiles = (n + TILE - 1) / TILE;
    count_launch();
    fn<<<(unsigned)tiles, 256, smem, st>>>((const K*)kin, (K*)kout, vin, vout, n, shift,
                                           (const u64*)digit_off, (u64*)status, tile_ctr, epoch, err);
}

void launch_onesweep(const void* kin, void* kout, const uint32_t* vin, uint32_t* vout, uint64_t n,
                     int key_words, int shift, const uint64_t* digit_off, uint64_t* status,
                     uint32_t* tile_ctr, uint32_t epoch, int* err, cudaStream_t st) {
    if (n == 0) return;
    bool hv = vin != nullptr;
    if (key_words == 1) {
        if (hv) launch_pass_t<u64, true>(kin, kout, vin, vout, n, shift, digit_off, status, tile_ctr, epoch, err, st);
        else launch_pass_t<u64, false>(kin, kout, vin, vout, n, shift, digit_off, status, tile_ctr, epoch, err, st);
    } else {
        if (hv) launch_pass_t<key128, true>(kin, kout, vin, vout, n, shift, digit_off, status, tile_ctr, epoch, err, st);
        else launch_pass_t<key128, false>(kin, kout, vin, vout, n, shift, digit_off, status, tile_ctr, epoch, err, st);
    }
}

}  // namespace hsk
