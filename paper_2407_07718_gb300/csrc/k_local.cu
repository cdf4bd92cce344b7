// k_local.cu -- stage S4 + S5 on chip: each minimizer-bucket group is cut by
// the top digit of its keys into 256 sub-segments, and every sub-segment that
// fits shared memory is sorted, run-length counted, histogrammed and filtered
// by one CTA without going back to HBM.
//
// The paper's tasks (Sec. 3.4) are independent groups of k-mers that each
// worker sorts on its own and then counts with one linear scan (Sec. 3.1).
// Here the tasks are cut fine enough to fit an SM: a bucket group never shares
// a k-mer value with another group, and within a group keys with different
// top digits differ, so every (group, top digit) sub-segment can be sorted and
// counted alone.  The global onesweep passes (k_sort.cu) stay as the path for
// sub-segments that do not fit.
//
//   k_part<MODE 0> -- supermer records -> key count per (group, top digit).
//   k_part<MODE 1> -- supermer records -> keys scattered to their
//                     sub-segments (a tile's keys are grouped by digit in
//                     shared memory first, so the writes are runs; the order
//                     inside a sub-segment is free, the sub-segment sort fixes it).
//   k_local_sort   -- per sub-segment: load into shared memory, MSD radix
//                     partitions (an 11-bit digit, then 8-bit digits where a
//                     bin stays large), runs counted inside each bin (key by
//                     key in small bins, by one warp peeling off distinct keys
//                     in larger ones), histogram, [lo, hi] filter; kept
//                     (key, count) pairs written at the start of the
//                     sub-segment's own range.  Launched in three tiers of
//                     capacity: the sub-segments that do not fit tier 0 go
//                     to tier 1 (1.5 times the capacity, two CTAs per SM),
//                     what does not fit there to tier 2 (three times, one
//                     CTA per SM); larger ones are heavy-hitter tasks
//                     (k_heavy_count), and what fits nothing is listed for
//                     the global path.
//   k_compact      -- kept pairs of all sub-segments -> one output array.
//   k_ov_gather    -- the listed sub-segments' keys -> one array for the
//                     global path.
#include "hsk_device.cuh"

namespace hsk {

constexpr int LP_NT = 256;

// ---------------------------------------------------------------------------
// partition by top digit (count, then scatter)
// ---------------------------------------------------------------------------
template <bool WIDE>
struct PartCfg {
    static constexpr int RW = WIDE ? 4 : 2;            // words per supermer record
    // keys grouped per scatter round; with 64-bit keys a smaller round lets a
    // fourth CTA fit an SM (long-read partition 11.55 -> 10.94 ms), with
    // 128-bit keys it did not pay (14.4 -> 16.5 ms)
    static constexpr int ROUND = 2048;
    static constexpr int CTAS = WIDE ? 3 : 4;  // scatter-pass CTAs per SM
    static constexpr int LR = ROUND / LP_NT;           // keys per thread and round
};
static_assert(EXP_TILE == 4 * LP_NT, "a thread sums the k-mer counts of four records");

// Dynamic shared memory of MODE 1: [keys grouped by digit][records][count prefix][counts]
size_t part_smem_bytes(int mode, int k) {
    if (mode == 0) return 0;
    const bool wide = k > 32;
    return (size_t)EXP_TILE * (wide ? 4 : 2) * 8 + (size_t)(EXP_TILE + 4) * 4 + EXP_TILE +
           (wide ? (size_t)PartCfg<true>::ROUND * 16 : (size_t)PartCfg<false>::ROUND * 8);
}

// Consecutive keys of a staged tile: key j is k-mer j - s_pre[r] of the
// record r with s_pre[r] <= j < s_pre[r + 1].  Moving forward only reads the
// next records' bounds, so a thread walking a run of keys finds its first
// record by binary search and the others by stepping.
template <bool WIDE>
struct TileWalk {
    using K = typename std::conditional<WIDE, key128, u64>::type;
    const u64* s_rec;
    const uint32_t* s_pre;
    uint32_t r, rb, re;
    u64 W[4];
    __device__ __forceinline__ void load() {
        constexpr int RW = PartCfg<WIDE>::RW;
        W[0] = s_rec[r * RW];
        W[1] = s_rec[r * RW + 1];
        W[2] = WIDE ? s_rec[r * RW + 2] : 0ULL;
        W[3] = WIDE ? s_rec[r * RW + 3] : 0ULL;
    }
    // start at key j < s_pre[nr] (the tile's key count)
    __device__ __forceinline__ void seek(uint32_t nr, uint32_t j) {
        uint32_t lo = 0, hi = nr;  // s_pre[lo] <= j < s_pre[hi]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_pre[mid] <= j) lo = mid;
            else hi = mid;
        }
        r = lo;
        rb = s_pre[lo];
        re = s_pre[lo + 1];
        load();
    }
    // canonical key j (j at or after the last key asked for, j < the tile's key count)
    __device__ __forceinline__ K key(uint32_t j, int k) {
        if (j >= re) {
            do {
                ++r;
                rb = re;
                re = s_pre[r + 1];
            } while (j >= re);
            load();
        }
        if constexpr (WIDE) return canonical128(record_kmer128(W, j - rb, k), k);
        else return canonical64(record_kmer64(W, j - rb, k), k);
    }
};

// The bases of a record from base p on, two bits each, most significant
// first: one 64-bit window of 32 bases, refilled from the record's words.
struct RecBases {
    u64 cur;
    uint32_t wi, off, left;
    __device__ __forceinline__ void start(const u64 (&W)[4], uint32_t p) {
        wi = p >> 5;
        off = (p & 31) * 2;
        left = 32;
        cur = funnel64(sel4(W, wi), sel4(W, wi + 1), off);
    }
    __device__ __forceinline__ uint32_t next(const u64 (&W)[4]) {
        const uint32_t b = (uint32_t)(cur >> 62);
        cur <<= 2;
        if (--left == 0) {
            ++wi;
            left = 32;
            cur = funnel64(sel4(W, wi), sel4(W, wi + 1), off);
        }
        return b;
    }
};

// Top 8-bit digit of the canonical code of every k-mer of a record (k >= 4).
// The canonical code is the smaller of the forward code and its reverse
// complement, so its first four bases are the smaller of the forward k-mer's
// first four bases and the reverse complement's first four (the k-mer's last
// four bases, complemented, in reverse order).  Two 8-bit windows roll along
// the record instead of the whole 2k-bit codes.
__device__ __forceinline__ uint32_t revcomp4(uint32_t x) {
    x = ~x & 0xFFu;
    return ((x & 3u) << 6) | ((x & 0xCu) << 2) | ((x >> 2) & 0xCu) | (x >> 6);
}
template <typename F>
__device__ __forceinline__ void record_top_digits(const u64 (&W)[4], uint32_t n, int k, F&& f) {
    if (n == 0) return;
    uint32_t fw = (uint32_t)(W[0] >> 56);  // bases 0..3
    RecBases lb;
    lb.start(W, (uint32_t)k - 4);           // bases k-4 .. k-1
    uint32_t last = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) last = (last << 2) | lb.next(W);
    uint32_t rc = revcomp4(last);
    f(min(fw, rc));
    RecBases fb;
    fb.start(W, 4u);
    for (uint32_t j = 1; j < n; ++j) {
        fw = ((fw << 2) | fb.next(W)) & 0xFFu;
        rc = (rc >> 2) | ((3u - lb.next(W)) << 6);
        f(min(fw, rc));
    }
}

// Work: one counter over all record tiles of all groups; tile g belongs to
// group tile_seg[g] and is tile g - tile_base[group] of it.
// MODE 0: sub_cnt[c * 256 + d] += keys of group c whose digit at `shift` is d.
//         Thread t holds records t, t + 256, ... of the tile (EXP_RPT of
//         them) and rolls through their k-mers: only the first and last four
//         bases when the digit is the key's top one (record_top_digits),
//         else the whole codes (record_kmers).
// MODE 1: every key to keys_out[cursor[c * 256 + d]++] (a reservation per
//         digit and round), never past sub_end[c * 256 + d].  The tile's
//         records are staged in shared memory with the prefix of their k-mer
//         counts; a round takes the tile's keys [j0, j0 + ROUND), LR
//         consecutive keys per thread, cut out of their records (TileWalk)
//         and held in registers, so every thread has the same number of keys
//         whatever the records' lengths.  The round is grouped by digit in
//         shared memory and written out as one run per digit.
// (Rolling is cheaper per key than cutting each key out, but a thread per
// record leaves lanes idle while the warp's longest record is expanded; in
// the count pass that costs less than cutting, in the scatter pass more.)
template <bool WIDE, int MODE>
__global__ void __launch_bounds__(LP_NT, MODE == 0 ? 4 : PartCfg<WIDE>::CTAS) k_part(const u64* __restrict__ rec, const u64* __restrict__ rec_base,
                                                const u64* __restrict__ tile_base, const uint32_t* __restrict__ tile_seg,
                                                uint32_t n_tiles, int k, int shift, uint32_t* tile_ctr,
                                                uint32_t* __restrict__ sub_cnt, unsigned long long* cursor,
                                                const u64* __restrict__ sub_end, void* __restrict__ keys_out,
                                                int* err) {
    using K = typename std::conditional<WIDE, key128, u64>::type;
    constexpr int RW = PartCfg<WIDE>::RW;
    constexpr int ROUND = PartCfg<WIDE>::ROUND;
    constexpr int LR = PartCfg<WIDE>::LR;
    extern __shared__ __align__(16) u64 smem_part[];
    K* s_keys = reinterpret_cast<K*>(smem_part);                    // MODE 1: a round grouped by digit
    u64* s_rec = smem_part + (size_t)ROUND * RW / 2;                 // MODE 1: the tile's records
    uint32_t* s_pre = reinterpret_cast<uint32_t*>(s_rec + (size_t)EXP_TILE * RW);  // [EXP_TILE + 1]
    uint8_t* s_nk = reinterpret_cast<uint8_t*>(s_pre + EXP_TILE + 4);              // [EXP_TILE]
    __shared__ uint32_t s_cnt[256], s_fill[256], s_dstart[256];
    __shared__ u64 s_gbase[256];
    __shared__ uint32_t s_scr32[9];
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x;
    s_cnt[tid] = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
        __syncthreads();
        const uint32_t g = s_tile;
        if (g >= n_tiles) break;
        const uint32_t c = tile_seg[g];
        const u64 tile = g - tile_base[c];
        const u64 rb = rec_base[c], n_rec = rec_base[c + 1] - rb;
        const u64 r0 = tile * EXP_TILE;
        const uint32_t nr = (uint32_t)(n_rec - r0 < (u64)EXP_TILE ? n_rec - r0 : (u64)EXP_TILE);
        const u64* trec = rec + (rb + r0) * RW;
        if constexpr (MODE == 0) {
            // this thread's records, in registers
            u64 W[EXP_RPT][4];
            uint32_t nk[EXP_RPT];
#pragma unroll
            for (int i = 0; i < EXP_RPT; ++i) {
                const uint32_t r = (uint32_t)i * LP_NT + tid;
                nk[i] = 0;
                W[i][0] = W[i][1] = W[i][2] = W[i][3] = 0;
                if (r < nr) {
                    const ulonglong2* q = reinterpret_cast<const ulonglong2*>(trec + (u64)r * RW);
                    const ulonglong2 a = q[0];
                    W[i][0] = a.x;
                    W[i][1] = a.y;
                    if (WIDE) {
                        const ulonglong2 b2 = q[1];
                        W[i][2] = b2.x;
                        W[i][3] = b2.y;
                    }
                    nk[i] = (uint32_t)(W[i][RW - 1] & 0xFF);
                }
            }
            if (k >= 4 && shift == 2 * k - 8) {  // the digit is the first four bases
#pragma unroll
                for (int i = 0; i < EXP_RPT; ++i)
                    record_top_digits(W[i], nk[i], k, [&](uint32_t d) { atomicAdd(&s_cnt[d], 1u); });
            } else {
#pragma unroll
                for (int i = 0; i < EXP_RPT; ++i)
                    record_kmers<WIDE>(W[i], nk[i], k, [&](uint32_t, const K& key) {
                        atomicAdd(&s_cnt[key_digit(key, shift, 0xFF)], 1u);
                    });
            }
            __syncthreads();
            const uint32_t v = s_cnt[tid];
            if (v) atomicAdd(sub_cnt + (u64)c * 256 + tid, v);
            s_cnt[tid] = 0;
        } else {
            // ---- stage the records (128-bit loads) and their k-mer counts
            {
                const ulonglong2* src = reinterpret_cast<const ulonglong2*>(trec);
                ulonglong2* dst = reinterpret_cast<ulonglong2*>(s_rec);
#pragma unroll
                for (int i = 0; i < EXP_RPT; ++i) {
                    const uint32_t r = (uint32_t)i * LP_NT + tid;
                    uint32_t n = 0;
                    if (r < nr) {
                        const ulonglong2 a = src[(size_t)r * (RW / 2)];
                        dst[(size_t)r * (RW / 2)] = a;
                        if (WIDE) {
                            const ulonglong2 b = src[(size_t)r * (RW / 2) + 1];
                            dst[(size_t)r * (RW / 2) + 1] = b;
                            n = (uint32_t)(b.y & 0xFF);
                        } else {
                            n = (uint32_t)(a.y & 0xFF);
                        }
                    }
                    s_nk[r] = (uint8_t)n;
                }
            }
            __syncthreads();
            uint32_t T;
            {
                // records 4t .. 4t+3: their counts' exclusive prefix
                const uint32_t q = reinterpret_cast<const uint32_t*>(s_nk)[tid];
                const uint32_t n0 = q & 0xFF, n1 = (q >> 8) & 0xFF, n2 = (q >> 16) & 0xFF, n3 = q >> 24;
                const uint32_t e = block_excl_sum<LP_NT, uint32_t>(n0 + n1 + n2 + n3, s_scr32, T);
                reinterpret_cast<uint4*>(s_pre)[tid] = make_uint4(e, e + n0, e + n0 + n1, e + n0 + n1 + n2);
                if (tid == 0) s_pre[EXP_TILE] = T;
            }
            __syncthreads();
            TileWalk<WIDE> walk{s_rec, s_pre};
            // Four barriers a round.  A thread clears its digit counter as soon
            // as it has read it, and the round's write-out needs no barrier
            // after it: the next round writes only registers and s_cnt before
            // its first barrier, and the next tile's staging comes after the
            // tile loop's barriers.
            K* out = reinterpret_cast<K*>(keys_out);
            const int lane = tid & 31, warp = tid >> 5;
            for (uint32_t j0 = 0; j0 < T; j0 += ROUND) {
                const uint32_t nround = T - j0 < (uint32_t)ROUND ? T - j0 : (uint32_t)ROUND;
                // this thread's keys: [jb, je), at most LR of them
                const uint32_t jb = j0 + (uint32_t)tid * LR;
                const uint32_t je = jb + LR < j0 + nround ? jb + LR : j0 + nround;
                K kr[LR];
                if (jb < je) {
                    walk.seek(nr, jb);
#pragma unroll
                    for (int i = 0; i < LR; ++i) {
                        if (jb + i < je) {
                            kr[i] = walk.key(jb + i, k);
                            atomicAdd(&s_cnt[key_digit(kr[i], shift, 0xFF)], 1u);
                        }
                    }
                }
                __syncthreads();
                const uint32_t cnt = s_cnt[tid];
                s_cnt[tid] = 0;
                const uint32_t winc = warp_incl_sum<uint32_t>(cnt);
                if (lane == 31) s_scr32[warp] = winc;
                __syncthreads();
                uint32_t ex = winc - cnt;
                for (int w = 0; w < warp; ++w) ex += s_scr32[w];
                s_dstart[tid] = ex;
                s_fill[tid] = ex;
                if (cnt) {
                    const u64 slot = (u64)c * 256 + tid;
                    u64 at = atomicAdd(cursor + slot, (unsigned long long)cnt);
                    if (at + cnt > sub_end[slot]) {
                        raise_error(err, HSK_DERR_BOUNDS);
                        at = ~0ULL;
                    }
                    s_gbase[tid] = at;
                }
                __syncthreads();
#pragma unroll
                for (int i = 0; i < LR; ++i)  // group the round by digit
                    if (jb + i < je) s_keys[atomicAdd(&s_fill[key_digit(kr[i], shift, 0xFF)], 1u)] = kr[i];
                __syncthreads();
                for (uint32_t i = tid; i < nround; i += LP_NT) {
                    const K key = s_keys[i];
                    const uint32_t d = key_digit(key, shift, 0xFF);
                    const u64 at = s_gbase[d];
                    if (at != ~0ULL) out[at + (i - s_dstart[d])] = key;
                }
            }
        }
    }
}

void launch_part(int mode, const uint64_t* records, const uint64_t* rec_base, const uint64_t* tile_base,
                 const uint32_t* tile_seg, uint32_t n_tiles, int k, int shift, uint32_t* tile_ctr,
                 uint32_t* sub_cnt, uint64_t* cursor, const uint64_t* sub_end, void* keys, int* err, int grid,
                 cudaStream_t st) {
    if (n_tiles == 0) return;
    count_launch();
    unsigned g = n_tiles < (uint32_t)grid ? n_tiles : (unsigned)grid;
    if (g < 1) g = 1;
    const size_t dyn = part_smem_bytes(mode, k);
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        kern<<<g, LP_NT, dyn, st>>>((const u64*)records, (const u64*)rec_base, (const u64*)tile_base, tile_seg,
                                    n_tiles, k, shift, tile_ctr, sub_cnt, (unsigned long long*)cursor,
                                    (const u64*)sub_end, keys, err);
    };
    if (k <= 32) {
        if (mode == 0) go(k_part<false, 0>);
        else go(k_part<false, 1>);
    } else {
        if (mode == 0) go(k_part<true, 0>);
        else go(k_part<true, 1>);
    }
}

// ---------------------------------------------------------------------------
// sort + count one sub-segment in shared memory
// ---------------------------------------------------------------------------
// Bins of at most ls_small<K>() keys are counted key by key (every key of
// the bin compares itself with the others); larger ones through the
// equal-to-first-key mask.  The best cut was measured per key width: 16 for
// 64-bit keys (long-read workload: 8 -> 41.1 ms, 16 -> 31.8, 32 -> 35.5) and
// 32 for 128-bit keys (short-read workload: 16 -> 35.6 ms, 32 -> 32.2).
#ifndef HSK_LS_SMALL_U64
#define HSK_LS_SMALL_U64 16
#endif
#ifndef HSK_LS_SMALL_U128
#define HSK_LS_SMALL_U128 32
#endif
template <typename K>
constexpr int ls_small() { return sizeof(K) == 8 ? HSK_LS_SMALL_U64 : HSK_LS_SMALL_U128; }

// Capacity of one CTA's two shared-memory key buffers, per tier.  Tier 0
// (the first pass) runs 3 CTAs per SM.  The sub-segments that do not fit go
// to tier 1, 1.5 times the capacity with two CTAs per SM, and what does not
// fit there to tier 2, three times the capacity with one 512-thread CTA per
// SM.  (Tier 1 took the long-read workload's second-pass keys at about twice
// the rate of tier 2, whose single CTA per SM leaves the SM idle while its
// warps wait at barriers.)  STACK and LIST bound the open bins (disjoint,
// > LS_MED keys each) and the bins over ls_small<K>() keys.
template <typename K, int TIER>
struct LocalCfg;
template <>
struct LocalCfg<u64, 0> {
    static constexpr int CAP = 4096, STACK = 33, LIST = CAP / (HSK_LS_SMALL_U64 + 1) + 1;  // 2 x 32 KB
};
template <>
struct LocalCfg<key128, 0> {
    static constexpr int CAP = 2048, STACK = 17, LIST = CAP / (HSK_LS_SMALL_U128 + 1) + 1;  // 2 x 32 KB
};
template <>
struct LocalCfg<u64, 1> {
    static constexpr int CAP = 6144, STACK = 49, LIST = CAP / (HSK_LS_SMALL_U64 + 1) + 1;  // 2 x 48 KB
};
template <>
struct LocalCfg<key128, 1> {
    static constexpr int CAP = 3072, STACK = 25, LIST = CAP / (HSK_LS_SMALL_U128 + 1) + 1;  // 2 x 48 KB
};
template <>
struct LocalCfg<u64, 2> {
    static constexpr int CAP = 12288, STACK = 97, LIST = CAP / (HSK_LS_SMALL_U64 + 1) + 1;  // 2 x 96 KB
};
template <>
struct LocalCfg<key128, 2> {
    static constexpr int CAP = 6144, STACK = 49, LIST = CAP / (HSK_LS_SMALL_U128 + 1) + 1;   // 2 x 96 KB
};
template <int TIER>
struct TierCfg {
    static constexpr int NT = TIER == 2 ? 512 : 256;          // threads per CTA
    static constexpr int CTAS = TIER == 0 ? 3 : TIER == 1 ? 2 : 1;  // CTAs per SM
};
#ifndef HSK_LS_D1
#define HSK_LS_D1 11
#endif
constexpr int LS_D1 = HSK_LS_D1;   // bits of the first partition's digit (compile-time knob)
constexpr int LS_B1 = 1 << LS_D1;  // its bins (8 consecutive bins per thread)
// A warp peels up to LS_PEEL distinct keys off a larger bin; what is left is
// rank-sorted when it holds at most LS_MED keys, else partitioned again.
// Measured on the long-read workload (on-chip stage): LS_MED 256 / LS_PEEL 8
// 31.8 ms, 128 / 8 30.3, 256 / 16 29.7, 128 / 32 29.0, 64 / 32 37.8.
constexpr int LS_MED = 128;
constexpr int LS_PEEL = 32;
constexpr int LS_HS = 128;         // count-histogram bins kept in shared memory
// open bins are disjoint and hold > LS_MED keys; listed bins hold > ls_small<K>()
#define HSK_LS_CHECK(K, T)                                                                        \
    static_assert(LocalCfg<K, T>::CAP / (LS_MED + 1) < LocalCfg<K, T>::STACK, "stack too small"); \
    static_assert(LocalCfg<K, T>::CAP / (ls_small<K>() + 1) < LocalCfg<K, T>::LIST, "list too small")
HSK_LS_CHECK(u64, 0);
HSK_LS_CHECK(u64, 1);
HSK_LS_CHECK(u64, 2);
HSK_LS_CHECK(key128, 0);
HSK_LS_CHECK(key128, 1);
HSK_LS_CHECK(key128, 2);

uint32_t local_cap_tier(int key_words, int tier) {
    if (key_words == 1) return tier == 0 ? LocalCfg<u64, 0>::CAP : tier == 1 ? LocalCfg<u64, 1>::CAP : LocalCfg<u64, 2>::CAP;
    return tier == 0 ? LocalCfg<key128, 0>::CAP : tier == 1 ? LocalCfg<key128, 1>::CAP : LocalCfg<key128, 2>::CAP;
}
uint32_t local_cap(int key_words) { return local_cap_tier(key_words, 0); }
uint32_t local_cap_big(int key_words) { return local_cap_tier(key_words, 2); }
static size_t local_smem_bytes(int key_words, int tier) {
    return (size_t)2 * local_cap_tier(key_words, tier) * 8 * key_words;
}

struct LsBin {
    uint32_t beg, len;
    int shift, buf;  // digit of the next partition; buffer holding the bin (0 = A, 1 = B)
};

// Counting inside one sub-segment.  After the partitions, keys that are
// equal share every digit and so one bin; a bin's runs are found without
// ordering it: a key starts a run when no earlier key of the bin equals it,
// and the run's count is the number of keys of the bin equal to it (bins of
// <= ls_small<K>() keys, one thread per key).  A warp takes larger bins by
// peeling off one distinct key at a time (warp_bin); what is left after
// LS_PEEL peels is rank-sorted and scanned, or, past LS_MED keys,
// partitioned again on the next 8-bit digit by the whole CTA.  Every run
// goes to `emit`.
template <typename K, typename Emit>
__device__ __forceinline__ void thread_bin(const K* v, uint32_t c, Emit& emit) {
    for (uint32_t i = 0; i < c; ++i) {
        const K x = v[i];
        bool head = true;
        uint32_t cnt = 0;
        for (uint32_t j = 0; j < c; ++j)
            if (key_eq(v[j], x)) {
                ++cnt;
                head = head && j >= i;
            }
        if (head) emit(x, cnt);
    }
}

// A warp counts bin [sb, sb + len) of `src` (buffer src_buf; the same range
// of `other` is free).  Peeling: the first remaining key's copies are
// counted with one ballot pass over the bin and emitted, the other keys are
// compacted into the other buffer, and so on -- a bin that holds a k-mer and
// a few variants of it (sequencing errors past the digits already used) takes
// one pass per distinct key.  The last <= 32 keys are counted lane-parallel.
// After LS_PEEL peels the rest is rank-sorted and scanned (<= LS_MED keys) or
// pushed for another partition.
template <int STACK, typename K, typename Emit>
__device__ __forceinline__ void warp_bin(K* src, K* other, uint32_t sb, uint32_t len, int next_shift, bool last_digit,
                                         int src_buf, LsBin* stack, int* sp, int* abort_flag, int* err, Emit& emit) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    K* cur = src;
    K* oth = other;
    int cur_buf = src_buf;
    uint32_t m = len;
    for (int it = 0; m > 0; ++it) {
        if (m <= 32) {
            K x{};
            bool head = false;
            uint32_t cnt = 0;
            if ((uint32_t)lane < m) {
                x = cur[sb + lane];
                head = true;
                for (uint32_t j = 0; j < m; ++j)
                    if (key_eq(cur[sb + j], x)) {
                        ++cnt;
                        head = head && j >= (uint32_t)lane;
                    }
            }
            if (head) emit(x, cnt);
            return;
        }
        if (it == LS_PEEL) break;
        const K v = cur[sb];
        uint32_t cnt = 0, kept = 0;
        for (uint32_t i0 = 0; i0 < m; i0 += 32) {
            const uint32_t i = i0 + lane;
            const bool in = i < m;
            const K x = in ? cur[sb + i] : v;
            const bool eq = in && key_eq(x, v);
            cnt += (uint32_t)__popc(__ballot_sync(0xffffffffu, eq));
            const bool rest = in && !eq;
            const uint32_t rm = __ballot_sync(0xffffffffu, rest);
            if (rest) oth[sb + kept + (uint32_t)__popc(rm & lt)] = x;
            kept += (uint32_t)__popc(rm);
        }
        if (lane == 0) emit(v, cnt);
        __syncwarp();
        K* t = cur;
        cur = oth;
        oth = t;
        cur_buf ^= 1;
        m = kept;
    }
    if (m <= (uint32_t)LS_MED) {  // many distinct keys left: rank sort into oth, then scan
        for (uint32_t i = lane; i < m; i += 32) {
            const K v = cur[sb + i];
            uint32_t r = 0;
            for (uint32_t j = 0; j < m; ++j) {
                const K u = cur[sb + j];
                r += (key_lt(u, v) || (j < i && key_eq(u, v))) ? 1u : 0u;
            }
            oth[sb + r] = v;
        }
        __syncwarp();
        const K* w = oth + sb;
        for (uint32_t i = lane; i < m; i += 32) {
            if (i > 0 && key_eq(w[i], w[i - 1])) continue;
            uint32_t j = i + 1;
            while (j < m && key_eq(w[j], w[i])) ++j;
            emit(w[i], j - i);
        }
        __syncwarp();
        return;
    }
    if (lane == 0) {
        if (last_digit) {  // keys equal on every digit yet different: cannot happen
            raise_error(err, HSK_DERR_BOUNDS);
            *abort_flag = 1;
        } else {
            const int p = atomicAdd(sp, 1);
            if (p < STACK) stack[p] = LsBin{sb, m, next_shift, cur_buf};
            else *abort_flag = 1;
        }
    }
}

// Keys of sub-segment (list entry) idx into pf: thread t takes keys t,
// t + 256, ...; nothing when idx is past the end or the sub-segment is too
// large for one CTA.
template <int CAP, typename K, int PFN>
__device__ __forceinline__ void ls_prefetch(K (&pf)[PFN], const K* keys, const u64* sub_off, const uint32_t* only,
                                            uint32_t n_sub, uint32_t idx) {
    if (idx >= n_sub) return;
    const uint32_t ps = only ? only[idx] : idx;
    const u64 pb = sub_off[ps], pm = sub_off[ps + 1] - pb;
    if (pm > (u64)CAP) return;
#pragma unroll
    for (int j = 0; j < PFN; ++j) {
        const uint32_t i = (uint32_t)j * LP_NT + threadIdx.x;
        if (i < pm) pf[j] = keys[pb + i];
    }
}

// Sub-segment s holds keys [sub_off[s], sub_off[s+1]) of `keys`; its top
// digit (bits shift0 and up) is common to all of them.  The first partition
// takes the next LS_D1 bits (count while loading, scan, scatter A -> B), so
// a bin holds about one distinct key; each thread then counts its 8
// consecutive bins, warps the larger ones.  Outputs: kc[s] kept pairs,
// written to keys[sub_off[s] + i] and kcount[sub_off[s] + i], i < kc[s]
// (in no particular order: stage S6 orders all pairs).  The counts of all
// runs go to the histogram, their number to n_distinct, the largest to max_count.
// Packed sets (grp_set != nullptr): group g belongs to set grp_set[g] and the
// statistics of its sub-segments (g * 256 + digit) go to that set's
// histogram hist + set * hist_len, n_distinct[set] and max_count[set].  A CTA
// takes sub-segments in ascending order, so the sets it meets ascend too; it
// keeps one set's statistics on chip and flushes them when the set changes.
template <typename K, int TIER>
__global__ void __launch_bounds__(TierCfg<TIER>::NT, TierCfg<TIER>::CTAS) k_local_sort(const u64* __restrict__ sub_off,
                                                      const uint32_t* __restrict__ only, uint32_t n_sub, int shift0,
                                                      K* keys, uint32_t* __restrict__ kcount,
                                                      uint32_t* __restrict__ kc, uint32_t* __restrict__ ov_list,
                                                      unsigned long long* ov_stats, uint32_t lo, uint32_t hi,
                                                      u64* __restrict__ hist, uint32_t hist_len,
                                                      uint32_t* max_count, unsigned long long* n_distinct,
                                                      const uint32_t* __restrict__ grp_set, uint32_t* claim,
                                                      int* err) {
    using Cfg = LocalCfg<K, TIER>;
    constexpr int CAP = Cfg::CAP;
    constexpr int NT = TierCfg<TIER>::NT;   // threads
    constexpr int BPT = LS_B1 / NT;       // first-partition bins per thread
    extern __shared__ __align__(16) unsigned char smem_local[];
    K* A = reinterpret_cast<K*>(smem_local);
    K* B = A + CAP;
    // s_cnt1: first-partition counts, then cursors (= bin ends after the
    // scatter); later its front holds the 8-bit partitions' counters/cursors
    __shared__ uint32_t s_cnt1[LS_B1];
    uint32_t* s_cnt = s_cnt1;              // [256]
    uint32_t* s_cur = s_cnt1 + 256;        // [256]
    __shared__ uint32_t s_list[Cfg::LIST]; // larger bins: start | length << 16
    __shared__ uint32_t s_eqf[CAP / 32];   // key equals the first key of its (larger) bin
    __shared__ uint32_t s_hist[LS_HS];
    __shared__ LsBin s_stack[Cfg::STACK];
    __shared__ uint32_t s_scr32[NT / 32 + 1];
    __shared__ int s_sp, s_abort, s_nl;
    __shared__ uint32_t s_kept, s_next;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t hs = hist_len < (uint32_t)LS_HS ? hist_len : (uint32_t)LS_HS;
    const int s1 = shift0 > LS_D1 ? shift0 - LS_D1 : 0;  // first partition's digit
    const int s2 = s1 > 8 ? s1 - 8 : 0;                 // then 8-bit digits
    for (int i = tid; i < LS_HS; i += NT) s_hist[i] = 0;
    u64 my_distinct = 0;
    uint32_t my_max = 0, my_ones = 0;
    u64 base = 0;
    uint32_t cur_set = 0xFFFFFFFFu;  // set whose statistics are held on chip (none yet)
    u64* hcur = hist;
    auto count_run = [&](uint32_t cnt) {
        if (cnt == 1) {
            ++my_ones;
        } else {
            const uint32_t b = cnt < hist_len - 1 ? cnt : hist_len - 1;
            if (b < hs) atomicAdd(&s_hist[b], 1u);
            else atomicAdd(reinterpret_cast<unsigned long long*>(hcur + b), 1ULL);
        }
        ++my_distinct;
        my_max = cnt > my_max ? cnt : my_max;
    };
    // the held statistics -> set `set` (all threads; leaves them cleared)
    auto flush_stats = [&](uint32_t set) {
        if (my_ones) atomicAdd(&s_hist[1], my_ones);  // hist_len >= 2: count 1 has its own bin
        __syncthreads();
        u64* h = hist + (u64)set * hist_len;
        for (uint32_t i = tid; i < hs; i += NT) {
            const uint32_t v = s_hist[i];
            if (v) {
                atomicAdd(reinterpret_cast<unsigned long long*>(h + i), (unsigned long long)v);
                s_hist[i] = 0;
            }
        }
        const u64 d = warp_incl_sum<u64>(my_distinct);
        uint32_t mx = my_max;
        for (int o = 16; o > 0; o >>= 1) {
            const uint32_t v = __shfl_xor_sync(0xffffffffu, mx, o);
            mx = v > mx ? v : mx;
        }
        if (lane == 31 && d) atomicAdd(n_distinct + set, (unsigned long long)d);
        if (lane == 0 && mx) atomicMax(max_count + set, mx);
        my_distinct = 0;
        my_max = my_ones = 0;
        __syncthreads();
    };
    // one run, from a single lane
    auto emit = [&](const K& key, uint32_t cnt) {
        count_run(cnt);
        if (cnt >= lo && cnt <= hi) {
            const uint32_t p = atomicAdd(&s_kept, 1u);
            keys[base + p] = key;
            kcount[base + p] = cnt;
        }
    };
    // runs of the lanes with head set, all lanes of the warp calling
    auto emit_warp = [&](bool head, const K& key, uint32_t cnt) {
        if (head) count_run(cnt);
        const bool keep = head && cnt >= lo && cnt <= hi;
        const uint32_t km = __ballot_sync(0xffffffffu, keep);
        if (km) {
            const int leader = __ffs(km) - 1;
            uint32_t p0 = 0;
            if (lane == leader) p0 = atomicAdd(&s_kept, (uint32_t)__popc(km));
            p0 = __shfl_sync(0xffffffffu, p0, leader);
            if (keep) {
                const uint32_t p = p0 + (uint32_t)__popc(km & ((1u << lane) - 1u));
                keys[base + p] = key;
                kcount[base + p] = cnt;
            }
        }
    };
    // Sub-segments are claimed one at a time; the next one's keys are loaded
    // into registers while the current one is sorted (first pass only).
    constexpr int PF = TIER == 0 ? CAP / NT : 0;
    constexpr int PFN = PF > 0 ? PF : 1;
    K pf[PFN];
    // the first partition's counters start at zero; each sub-segment clears
    // them again after its last barrier, ready for the next one
#pragma unroll
    for (int j = 0; j < BPT; ++j) s_cnt1[tid * BPT + j] = 0;
    if (tid == 0) s_next = atomicAdd(claim, 1u);
    __syncthreads();
    uint32_t si = s_next;
    if (PF) ls_prefetch<CAP>(pf, keys, sub_off, only, n_sub, si);
    while (si < n_sub) {
        const uint32_t s = only ? only[si] : si;
        base = sub_off[s];
        const u64 n64 = sub_off[s + 1] - base;
        __syncthreads();  // every thread has read s_next; the last sub-segment's shared state is free
        if (tid == 0) s_next = atomicAdd(claim, 1u);
        {
            const uint32_t set = grp_set ? grp_set[s >> 8] : 0u;  // CTA-uniform
            if (set != cur_set) {
                if (cur_set != 0xFFFFFFFFu) flush_stats(cur_set);
                cur_set = set;
                hcur = hist + (u64)set * hist_len;
            }
        }
        if (n64 == 0 || n64 > (u64)CAP) {
            if (tid == 0) {
                kc[s] = 0;
                if (n64) {
                    ov_list[atomicAdd(reinterpret_cast<unsigned int*>(ov_stats), 1u)] = s;
                    atomicAdd(ov_stats + 1, (unsigned long long)n64);
                }
            }
            __syncthreads();
            si = s_next;
            if (PF) ls_prefetch<CAP>(pf, keys, sub_off, only, n_sub, si);
            continue;
        }
        const uint32_t n = (uint32_t)n64;
        if (tid == 0) {
            s_sp = 0;
            s_abort = 0;
            s_kept = 0;
            s_nl = 0;
        }
        if (shift0 == 0) {  // the top digit is the whole key: one run
            __syncthreads();
            if (tid == 0) {
                emit(keys[base], n);
                kc[s] = s_kept;
            }
            si = s_next;
            if (PF) ls_prefetch<CAP>(pf, keys, sub_off, only, n_sub, si);
            continue;
        }
        // ---- first partition: load + count, scan, scatter A -> B
        if (PF > 0) {
#pragma unroll
            for (int j = 0; j < PFN; ++j) {
                const uint32_t i = (uint32_t)j * NT + tid;
                if (i < n) {
                    A[i] = pf[j];
                    atomicAdd(&s_cnt1[key_digit(pf[j], s1, LS_B1 - 1)], 1u);
                }
            }
        } else {
            for (uint32_t i = tid; i < n; i += NT) {
                const K v = keys[base + i];
                A[i] = v;
                atomicAdd(&s_cnt1[key_digit(v, s1, LS_B1 - 1)], 1u);
            }
        }
        __syncthreads();
        const uint32_t nxt = s_next;
        if (PF) ls_prefetch<CAP>(pf, keys, sub_off, only, n_sub, nxt);
        uint32_t bc[BPT], sum = 0;
#pragma unroll
        for (int j = 0; j < BPT; ++j) {
            bc[j] = s_cnt1[tid * BPT + j];
            sum += bc[j];
        }
        // exclusive prefix of the per-thread sums: warp scan, then every warp
        // adds the totals of the warps before it (one barrier)
        const uint32_t winc = warp_incl_sum<uint32_t>(sum);
        if (lane == 31) s_scr32[warp] = winc;
        __syncthreads();
        uint32_t my0 = winc - sum;
        for (int w = 0; w < warp; ++w) my0 += s_scr32[w];
        {
            uint32_t run = my0;
#pragma unroll
            for (int j = 0; j < BPT; ++j) {
                s_cnt1[tid * BPT + j] = run;
                run += bc[j];
            }
        }
        __syncthreads();
        for (uint32_t i = tid; i < n; i += NT) {
            const K v = A[i];
            B[atomicAdd(&s_cnt1[key_digit(v, s1, LS_B1 - 1)], 1u)] = v;
        }
        __syncthreads();
        // ---- every key: its bin is [end of bin d-1, end of bin d).  In a
        // small bin the key counts its equals and emits at the first of them;
        // in a larger bin it only marks whether it equals the bin's first key,
        // and the bin's first key lists the bin.  The mask bit is set for the
        // small bins' keys too, so its zero bits are exactly the larger bins'
        // keys that differ from their bin's first key
        for (uint32_t i0 = 0; i0 < n; i0 += NT) {
            const uint32_t i = i0 + tid;
            bool head = false, eqf = false;
            uint32_t cnt = 0;
            K v{};
            if (i < n) {
                v = B[i];
                const uint32_t d = key_digit(v, s1, LS_B1 - 1);
                const uint32_t be = s_cnt1[d], bs = d ? s_cnt1[d - 1] : 0u;
                if (be - bs <= (uint32_t)ls_small<K>()) {
                    head = true;
                    eqf = true;  // counted here: the mask marks it done
                    for (uint32_t j = bs; j < be; ++j)
                        if (key_eq(B[j], v)) {
                            ++cnt;
                            head = head && j >= i;
                        }
                } else {
                    eqf = key_eq(v, B[bs]);
                    if (i == bs) s_list[atomicAdd(&s_nl, 1)] = bs | ((be - bs) << 16);
                }
            }
            const uint32_t fm = __ballot_sync(0xffffffffu, eqf);
            if (lane == 0 && i0 + (uint32_t)warp * 32 < n) s_eqf[(i0 >> 5) + warp] = fm;
            emit_warp(head, v, cnt);
        }
        __syncthreads();
        {
            // ---- larger bins of <= LS_MED keys.  Their keys that differ from
            // the bin's first key are few (sequencing-error variants of a
            // k-mer that shares the bin's digits): each counts its equals
            // among them through the mask's zero bits, key by key in parallel.
            // The first key's count is a popcount of the mask, one thread per bin.
            for (uint32_t i0 = 0; i0 < n; i0 += NT) {
                const uint32_t i = i0 + tid;
                bool head = false;
                uint32_t cnt = 0;
                K v{};
                if (i < n && !((s_eqf[i >> 5] >> (i & 31)) & 1u)) {
                    v = B[i];
                    const uint32_t d = key_digit(v, s1, LS_B1 - 1);
                    const uint32_t be = s_cnt1[d], bs = d ? s_cnt1[d - 1] : 0u;
                    if (be - bs > (uint32_t)ls_small<K>() && be - bs <= (uint32_t)LS_MED) {
                        head = true;
                        const uint32_t w0 = bs >> 5, w1 = (be - 1) >> 5;
                        for (uint32_t w = w0; w <= w1; ++w) {
                            uint32_t zm = ~s_eqf[w];
                            if (w == w0) zm &= 0xFFFFFFFFu << (bs & 31);
                            if (w == w1 && ((be - 1) & 31) != 31) zm &= (2u << ((be - 1) & 31)) - 1u;
                            for (; zm; zm &= zm - 1) {
                                const uint32_t j = w * 32 + (uint32_t)(__ffs(zm) - 1);
                                if (key_eq(B[j], v)) {
                                    ++cnt;
                                    head = head && j >= i;
                                }
                            }
                        }
                    }
                }
                emit_warp(head, v, cnt);
            }
            const int nl = s_nl;
            for (int q = tid; q < nl; q += NT) {
                const uint32_t bs = s_list[q] & 0xFFFFu, len = s_list[q] >> 16, be = bs + len;
                if (len > (uint32_t)LS_MED) continue;
                uint32_t c1 = 0;
                for (uint32_t w = bs >> 5; w <= (be - 1) >> 5; ++w) {
                    uint32_t m = s_eqf[w];
                    if (w == bs >> 5) m &= 0xFFFFFFFFu << (bs & 31);
                    if (w == (be - 1) >> 5 && ((be - 1) & 31) != 31) m &= (2u << ((be - 1) & 31)) - 1u;
                    c1 += (uint32_t)__popc(m);
                }
                emit(B[bs], c1);
            }
            // ---- bins of more than LS_MED keys: one warp each; the first
            // key's copies counted from the mask, the other keys compacted into
            // A and counted there
            for (int q = warp; q < nl; q += NT / 32) {
                const uint32_t bs = s_list[q] & 0xFFFFu, len = s_list[q] >> 16, be = bs + len;
                if (len <= (uint32_t)LS_MED) continue;
                const uint32_t w0 = bs >> 5, w1 = (be - 1) >> 5;
                uint32_t c1 = 0;
                for (uint32_t w = w0 + lane; w <= w1; w += 32) {
                    uint32_t m = s_eqf[w];
                    if (w == w0) m &= 0xFFFFFFFFu << (bs & 31);
                    if (w == w1 && ((be - 1) & 31) != 31) m &= (2u << ((be - 1) & 31)) - 1u;
                    c1 += (uint32_t)__popc(m);
                }
                for (int o = 16; o > 0; o >>= 1) c1 += __shfl_xor_sync(0xffffffffu, c1, o);
                if (lane == 0) emit(B[bs], c1);
                if (c1 == len) continue;
                // the keys at the mask's zero bits, compacted: each lane takes
                // one mask word, a warp scan of the words' counts places them
                uint32_t kept = 0;
                for (uint32_t wb = w0; wb <= w1; wb += 32) {
                    const uint32_t w = wb + lane;
                    uint32_t zm = 0;
                    if (w <= w1) {
                        zm = ~s_eqf[w];
                        if (w == w0) zm &= 0xFFFFFFFFu << (bs & 31);
                        if (w == w1 && ((be - 1) & 31) != 31) zm &= (2u << ((be - 1) & 31)) - 1u;
                    }
                    const uint32_t nz = (uint32_t)__popc(zm);
                    const uint32_t incl = warp_incl_sum<uint32_t>(nz);
                    uint32_t at = bs + kept + incl - nz;
                    for (; zm; zm &= zm - 1) A[at++] = B[w * 32 + (uint32_t)(__ffs(zm) - 1)];
                    kept += __shfl_sync(0xffffffffu, incl, 31);
                }
                __syncwarp();
                warp_bin<Cfg::STACK>(A, B, bs, kept, s2, s1 == 0, 0, s_stack, &s_sp, &s_abort, err, emit);
            }
        }
        __syncthreads();
        // ---- further 8-bit partitions of large bins that are not all equal
        for (;;) {
            const int sp = s_sp;
            if (sp == 0 || s_abort) break;
            const LsBin bin = s_stack[sp - 1];
            __syncthreads();
            if (tid == 0) {
                s_sp = sp - 1;
                s_nl = 0;
            }
            K* X = bin.buf ? B : A;
            K* Y = bin.buf ? A : B;
            if (tid < 256) s_cnt[tid] = 0;
            __syncthreads();
            for (uint32_t i = tid; i < bin.len; i += NT)
                atomicAdd(&s_cnt[key_digit(X[bin.beg + i], bin.shift, 0xFF)], 1u);
            __syncthreads();
            const uint32_t cnt = tid < 256 ? s_cnt[tid] : 0u;  // sub-bin (digit) tid
            uint32_t t2;
            const uint32_t ex = block_excl_sum<NT, uint32_t>(cnt, s_scr32, t2);
            if (tid < 256) s_cur[tid] = ex;
            __syncthreads();
            for (uint32_t i = tid; i < bin.len; i += NT) {
                const K v = X[bin.beg + i];
                Y[bin.beg + atomicAdd(&s_cur[key_digit(v, bin.shift, 0xFF)], 1u)] = v;
            }
            __syncthreads();
            const uint32_t sb = bin.beg + ex;
            if (cnt == 1) emit(Y[sb], 1u);
            else if (cnt > 1 && cnt <= (uint32_t)ls_small<K>()) thread_bin(Y + sb, cnt, emit);
            else if (cnt > (uint32_t)ls_small<K>())
                s_list[atomicAdd(&s_nl, 1)] = sb | (cnt << 16);
            __syncthreads();
            const int nl2 = s_nl;
            for (int q = warp; q < nl2; q += NT / 32)
                warp_bin<Cfg::STACK>(Y, X, s_list[q] & 0xFFFFu, s_list[q] >> 16, bin.shift > 8 ? bin.shift - 8 : 0,
                                     bin.shift == 0, bin.buf ^ 1, s_stack, &s_sp, &s_abort, err, emit);
            __syncthreads();
        }
        // The partition loop exits on a check made right after a barrier (the
        // one after the larger bins, or its own last one), so every run has
        // been emitted and the counters are no longer read: no barrier needed
        // before the kept count is stored and the counters cleared.
        // (s_abort: an impossible bin was met; raise_error has been called.)
        if (tid == 0) kc[s] = s_kept;
#pragma unroll
        for (int j = 0; j < BPT; ++j) s_cnt1[tid * BPT + j] = 0;
        si = nxt;
    }
    if (cur_set != 0xFFFFFFFFu) flush_stats(cur_set);
}

void launch_local_sort(const uint64_t* sub_off, const uint32_t* only, uint32_t n_sub, int tier, int shift0,
                       int key_words, void* keys, uint32_t* kcount, uint32_t* kc, uint32_t* ov_list,
                       uint64_t* ov_stats, uint32_t lo, uint32_t hi, uint64_t* hist, uint32_t hist_len,
                       uint32_t* max_count, uint64_t* n_distinct, const uint32_t* grp_set, uint32_t* claim,
                       int* err, int num_sms, cudaStream_t st) {
    if (n_sub == 0) return;
    count_launch();
    const size_t dyn = local_smem_bytes(key_words, tier);
    const int nt = tier == 2 ? TierCfg<2>::NT : TierCfg<0>::NT;
    auto go = [&](auto kern, auto* kp) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nt, dyn);
        if (occ < 1) occ = 1;
        uint64_t want = n_sub;
        uint64_t g = (uint64_t)num_sms * occ;
        if (want < g) g = want;
        kern<<<(unsigned)g, nt, dyn, st>>>((const u64*)sub_off, only, n_sub, shift0, kp, kcount, kc, ov_list,
                                              (unsigned long long*)ov_stats, lo, hi, (u64*)hist, hist_len,
                                              max_count, (unsigned long long*)n_distinct, grp_set, claim, err);
    };
    if (key_words == 1) {
        if (tier == 2) go(k_local_sort<u64, 2>, (u64*)keys);
        else if (tier == 1) go(k_local_sort<u64, 1>, (u64*)keys);
        else go(k_local_sort<u64, 0>, (u64*)keys);
    } else {
        if (tier == 2) go(k_local_sort<key128, 2>, (key128*)keys);
        else if (tier == 1) go(k_local_sort<key128, 1>, (key128*)keys);
        else go(k_local_sort<key128, 0>, (key128*)keys);
    }
}

// ---------------------------------------------------------------------------
// heavy-hitter sub-segments (64-bit keys): the k-mer list of a task
// ---------------------------------------------------------------------------
// Sec. 3.5: a task whose size exceeds a constant times the mean task size
// holds heavy hitters (many copies of a few k-mers, from genomic repeats);
// such a task is transformed into a k-mer list -- one (k-mer, count) tuple
// per distinct k-mer -- instead of being counted the normal way.  Here the
// tasks are the sub-segments, a heavy one is one over the largest on-chip
// tier's capacity (about nine times the mean sub-segment), and since a
// sub-segment holds every copy of each of its k-mers, its k-mer list is the
// exact count: one CTA folds the sub-segment's keys into a shared-memory table
// (open addressing, a 64-bit compare-and-swap claims a slot, an atomic add
// counts), then every slot is one distinct k-mer with its count, which goes to
// the histogram and the [lo, hi] filter like any run.  A sub-segment whose
// distinct keys would fill the table past HV_FILL is listed for the global
// radix path instead.
constexpr int HV_NT = 1024;
constexpr int HV_SLOTS = 16384;               // 128 KB keys + 64 KB counts
constexpr int HV_PF = 8;                      // keys per thread loaded ahead in one round
constexpr int HV_FILL = HV_SLOTS * 7 / 8;     // most distinct keys held before giving up
constexpr int HV_LIST = HV_FILL + HV_NT;      // claimed slots (each thread claims at most one past HV_FILL)
static_assert(HV_LIST < HV_SLOTS, "the table never fills: every probe sequence ends");
constexpr u64 HV_EMPTY = ~0ULL;               // never a canonical key (all-T's reverse complement is smaller)

size_t heavy_smem_bytes() { return (size_t)HV_SLOTS * (8 + 4) + (size_t)HV_LIST * 2; }

__global__ void __launch_bounds__(HV_NT, 1) k_heavy_count(const u64* __restrict__ sub_off,
                                                          const uint32_t* __restrict__ list, uint32_t n_list,
                                                          u64* keys, uint32_t* __restrict__ kcount,
                                                          uint32_t* __restrict__ kc, uint32_t* __restrict__ ov_list,
                                                          unsigned long long* ov_stats, uint32_t lo, uint32_t hi,
                                                          u64* __restrict__ hist, uint32_t hist_len,
                                                          uint32_t* max_count, unsigned long long* n_distinct,
                                                          const uint32_t* __restrict__ grp_set, uint32_t* claim,
                                                          int* err) {
    extern __shared__ __align__(16) unsigned char smem_hv[];
    u64* tk = reinterpret_cast<u64*>(smem_hv);
    uint32_t* tc = reinterpret_cast<uint32_t*>(tk + HV_SLOTS);
    uint16_t* s_slot = reinterpret_cast<uint16_t*>(tc + HV_SLOTS);  // slots claimed for this task
    __shared__ uint32_t s_used, s_fail, s_kept, s_next, s_max;
    __shared__ unsigned long long s_distinct;
    const int tid = threadIdx.x, lane = tid & 31;
    // the table starts empty once; each task resets only the slots it claimed
    for (int i = tid; i < HV_SLOTS; i += HV_NT) {
        tk[i] = HV_EMPTY;
        tc[i] = 0;
    }
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            s_next = atomicAdd(claim, 1u);
            s_used = 0;
            s_fail = 0;
            s_kept = 0;
            s_max = 0;
            s_distinct = 0;
        }
        __syncthreads();
        const uint32_t si = s_next;
        if (si >= n_list) break;
        const uint32_t s = list[si];
        const u64 base = sub_off[s], n = sub_off[s + 1] - base;
        const uint32_t set = grp_set ? grp_set[s >> 8] : 0u;
        // fold the keys into the table, HV_PF keys per thread and round loaded
        // ahead; the copies of a key within a warp are added by one lane
        // (heavy hitters repeat inside a warp's keys)
        for (u64 r0 = 0; r0 < n; r0 += (u64)HV_NT * HV_PF) {
            if (__any_sync(0xffffffffu, *(volatile uint32_t*)&s_fail != 0)) break;
            u64 kr[HV_PF];
#pragma unroll
            for (int j = 0; j < HV_PF; ++j) {
                const u64 i = r0 + (u64)j * HV_NT + tid;
                kr[j] = i < n ? keys[base + i] : HV_EMPTY;
            }
#pragma unroll
            for (int j = 0; j < HV_PF; ++j) {
                if (__any_sync(0xffffffffu, *(volatile uint32_t*)&s_fail != 0)) break;  // checked before every claim
                const u64 key = kr[j];
                const uint32_t peers = __match_any_sync(0xffffffffu, key);
                if (key == HV_EMPTY || lane != __ffs(peers) - 1) continue;
                const uint32_t copies = (uint32_t)__popc(peers);
                uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ULL) >> 50) & (HV_SLOTS - 1);  // 14 bits
                for (int probe = 0; probe < HV_SLOTS; ++probe) {
                    const u64 prev = atomicCAS(reinterpret_cast<unsigned long long*>(&tk[h]), HV_EMPTY, key);
                    if (prev == HV_EMPTY || prev == key) {
                        atomicAdd(&tc[h], copies);
                        if (prev == HV_EMPTY) {
                            const uint32_t q = atomicAdd(&s_used, 1u);
                            if (q < (uint32_t)HV_LIST) s_slot[q] = (uint16_t)h;
                            if (q + 1 > (uint32_t)HV_FILL) s_fail = 1;
                        }
                        break;
                    }
                    h = (h + 1) & (HV_SLOTS - 1);
                }
            }
        }
        __syncthreads();
        const uint32_t used = s_used < (uint32_t)HV_LIST ? s_used : (uint32_t)HV_LIST;
        const bool fail = s_fail != 0;
        // every claimed slot is one distinct k-mer of the task with its exact
        // count (or, after a failure, is only cleared)
        u64* hset = hist + (u64)set * hist_len;
        uint32_t my_max = 0;
        unsigned long long my_d = 0;
        for (uint32_t q = tid; q < used; q += HV_NT) {
            const uint32_t slot = s_slot[q];
            const uint32_t cnt = tc[slot];
            const u64 key = tk[slot];
            tk[slot] = HV_EMPTY;
            tc[slot] = 0;
            if (fail) continue;
            ++my_d;
            my_max = cnt > my_max ? cnt : my_max;
            const uint32_t b = cnt < hist_len - 1 ? cnt : hist_len - 1;
            atomicAdd(reinterpret_cast<unsigned long long*>(hset + b), 1ULL);
            if (cnt >= lo && cnt <= hi) {
                const uint32_t p = atomicAdd(&s_kept, 1u);
                keys[base + p] = key;  // the task's own range: every key is in the table already
                kcount[base + p] = cnt;
            }
        }
        if (fail) {  // too many distinct keys: the global path takes it
            if (tid == 0) {
                kc[s] = 0;
                ov_list[atomicAdd(reinterpret_cast<unsigned int*>(ov_stats), 1u)] = s;
                atomicAdd(ov_stats + 1, (unsigned long long)n);
            }
            continue;
        }
        if (my_d) atomicAdd(&s_distinct, my_d);
        if (my_max) atomicMax(&s_max, my_max);
        __syncthreads();
        if (tid == 0) {
            kc[s] = s_kept;
            if (s_distinct) atomicAdd(n_distinct + set, s_distinct);
            if (s_max) atomicMax(max_count + set, s_max);
        }
    }
}

void launch_heavy_count(const uint64_t* sub_off, const uint32_t* list, uint32_t n_list, void* keys,
                        uint32_t* kcount, uint32_t* kc, uint32_t* ov_list, uint64_t* ov_stats, uint32_t lo,
                        uint32_t hi, uint64_t* hist, uint32_t hist_len, uint32_t* max_count, uint64_t* n_distinct,
                        const uint32_t* grp_set, uint32_t* claim, int* err, int num_sms, cudaStream_t st) {
    if (n_list == 0) return;
    count_launch();
    const size_t dyn = heavy_smem_bytes();
    cudaFuncSetAttribute(k_heavy_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    const unsigned g = n_list < (uint32_t)num_sms ? n_list : (unsigned)num_sms;
    k_heavy_count<<<g, HV_NT, dyn, st>>>((const u64*)sub_off, list, n_list, (u64*)keys, kcount, kc, ov_list,
                                         (unsigned long long*)ov_stats, lo, hi, (u64*)hist, hist_len, max_count,
                                         (unsigned long long*)n_distinct, grp_set, claim, err);
}

// ---------------------------------------------------------------------------
// kept pairs -> output; listed sub-segments -> one array
// ---------------------------------------------------------------------------
// Warp w copies the kc[s] kept pairs of sub-segment s (from its range start)
// to out_keys[out_off[s] ...], for s = w, w + warps, ...  With n_groups > 0
// the offsets are digit-major: sub-segment s = group g, top digit d reads
// out_off[d * n_groups + g] (all groups' digit-0 pairs first, then digit 1,
// ...), so the output comes out partitioned by the top digit.
template <typename K>
__global__ void __launch_bounds__(256) k_compact(const u64* __restrict__ sub_off, const uint32_t* __restrict__ kc,
                                                 const u64* __restrict__ out_off, uint32_t n_sub, uint32_t n_groups,
                                                 const K* __restrict__ keys, const uint32_t* __restrict__ kcount,
                                                 K* __restrict__ out_keys, uint32_t* __restrict__ out_counts,
                                                 u64 out_cap, int* err) {
    const int lane = threadIdx.x & 31;
    const u64 nwarps = (u64)gridDim.x * 8;
    for (u64 s = (u64)blockIdx.x * 8 + (threadIdx.x >> 5); s < n_sub; s += nwarps) {
        const uint32_t n = kc[s];
        if (!n) continue;
        const u64 src = sub_off[s], dst = n_groups ? out_off[(s & 255) * n_groups + (s >> 8)] : out_off[s];
        if (dst + n > out_cap) {
            if (lane == 0) raise_error(err, HSK_DERR_BOUNDS);
            continue;
        }
        for (uint32_t i = lane; i < n; i += 32) {
            out_keys[dst + i] = keys[src + i];
            out_counts[dst + i] = kcount[src + i];
        }
    }
}

void launch_compact(const uint64_t* sub_off, const uint32_t* kc, const uint64_t* out_off, uint32_t n_sub,
                    uint32_t n_groups, int key_words, const void* keys, const uint32_t* kcount, void* out_keys,
                    uint32_t* out_counts, uint64_t out_cap, int* err, int grid, cudaStream_t st) {
    if (n_sub == 0) return;
    count_launch();
    uint64_t want = ((uint64_t)n_sub + 7) / 8;
    unsigned g = (unsigned)(want < (uint64_t)grid ? want : (uint64_t)grid);
    if (key_words == 1)
        k_compact<u64><<<g, 256, 0, st>>>((const u64*)sub_off, kc, (const u64*)out_off, n_sub, n_groups,
                                          (const u64*)keys, kcount, (u64*)out_keys, out_counts, out_cap, err);
    else
        k_compact<key128><<<g, 256, 0, st>>>((const u64*)sub_off, kc, (const u64*)out_off, n_sub, n_groups,
                                             (const key128*)keys, kcount, (key128*)out_keys, out_counts, out_cap,
                                             err);
}

// kc_t[d * n_groups + g] = kc[g * 256 + d]: the kept counts in digit-major order
__global__ void __launch_bounds__(256) k_transpose_kc(const uint32_t* __restrict__ kc, uint32_t n_groups,
                                                      uint32_t* __restrict__ kc_t) {
    const u64 n = (u64)n_groups * 256;
    for (u64 s = (u64)blockIdx.x * 256 + threadIdx.x; s < n; s += (u64)gridDim.x * 256)
        kc_t[(s & 255) * n_groups + (s >> 8)] = kc[s];
}

void launch_transpose_kc(const uint32_t* kc, uint32_t n_groups, uint32_t* kc_t, int grid, cudaStream_t st) {
    if (n_groups == 0) return;
    count_launch();
    const u64 n = (u64)n_groups * 256;
    const unsigned g = (unsigned)((n + 255) / 256 < (u64)grid ? (n + 255) / 256 : (u64)grid);
    k_transpose_kc<<<g, 256, 0, st>>>(kc, n_groups, kc_t);
}

// One CTA: ov_pre[j] = sum of the sizes of listed sub-segments before j.
__global__ void __launch_bounds__(256) k_ov_prefix(const u64* __restrict__ sub_off, const uint32_t* __restrict__ ov_list,
                                                   uint32_t n_ov, u64* __restrict__ ov_pre) {
    __shared__ u64 s_scr[9];
    u64 carry = 0;
    for (uint32_t j0 = 0; j0 < n_ov; j0 += 256) {
        const uint32_t j = j0 + threadIdx.x;
        u64 v = 0;
        if (j < n_ov) {
            const uint32_t s = ov_list[j];
            v = sub_off[s + 1] - sub_off[s];
        }
        u64 total;
        const u64 e = block_excl_sum<256, u64>(v, s_scr, total);
        if (j < n_ov) ov_pre[j] = carry + e;
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) ov_pre[n_ov] = carry;
}

// CTA j (stride gridDim.x) copies listed sub-segment j to dst[ov_pre[j] ...].
template <typename K>
__global__ void __launch_bounds__(256) k_ov_gather(const u64* __restrict__ sub_off, const uint32_t* __restrict__ ov_list,
                                                   uint32_t n_ov, const u64* __restrict__ ov_pre,
                                                   const K* __restrict__ keys, K* __restrict__ dst, u64 dst_cap,
                                                   int* err) {
    for (uint32_t j = blockIdx.x; j < n_ov; j += gridDim.x) {
        const uint32_t s = ov_list[j];
        const u64 src = sub_off[s], n = sub_off[s + 1] - src, o = ov_pre[j];
        if (o + n > dst_cap) {
            if (threadIdx.x == 0) raise_error(err, HSK_DERR_BOUNDS);
            continue;
        }
        for (u64 i = threadIdx.x; i < n; i += 256) dst[o + i] = keys[src + i];
    }
}

void launch_ov_gather(const uint64_t* sub_off, const uint32_t* ov_list, uint32_t n_ov, uint64_t* ov_pre,
                      int key_words, const void* keys, void* dst, uint64_t dst_cap, int* err, int grid,
                      cudaStream_t st) {
    if (n_ov == 0) return;
    count_launch(2);
    k_ov_prefix<<<1, 256, 0, st>>>((const u64*)sub_off, ov_list, n_ov, (u64*)ov_pre);
    unsigned g = n_ov < (uint32_t)grid ? n_ov : (unsigned)grid;
    if (key_words == 1)
        k_ov_gather<u64><<<g, 256, 0, st>>>((const u64*)sub_off, ov_list, n_ov, (const u64*)ov_pre,
                                            (const u64*)keys, (u64*)dst, dst_cap, err);
    else
        k_ov_gather<key128><<<g, 256, 0, st>>>((const u64*)sub_off, ov_list, n_ov, (const u64*)ov_pre,
                                               (const key128*)keys, (key128*)dst, dst_cap, err);
}

}  // namespace hsk
