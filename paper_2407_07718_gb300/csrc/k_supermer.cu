// k_supermer.cu -- stages S2 and S3: canonical k-mers, hash-scored minimizers
// and supermers scattered into minimizer-hashed buckets.
//
// Sec. 3.2: every m-mer is scored by a hash (MurmurHash3's 32-bit finalizer
// of the canonical m-mer folded to 32 bits, XOR a seed); a k-mer's minimizer
// is its lowest-scoring m-mer, and the same hash value decides the k-mer's
// target: bucket = score mod B (B a power of two).  Sec. 2.4: consecutive
// k-mers with the same target form a supermer whose overlapping bases are
// stored once.  Sec. 3.4: the buckets are the paper's tasks -- a k-mer value
// never lands in two of them, because canonical m-mers give a k-mer and its
// reverse complement the same minimizer score.
//
// GPU design (replaces the paper's per-read monotone deque): a warp walks a
// tile of 1024 consecutive window starts in 32 steps, lane l handling window
// 32*s + l.  The packed bases and masks of the tile are staged in shared
// memory with 128-bit loads.  Each lane computes one new m-mer score per step;
// the window minimum over w = k-m+1 scores comes from minima over 32-lane
// blocks kept in registers: for w <= 33 the minima of runs of D = 2^L <= w
// scores (doubling with shuffles, each block's computed once and carried to
// the next step), for w > 33 suffix and prefix minima of the blocks (van
// Herk / Gil-Werman with 32-lane blocks).  Supermer
// cuts (bucket change, invalid window, cap of nmax k-mers, tile end) come
// from ballots of run starts (the latest start at or before a lane is the
// highest set bit below it).  The walk runs once (DESC): every
// supermer becomes an 8-byte descriptor (start base, k-mer count, bucket),
// buffered per warp in shared memory and appended to a global list with one
// atomic per buffer; per-bucket record and k-mer counts are kept in shared
// memory.  A second, light kernel scatters records into their buckets from
// the descriptors.  DUMP mode writes per-window keys and scores for the stage
// test.
#include "hsk_device.cuh"

namespace hsk {

constexpr int SM_WARPS = SM_CTA_WARPS;
constexpr int SM_STEPS = 32;
constexpr int SM_TW = 32 * SM_STEPS;      // windows per warp tile
constexpr int SM_PW = SM_TW / 32 + 6;     // packed words staged per warp (even)
constexpr int SM_MW = SM_TW / 64 + 4;     // mask words staged per warp (even)
constexpr int SM_DBUF = 128;              // descriptors buffered per warp
constexpr int SM_VW = SM_TW / 64;         // valid-window words per warp
static_assert(SM_TW == (int)SM_TILE_BASES, "tile size");
static_assert(SM_PW * 32 <= (int)SM_TILE_REACH && SM_MW * 64 <= (int)SM_TILE_REACH,
              "a tile's staged words must lie within its declared reach");

// The bucket table sets the walk's shared memory, so it differs from call to
// call.  Serving slots launch the walk from several host threads at once, and
// the per-kernel opt-in limit is process-wide: every thread sets it to the
// size of the largest table (SM_MAX_BUCKETS buckets), never to its own, so
// one thread cannot lower it under another's launch.
constexpr uint32_t SM_MAX_BUCKETS = 8192;
size_t supermer_smem_bytes(int mode, uint32_t n_buckets) {
    size_t s = (size_t)SM_WARPS * (SM_PW + 2 * SM_MW + SM_VW) * sizeof(u64);
    if (mode == SM_DESC) s += (size_t)SM_WARPS * SM_DBUF * sizeof(u64) + (size_t)n_buckets * 2 * sizeof(uint32_t);
    return s;
}

// MurmurHash3's 32-bit finalizer (A. Appleby, public domain).
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// Score of the m-mer at local base q of the staged words.  Hash order (the
// paper's choice, Sec. 3.2): MurmurHash3's finalizer of the canonical m-mer.
// Lexical order (the alternative the paper compares against): the canonical
// m-mer's code itself -- its top 32 bits when m > 16, so that the score stays
// 32-bit (m-mers sharing their first 16 bases then tie, which only groups them
// in one bucket).  Either way the score is a function of the canonical m-mer,
// so a k-mer and its reverse complement share their minimizer and bucket.
template <bool LEX>
__device__ __forceinline__ uint32_t mmer_score(const u64* pk, int q, int m, uint32_t seed) {
    u64 f = extract_k64(pk, (u64)q, m);
    u64 r = revcomp64(f, m);
    u64 c = f < r ? f : r;
    if constexpr (LEX) return m > 16 ? (uint32_t)(c >> (2 * m - 32)) : (uint32_t)c;
    else return fmix32((uint32_t)c ^ (uint32_t)(c >> 32) ^ seed);
}

// Minimum of v over lanes [lane, 31] (suffix) and over [0, lane] (prefix).
__device__ __forceinline__ uint32_t lane_suffix_min(uint32_t v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_down_sync(0xffffffffu, v, d);
        if (lane + d < 32) v = min(v, o);
    }
    return v;
}
__device__ __forceinline__ uint32_t lane_prefix_min(uint32_t v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v = min(v, o);
    }
    return v;
}

// min(v[lane .. lane + 2^L - 1]) within the block (lanes past 31 ignored).
__device__ __forceinline__ uint32_t lane_range_min_trunc(uint32_t v, int L, int lane) {
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        if (j < L) {
            const uint32_t o = __shfl_down_sync(0xffffffffu, v, 1 << j);
            if (lane + (1 << j) < 32) v = min(v, o);
        }
    }
    return v;
}
// min(v[0 .. lane]) for lanes below n (n <= 32; other lanes: partial).
__device__ __forceinline__ uint32_t lane_prefix_min_upto(uint32_t v, int n, int lane) {
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        if ((1 << j) < n) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, v, 1 << j);
            if (lane >= (1 << j)) v = min(v, o);
        }
    }
    return v;
}

// Window minimum for 33 <= w <= 65 (three score registers): a window that
// starts at lane l of block 0 always runs past the block's end, so it is the
// suffix of block 0 from l, then either a prefix of block 1 or all of block
// 1 and a prefix of block 2 (van Herk / Gil-Werman with 32-lane blocks).
// sm0 = suffix minima of block 0, pm1 / pm2 = prefix minima of blocks 1 / 2.
__device__ __forceinline__ uint32_t window_min_wide(uint32_t sm0, uint32_t pm1, uint32_t pm2, int w, int lane) {
    const int e = lane + w - 1;  // last position of the window, 32 <= e <= 95
    const uint32_t a = __shfl_sync(0xffffffffu, pm1, (e - 32) & 31);
    const uint32_t b = __shfl_sync(0xffffffffu, pm2, (e - 64) & 31);
    const uint32_t full1 = __shfl_sync(0xffffffffu, pm1, 31);
    return min(sm0, e < 64 ? a : min(full1, b));
}

// Bit t (most significant first) = OR of bits [t, t + L) of the 128-bit
// value a:b, for t = 0..63 and 1 <= L <= 64: OR over windows of doubling
// width, then two overlapping windows of that width.
__device__ __forceinline__ u64 window_or64(u64 a, u64 b, int L) {
    u64 hi = a, lo = b;
    int width = 1;
    while (2 * width <= L) {
        hi |= (hi << width) | (lo >> (64 - width));
        lo |= lo << width;
        width *= 2;
    }
    const int d = L - width;  // 0 <= d < width
    return d ? hi | (hi << d) | (lo >> (64 - d)) : hi;
}

// Bits [2*nb, 64) of word x cleared when the record holds only nb (< 32) more bases.
__device__ __forceinline__ u64 keep_bases(u64 x, int nb) {
    if (nb >= 32) return x;
    if (nb <= 0) return 0;
    return x & (~0ULL << (64 - 2 * nb));
}

// Descriptor of a supermer: start base (40 bits), k-mers (8 bits), bucket (16 bits).
__device__ __forceinline__ u64 make_desc(u64 pos, uint32_t n, uint32_t b) {
    return pos | ((u64)n << 40) | ((u64)b << 48);
}

template <int MODE, bool WIDE, int NREG, bool LEX>
__global__ void __launch_bounds__(SM_WARPS * 32) k_supermer(const SmParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    u64* s_pk = reinterpret_cast<u64*>(smem);
    u64* s_iv = s_pk + SM_WARPS * SM_PW;
    u64* s_rs = s_iv + SM_WARPS * SM_MW;
    u64* s_val = s_rs + SM_WARPS * SM_MW;
    u64* s_desc = s_val + SM_WARPS * SM_VW;                                      // DESC
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(s_desc + SM_WARPS * SM_DBUF);  // DESC
    uint32_t* s_km = s_cnt + P.n_buckets;                                        // DESC

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t B = P.n_buckets;
    const int k = P.k, m = P.m, w = P.w, nmax = P.nmax;

    if (MODE == SM_DESC) {
        for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) s_cnt[b] = s_km[b] = 0;
        __syncthreads();
    }

    u64* wpk = s_pk + warp * SM_PW;
    u64* wiv = s_iv + warp * SM_MW;
    u64* wrs = s_rs + warp * SM_MW;
    u64* wval = s_val + warp * SM_VW;
    u64* wdesc = s_desc + warp * SM_DBUF;
    int nbuf = 0;  // descriptors buffered by this warp (warp-uniform)
    const u64 n_tiles = P.tile_end ? P.tile_end : (P.n_bases + SM_TW - 1) / SM_TW;

    // append the buffered descriptors to the global list (one atomic per flush)
    auto flush = [&]() {
        if (nbuf == 0) return;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(P.desc_count, (unsigned long long)nbuf);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (int i = lane; i < nbuf; i += 32)
            if (base + i < P.desc_cap) P.desc[base + i] = wdesc[i];
        __syncwarp();
        nbuf = 0;
    };

    for (u64 t = P.tile_begin + (u64)blockIdx.x * SM_WARPS + warp; t < n_tiles; t += (u64)gridDim.x * SM_WARPS) {
        const u64 p0 = t * SM_TW;
        // buckets of the tile's set (packed sets: the set holding tile t)
        uint32_t bbase = 0, bmask = B - 1u;
        if (P.n_sets) {
            uint32_t lo = 0, hi = P.n_sets;  // set_tile0[lo] <= t < set_tile0[hi]
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if ((u64)P.set_tile0[mid] <= t) lo = mid;
                else hi = mid;
            }
            bbase = P.set_bucket[lo];
            bmask = P.set_bmask[lo];
        }
        // ---- stage packed bases and masks (128-bit loads; p0 is 1024-aligned)
        {
            const u64 pw0 = p0 >> 5, mw0 = p0 >> 6;
            for (int i = lane; i < SM_PW / 2; i += 32) {
                u64 g = pw0 + 2 * i;
                ulonglong2 v = make_ulonglong2(0, 0);
                if (g + 1 < P.n_packed_words) v = *reinterpret_cast<const ulonglong2*>(P.packed + g);
                else if (g < P.n_packed_words) v.x = P.packed[g];
                wpk[2 * i] = v.x;
                wpk[2 * i + 1] = v.y;
            }
            for (int i = lane; i < SM_MW / 2; i += 32) {
                u64 g = mw0 + 2 * i;
                ulonglong2 a = make_ulonglong2(~0ULL, ~0ULL), b = make_ulonglong2(0, 0);
                if (g + 1 < P.n_mask_words) {
                    a = *reinterpret_cast<const ulonglong2*>(P.invalid + g);
                    b = *reinterpret_cast<const ulonglong2*>(P.start + g);
                } else if (g < P.n_mask_words) {
                    a.x = P.invalid[g];
                    b.x = P.start[g];
                }
                wiv[2 * i] = a.x;
                wiv[2 * i + 1] = a.y;
                wrs[2 * i] = b.x;
                wrs[2 * i + 1] = b.y;
            }
            __syncwarp();
            // window starts of the tile whose k bases are all valid and in one
            // read: no invalid base in [p, p+k), no read start in (p, p+k)
            if (lane < SM_TW / 64) {
                const int o = lane;
                u64 bad = window_or64(wiv[o], wiv[o + 1], k);
                if (k > 1) {
                    const u64 a = (wrs[o] << 1) | (wrs[o + 1] >> 63);
                    const u64 b = (wrs[o + 1] << 1) | (wrs[o + 2] >> 63);
                    bad |= window_or64(a, b, k - 1);
                }
                wval[o] = ~bad;
            }
            __syncwarp();
        }

        // rolling m-mer scores: X[r] = score at local base 32*(s + r) + lane
        uint32_t X[NREG];
#pragma unroll
        for (int r = 0; r < NREG; ++r) X[r] = mmer_score<LEX>(wpk, 32 * r + lane, m, P.seed32);
        // wide windows (three registers): prefix minima of block 1, carried
        // from one step to the next as block 2's
        uint32_t pm_next = 0;
        if constexpr (NREG == 3) pm_next = lane_prefix_min(X[1], lane);
        // narrow windows (two registers, w <= 33): with D = 2^L <= w < 2D, a
        // window is two overlapping runs of D scores.  t_cur = min over runs
        // of D starting at each lane of block 0, counted within the block
        // only; computed for each block when it enters as block 1, carried.
        int nL = 0;
        while ((2 << nL) <= w) ++nL;
        const int nD = 1 << nL;
        uint32_t t_cur = 0;
        if constexpr (NREG == 2) t_cur = lane_range_min_trunc(X[0], nL, lane);

        int c_valid = 0, c_runstart = -1;   // carry from lane 31 of the previous step
        uint32_t c_b = 0;
        int pv = 0, plp = 0, psm = 0;       // previous step, for delayed emission
        uint32_t pb = 0, pvmask = 0, psmask = 0;

        // emit the supermers that end in the previous step (end = valid and the
        // next window is invalid or starts a new supermer)
        auto emit_prev = [&](int nv, int ns) {
            const bool end = pv && (!nv || ns);
            const uint32_t ends = __ballot_sync(0xffffffffu, end);
            if (!ends) return;
            const int cnt = __popc(ends);
            if (nbuf + cnt > SM_DBUF) flush();
            if (end) {
                const int n = plp - psm + 1;
                atomicAdd(&s_cnt[pb], 1u);
                atomicAdd(&s_km[pb], (uint32_t)n);
                wdesc[nbuf + __popc(ends & ((1u << lane) - 1u))] = make_desc(p0 + psm, (uint32_t)n, pb);
            }
            nbuf += cnt;
            __syncwarp();
        };

        for (int s = 0; s < SM_STEPS; ++s) {
            const int lp = 32 * s + lane;
            const u64 p = p0 + lp;
            int valid = (p + k <= P.n_bases) && ((wval[lp >> 6] >> (63 - (lp & 63))) & 1);
            uint32_t mh;
            if constexpr (NREG == 3) {
                const uint32_t pm2 = lane_prefix_min(X[2], lane);
                mh = window_min_wide(lane_suffix_min(X[0], lane), pm_next, pm2, w, lane);
                pm_next = pm2;
            } else {
                // block 1's runs within block 1, and its prefix minima that
                // complete block 0's runs reaching into it (lanes past 32 - D)
                const uint32_t t_new = lane_range_min_trunc(X[1], nL, lane);
                const uint32_t pm1 = lane_prefix_min_upto(X[1], nD - 1, lane);
                const int i1 = lane + nD - 33;  // last lane of block 1 in this lane's run
                const uint32_t pv = __shfl_sync(0xffffffffu, pm1, i1 & 31);
                const uint32_t tc = i1 >= 0 ? min(t_cur, pv) : t_cur;
                // the second run starts at q = lane + w - D (in block 1 when q >= 32,
                // where its run lies inside block 1 because w <= 33)
                const int q = lane + w - nD;
                const uint32_t a = __shfl_sync(0xffffffffu, tc, q & 31);
                const uint32_t b = __shfl_sync(0xffffffffu, t_new, (q - 32) & 31);
                mh = min(tc, q < 32 ? a : b);
                t_cur = t_new;
            }
            const uint32_t b = bbase + (mh & bmask);

            if (MODE == SM_DUMP) {
                if (p < P.n_bases) {
                    P.dump_valid[p] = (uint8_t)valid;
                    if (valid) {
                        if (!WIDE) {
                            P.dump_key[2 * p] = canonical64(extract_k64(wpk, lp, k), k);
                            P.dump_key[2 * p + 1] = 0;
                        } else {
                            key128 c = canonical128(extract_k128(wpk, lp, k), k);
                            P.dump_key[2 * p] = c.lo;
                            P.dump_key[2 * p + 1] = c.hi;
                        }
                        P.dump_minhash[p] = mh;
                    }
                }
            } else {
                // flags of neighbouring lanes come from ballots; only the
                // bucket of the lane before needs a shuffle
                const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
                uint32_t prev_b = __shfl_up_sync(0xffffffffu, b, 1);
                int prev_valid = lane ? (int)((vmask >> (lane - 1)) & 1u) : c_valid;
                if (lane == 0) prev_b = c_b;
                const int start0 = valid && !(prev_valid && prev_b == b);
                // the latest run start at or before this window
                const uint32_t smask0 = __ballot_sync(0xffffffffu, start0);
                const uint32_t le = smask0 & (0xFFFFFFFFu >> (31 - lane));
                const int rs = le ? 32 * s + (31 - __clz(le)) : c_runstart;
                const int pos_in_run = lp - rs;
                // pos_in_run / nmax by a multiply: exact for pos_in_run < 2^24
                const int q = (int)__umulhi((uint32_t)pos_in_run, P.nmax_magic);
                const int start = valid && (start0 || pos_in_run == q * nmax);
                const int smstart = rs + q * nmax;
                const uint32_t smask = __ballot_sync(0xffffffffu, start);
                if (s > 0) {
                    // the window after this lane's window of the previous step
                    const int nv = lane < 31 ? (int)((pvmask >> (lane + 1)) & 1u) : (int)(vmask & 1u);
                    const int ns = lane < 31 ? (int)((psmask >> (lane + 1)) & 1u) : (int)(smask & 1u);
                    emit_prev(nv, ns);
                }
                c_valid = (int)(vmask >> 31);
                c_b = __shfl_sync(0xffffffffu, b, 31);
                if (smask0) c_runstart = 32 * s + (31 - __clz(smask0));
                pv = valid;
                pvmask = vmask;
                psmask = smask;
                pb = b;
                plp = lp;
                psm = smstart;
            }
            // roll the scores forward by one step
#pragma unroll
            for (int r = 0; r + 1 < NREG; ++r) X[r] = X[r + 1];
            X[NREG - 1] = mmer_score<LEX>(wpk, 32 * (s + NREG) + lane, m, P.seed32);
        }
        if (MODE != SM_DUMP) {  // the tile edge ends every open supermer
            const int nv = lane < 31 ? (int)((pvmask >> (lane + 1)) & 1u) : 0;
            const int ns = lane < 31 ? (int)((psmask >> (lane + 1)) & 1u) : 0;
            emit_prev(nv, ns);
        }
        __syncwarp();
    }

    if (MODE == SM_DESC) {
        flush();
        __syncthreads();
        for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) {
            if (s_cnt[b]) atomicAdd(P.bucket_rec + b, s_cnt[b]);
            if (s_km[b]) atomicAdd(reinterpret_cast<unsigned long long*>(P.bucket_kmers + b),
                                   (unsigned long long)s_km[b]);
        }
    }
}

template <int MODE>
static void launch_mode(const SmParams& p, cudaStream_t st) {
    size_t sm = supermer_smem_bytes(MODE, p.n_buckets);
    const size_t sm_cap = supermer_smem_bytes(MODE, SM_MAX_BUCKETS);
    bool wide = p.k > 32;
    int nreg = (p.w <= 33) ? 2 : 3;
    unsigned grid = p.grid;
    count_launch();
#define HSK_SM_LAUNCH(W, NR)                                                                 \
    do {                                                                                     \
        auto fn = p.lexical ? k_supermer<MODE, W, NR, true> : k_supermer<MODE, W, NR, false>; \
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_cap);  \
        fn<<<grid, SM_WARPS * 32, sm, st>>>(p);                                              \
    } while (0)
    if (!wide && nreg == 2) HSK_SM_LAUNCH(false, 2);
    else if (!wide) HSK_SM_LAUNCH(false, 3);
    else if (nreg == 2) HSK_SM_LAUNCH(true, 2);
    else HSK_SM_LAUNCH(true, 3);
#undef HSK_SM_LAUNCH
}

void launch_supermer(int mode, const SmParams& p, cudaStream_t st) {
    if (p.n_bases == 0) return;
    if (mode == SM_DESC) launch_mode<SM_DESC>(p, st);
    else launch_mode<SM_DUMP>(p, st);
}

int supermer_max_ctas_per_sm(int mode, bool wide, int nreg, uint32_t n_buckets) {
    size_t sm = supermer_smem_bytes(mode, n_buckets);
    int n = 0;
    const void* fn = wide ? (nreg == 2 ? (const void*)k_supermer<SM_DESC, true, 2, false>
                                       : (const void*)k_supermer<SM_DESC, true, 3, false>)
                          : (nreg == 2 ? (const void*)k_supermer<SM_DESC, false, 2, false>
                                       : (const void*)k_supermer<SM_DESC, false, 3, false>);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)supermer_smem_bytes(mode, SM_MAX_BUCKETS));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, SM_WARPS * 32, sm) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
}

// ---------------------------------------------------------------------------
// records from descriptors
// ---------------------------------------------------------------------------
// A slot in the supermer's bucket from the bucket's cursor, the record's
// bases gathered from the packed reads (the descriptors of a warp come from
// one tile, so these reads hit L1/L2).  The kernel waits on memory: each
// thread takes SD descriptors at a time and issues their loads and cursor
// atomics together (SD = 4: long-read S3 5.35 -> 4.40 ms; 8 was slower).
template <bool WIDE>
__global__ void __launch_bounds__(256) k_scatter_desc(const u64* __restrict__ desc, u64 n_desc,
                                                      const u64* __restrict__ packed, int k,
                                                      const u64* __restrict__ bucket_off, uint32_t* cursor,
                                                      u64* __restrict__ records, u64 n_records, int* err) {
    constexpr int SD = 4;
    const u64 stride = (u64)gridDim.x * blockDim.x * SD;
    for (u64 i0 = (u64)blockIdx.x * blockDim.x * SD + threadIdx.x; i0 < n_desc; i0 += stride) {
        u64 dd[SD], slot[SD];
#pragma unroll
        for (int j = 0; j < SD; ++j) {
            const u64 i = i0 + (u64)j * blockDim.x;
            dd[j] = i < n_desc ? desc[i] : ~0ULL;
        }
#pragma unroll
        for (int j = 0; j < SD; ++j) {
            slot[j] = ~0ULL;
            if (dd[j] != ~0ULL) {
                const uint32_t b = (uint32_t)(dd[j] >> 48);
                slot[j] = bucket_off[b] + atomicAdd(cursor + (size_t)b * SCATTER_CURSOR_STRIDE, 1u);
            }
        }
#pragma unroll
        for (int j = 0; j < SD; ++j) {
            if (dd[j] == ~0ULL) continue;
            const u64 d = dd[j];
            const u64 pos = d & ((1ULL << 40) - 1);
            const uint32_t n = (uint32_t)(d >> 40) & 0xFF, b = (uint32_t)(d >> 48);
            if (slot[j] >= n_records || slot[j] >= bucket_off[b + 1]) {
                raise_error(err, HSK_DERR_BOUNDS);
                continue;
            }
            const int nb = (int)n + k - 1;  // bases in the record
            if (!WIDE) {
                u64 a = keep_bases(extract_k64(packed, pos, 32), nb);
                u64 c = keep_bases(extract_k64(packed, pos + 32, 32), nb - 32) | (u64)n;
                reinterpret_cast<ulonglong2*>(records)[slot[j]] = make_ulonglong2(a, c);
            } else {
                u64 r[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) r[q] = keep_bases(extract_k64(packed, pos + 32 * q, 32), nb - 32 * q);
                r[3] |= (u64)n;
                ulonglong2* dst = reinterpret_cast<ulonglong2*>(records) + 2 * slot[j];
                dst[0] = make_ulonglong2(r[0], r[1]);
                dst[1] = make_ulonglong2(r[2], r[3]);
            }
        }
    }
}

void launch_scatter_desc(const uint64_t* desc, uint64_t n_desc, const uint64_t* packed, int k,
                         const uint64_t* bucket_off, uint32_t* cursor, uint64_t* records, uint64_t n_records,
                         int* err, int grid, cudaStream_t st) {
    if (n_desc == 0) return;
    count_launch();
    uint64_t need = (n_desc + 4 * 256 - 1) / (4 * 256);  // four descriptors a thread
    unsigned g = (unsigned)(need < (uint64_t)grid ? need : (uint64_t)grid);
    if (k <= 32)
        k_scatter_desc<false><<<g, 256, 0, st>>>((const u64*)desc, n_desc, (const u64*)packed, k,
                                                 (const u64*)bucket_off, cursor, (u64*)records, n_records, err);
    else
        k_scatter_desc<true><<<g, 256, 0, st>>>((const u64*)desc, n_desc, (const u64*)packed, k,
                                                (const u64*)bucket_off, cursor, (u64*)records, n_records, err);
}

// ---------------------------------------------------------------------------
// exclusive scan of uint32 counts -> uint64 offsets (decoupled look-back)
// ---------------------------------------------------------------------------
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = 256 * SCAN_ITEMS;

uint64_t scan_status_words(uint64_t n) { return ((n + SCAN_TILE - 1) / SCAN_TILE + 1) * LB_PAD; }

__global__ void __launch_bounds__(256) k_scan_u32(const uint32_t* __restrict__ in, uint64_t n,
                                                  u64* __restrict__ out, u64* status,
                                                  uint32_t* tile_ctr, uint32_t epoch, int* err) {
    __shared__ uint32_t s_tile;
    __shared__ u64 s_scr[9];
    __shared__ u64 s_prefix;
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const u64 tile = s_tile;
    const u64 base = tile * SCAN_TILE + (u64)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    u64 sum = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = base + i < n ? in[base + i] : 0u;
        sum += v[i];
    }
    u64 total;
    u64 excl = block_excl_sum<256, u64>(sum, s_scr, total);
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
    }
    __syncthreads();
    u64 run = s_prefix + excl;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (base < n && base + SCAN_ITEMS >= n) out[n] = run;  // total
}

void launch_scan_u32(const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* status,
                     uint32_t* tile_ctr, uint32_t epoch, int* err, cudaStream_t st) {
    if (n == 0) {
        cudaMemsetAsync(out, 0, sizeof(uint64_t), st);
        return;
    }
    uint64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    count_launch();
    k_scan_u32<<<(unsigned)tiles, 256, 0, st>>>(in, n, (u64*)out, (u64*)status, tile_ctr, epoch, err);
}

}  // namespace hsk
