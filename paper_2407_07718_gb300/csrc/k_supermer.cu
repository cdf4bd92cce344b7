// k_supermer.cu -- stages S2 and S3: canonical k-mers, hash-scored minimizers
// and supermers scattered into minimizer-hashed buckets.
//
// Sec. 3.2: every m-mer is scored by a hash (here MurmurHash3's fmix64 of the
// canonical m-mer XOR a seed); a k-mer's minimizer is its lowest-scoring
// m-mer, and the same hash value decides the k-mer's target: bucket
// score mod B (B a power of two).  Sec. 2.4: consecutive k-mers with the same target
// form a supermer whose overlapping bases are stored once.  Sec. 3.4: the
// buckets are the paper's tasks -- a k-mer value never lands in two of them,
// because canonical m-mers give a k-mer and its reverse complement the same
// minimizer score.
//
// GPU design (replaces the paper's per-read monotone deque): a warp walks a
// tile of 1024 consecutive window starts in 32 steps, lane l handling window
// 32*s + l.  The packed bases and masks of the tile are staged in shared
// memory with 128-bit loads.  Each lane computes one new m-mer score per step;
// the window minimum over w = k-m+1 scores comes from a log-step doubling of
// minima across lanes with shuffles (a sparse table in registers).  Supermer
// cuts (bucket change, invalid window, cap of nmax k-mers, tile end) come
// from a warp max-scan of run starts.  The same walk runs three times:
// COUNT (records per bucket and CTA, k-mers per bucket), SCATTER (write
// records at scanned offsets; per-CTA shared-memory cursors, no global
// atomics) and DUMP (per-window key and score, for the stage test).
#include "hsk_device.cuh"

namespace hsk {

constexpr int SM_WARPS = 8;
constexpr int SM_STEPS = 32;
constexpr int SM_TW = 32 * SM_STEPS;      // windows per warp tile
constexpr int SM_PW = SM_TW / 32 + 6;     // packed words staged per warp (even)
constexpr int SM_MW = SM_TW / 64 + 4;     // mask words staged per warp (even)

size_t supermer_smem_bytes(int mode, uint32_t n_buckets) {
    size_t s = (size_t)SM_WARPS * (SM_PW + 2 * SM_MW) * sizeof(u64);
    if (mode == SM_COUNT) s += (size_t)n_buckets * 2 * sizeof(uint32_t);
    if (mode == SM_SCATTER) s += (size_t)n_buckets * (sizeof(u64) + sizeof(uint32_t));
    return s;
}

// Score of the m-mer at local base q of the staged words.
__device__ __forceinline__ u64 mmer_score(const u64* pk, int q, int m, u64 seed) {
    u64 f = extract_k64(pk, (u64)q, m);
    u64 r = revcomp64(f, m);
    return fmix64((f < r ? f : r) ^ seed);
}

// Value at index lane + d (0 <= d < 32) of the 32*NREG-long sequence held as
// A[0..NREG) (A[r] holds indices 32r .. 32r+31), starting from register r.
template <int NREG>
__device__ __forceinline__ u64 seq_at(const u64 (&A)[NREG], int r, int d, int lane) {
    int src = (lane + d) & 31;
    u64 a = __shfl_sync(0xffffffffu, A[r], src);
    u64 b = ~0ULL;
    if (r + 1 < NREG) b = __shfl_sync(0xffffffffu, A[r + 1], src);
    return lane + d < 32 ? a : b;
}

// min(X[lane .. lane + w - 1]) with X given as NREG registers, w <= 32*NREG - 31.
template <int NREG>
__device__ __forceinline__ u64 window_min(const u64 (&X)[NREG], int w, int lane) {
    u64 A[NREG];
#pragma unroll
    for (int r = 0; r < NREG; ++r) A[r] = X[r];
    int width = 1;
    while (2 * width <= w) {
        if (width == 32) {
#pragma unroll
            for (int r = 0; r < NREG; ++r) {
                u64 nx = r + 1 < NREG ? A[r + 1] : ~0ULL;
                A[r] = A[r] < nx ? A[r] : nx;
            }
        } else {
            u64 nx[NREG];
#pragma unroll
            for (int r = 0; r < NREG; ++r) nx[r] = seq_at<NREG>(A, r, width, lane);
#pragma unroll
            for (int r = 0; r < NREG; ++r) A[r] = A[r] < nx[r] ? A[r] : nx[r];
        }
        width *= 2;
    }
    int d = w - width;  // 0 <= d < width <= 32 (d < 32 because w <= 64)
    u64 o = d == 0 ? A[0] : seq_at<NREG>(A, 0, d, lane);
    return A[0] < o ? A[0] : o;
}

__device__ __forceinline__ int warp_incl_max(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v = v > o ? v : o;
    }
    return v;
}

// Bits [2*nb, 64) of word x cleared when the record holds only nb (< 32) more bases.
__device__ __forceinline__ u64 keep_bases(u64 x, int nb) {
    if (nb >= 32) return x;
    if (nb <= 0) return 0;
    return x & (~0ULL << (64 - 2 * nb));
}

template <int MODE, bool WIDE, int NREG>
__global__ void __launch_bounds__(256) k_supermer(const SmParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    u64* s_pk = reinterpret_cast<u64*>(smem);
    u64* s_iv = s_pk + SM_WARPS * SM_PW;
    u64* s_rs = s_iv + SM_WARPS * SM_MW;
    unsigned char* s_b = reinterpret_cast<unsigned char*>(s_rs + SM_WARPS * SM_MW);
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(s_b);           // COUNT
    uint32_t* s_km = s_cnt + P.n_buckets;                          // COUNT
    u64* s_base = reinterpret_cast<u64*>(s_b);                     // SCATTER
    uint32_t* s_cur = reinterpret_cast<uint32_t*>(s_base + P.n_buckets);  // SCATTER

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t B = P.n_buckets;
    const int k = P.k, m = P.m, w = P.w, nmax = P.nmax;

    if (MODE == SM_COUNT) {
        for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) s_cnt[b] = s_km[b] = 0;
    } else if (MODE == SM_SCATTER) {
        for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) {
            s_base[b] = P.cta_off[(u64)b * P.grid + blockIdx.x];
            s_cur[b] = 0;
        }
    }
    __syncthreads();

    u64* wpk = s_pk + warp * SM_PW;
    u64* wiv = s_iv + warp * SM_MW;
    u64* wrs = s_rs + warp * SM_MW;
    const u64 n_tiles = (P.n_bases + SM_TW - 1) / SM_TW;

    for (u64 t = (u64)blockIdx.x * SM_WARPS + warp; t < n_tiles; t += (u64)gridDim.x * SM_WARPS) {
        const u64 p0 = t * SM_TW;
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
        }

        // rolling m-mer scores: X[r] = score at local base 32*(s + r) + lane
        u64 X[NREG];
#pragma unroll
        for (int r = 0; r < NREG; ++r) X[r] = mmer_score(wpk, 32 * r + lane, m, P.seed);

        int c_valid = 0, c_runstart = -1;   // carry from lane 31 of the previous step
        uint32_t c_b = 0;
        int pv = 0, pstart = 0, plp = 0, psm = 0;  // previous step, for delayed emission
        uint32_t pb = 0;

        auto emit = [&](uint32_t b, int sm_start, int lp_end) {
            int n = lp_end - sm_start + 1;
            if (MODE == SM_COUNT) {
                atomicAdd(&s_cnt[b], 1u);
                atomicAdd(&s_km[b], (uint32_t)n);
            } else if (MODE == SM_SCATTER) {
                u64 slot = s_base[b] + atomicAdd(&s_cur[b], 1u);
                if (slot >= P.n_records_cap) {
                    raise_error(P.err, HSK_DERR_BOUNDS);
                    return;
                }
                int nb = n + k - 1;  // bases in the record
                u64* dst = reinterpret_cast<u64*>(P.records) + slot * (u64)P.rec_words;
                if (!WIDE) {
                    u64 a = extract_k64(wpk, (u64)sm_start, 32);
                    u64 c = extract_k64(wpk, (u64)(sm_start + 32), 32);
                    a = keep_bases(a, nb);
                    c = keep_bases(c, nb - 32) | (u64)n;
                    *reinterpret_cast<ulonglong2*>(dst) = make_ulonglong2(a, c);
                } else {
                    u64 r[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        r[i] = keep_bases(extract_k64(wpk, (u64)(sm_start + 32 * i), 32), nb - 32 * i);
                    r[3] |= (u64)n;
                    reinterpret_cast<ulonglong2*>(dst)[0] = make_ulonglong2(r[0], r[1]);
                    reinterpret_cast<ulonglong2*>(dst)[1] = make_ulonglong2(r[2], r[3]);
                }
            }
        };

        for (int s = 0; s < SM_STEPS; ++s) {
            const int lp = 32 * s + lane;
            const u64 p = p0 + lp;
            int valid = (p + k <= P.n_bases) && mask_bits(wiv, lp, k) == 0 &&
                        (k == 1 || mask_bits(wrs, lp + 1, k - 1) == 0);
            const u64 mh = window_min<NREG>(X, w, lane);
            const uint32_t b = bucket_of(mh, B);

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
                int prev_valid = __shfl_up_sync(0xffffffffu, valid, 1);
                uint32_t prev_b = __shfl_up_sync(0xffffffffu, b, 1);
                if (lane == 0) {
                    prev_valid = c_valid;
                    prev_b = c_b;
                }
                int start0 = valid && !(prev_valid && prev_b == b);
                int rs = warp_incl_max(start0 ? lp : -1);
                rs = rs > c_runstart ? rs : c_runstart;
                int pos_in_run = lp - rs;
                int q = pos_in_run / nmax;
                int start = valid && (start0 || pos_in_run - q * nmax == 0);
                int smstart = rs + q * nmax;
                if (s > 0) {  // emit supermers that ended in the previous step
                    int nv = __shfl_down_sync(0xffffffffu, pv, 1);
                    int ns = __shfl_down_sync(0xffffffffu, pstart, 1);
                    int v0 = __shfl_sync(0xffffffffu, valid, 0);
                    int s0 = __shfl_sync(0xffffffffu, start, 0);
                    if (lane == 31) {
                        nv = v0;
                        ns = s0;
                    }
                    if (pv && (!nv || ns)) emit(pb, psm, plp);
                }
                c_valid = __shfl_sync(0xffffffffu, valid, 31);
                c_b = __shfl_sync(0xffffffffu, b, 31);
                c_runstart = __shfl_sync(0xffffffffu, rs, 31);
                pv = valid;
                pstart = start;
                pb = b;
                plp = lp;
                psm = smstart;
            }
            // roll the scores forward by one step
#pragma unroll
            for (int r = 0; r + 1 < NREG; ++r) X[r] = X[r + 1];
            X[NREG - 1] = mmer_score(wpk, 32 * (s + NREG) + lane, m, P.seed);
        }
        if (MODE != SM_DUMP) {  // the tile edge ends every open supermer
            int nv = __shfl_down_sync(0xffffffffu, pv, 1);
            int ns = __shfl_down_sync(0xffffffffu, pstart, 1);
            if (lane == 31) {
                nv = 0;
                ns = 0;
            }
            if (pv && (!nv || ns)) emit(pb, psm, plp);
        }
        __syncwarp();
    }

    if (MODE == SM_COUNT) {
        __syncthreads();
        for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) {
            P.cta_counts[(u64)b * P.grid + blockIdx.x] = s_cnt[b];
            if (s_km[b]) atomicAdd(reinterpret_cast<unsigned long long*>(P.bucket_kmers + b),
                                   (unsigned long long)s_km[b]);
        }
    }
}

template <int MODE>
static void launch_mode(const SmParams& p, cudaStream_t st) {
    size_t sm = supermer_smem_bytes(MODE, p.n_buckets);
    bool wide = p.k > 32;
    int nreg = (p.w <= 33) ? 2 : 3;
    unsigned grid = p.grid;
    count_launch();
#define HSK_SM_LAUNCH(W, NR)                                                                 \
    do {                                                                                     \
        auto fn = k_supermer<MODE, W, NR>;                                                   \
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);      \
        fn<<<grid, 256, sm, st>>>(p);                                                        \
    } while (0)
    if (!wide && nreg == 2) HSK_SM_LAUNCH(false, 2);
    else if (!wide) HSK_SM_LAUNCH(false, 3);
    else if (nreg == 2) HSK_SM_LAUNCH(true, 2);
    else HSK_SM_LAUNCH(true, 3);
#undef HSK_SM_LAUNCH
}

void launch_supermer(int mode, const SmParams& p, cudaStream_t st) {
    if (p.n_bases == 0) return;
    if (mode == SM_COUNT) launch_mode<SM_COUNT>(p, st);
    else if (mode == SM_SCATTER) launch_mode<SM_SCATTER>(p, st);
    else launch_mode<SM_DUMP>(p, st);
}

int supermer_max_ctas_per_sm(int mode, bool wide, int nreg, uint32_t n_buckets) {
    size_t sm = supermer_smem_bytes(mode, n_buckets);
    int n = 0;
    const void* fn = nullptr;
    if (mode == SM_SCATTER) {
        fn = wide ? (nreg == 2 ? (const void*)k_supermer<SM_SCATTER, true, 2> : (const void*)k_supermer<SM_SCATTER, true, 3>)
                  : (nreg == 2 ? (const void*)k_supermer<SM_SCATTER, false, 2> : (const void*)k_supermer<SM_SCATTER, false, 3>);
    } else {
        fn = wide ? (nreg == 2 ? (const void*)k_supermer<SM_COUNT, true, 2> : (const void*)k_supermer<SM_COUNT, true, 3>)
                  : (nreg == 2 ? (const void*)k_supermer<SM_COUNT, false, 2> : (const void*)k_supermer<SM_COUNT, false, 3>);
    }
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 256, sm) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
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

__global__ void k_gather_stride(const u64* __restrict__ off, uint32_t B, uint32_t stride,
                                u64* __restrict__ out) {
    uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b <= B) out[b] = off[(u64)b * stride];
}

void launch_gather_stride(const uint64_t* off, uint32_t B, uint32_t stride, uint64_t* out,
                          cudaStream_t st) {
    count_launch();
    k_gather_stride<<<(B + 1 + 255) / 256, 256, 0, st>>>((const u64*)off, B, stride, (u64*)out);
}

}  // namespace hsk
