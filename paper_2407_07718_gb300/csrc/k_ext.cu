// k_ext.cu -- extension information of the kept k-mers (Sec. 3.3.2): the
// read and position of every occurrence of every k-mer the filter kept.
//
// After a count, the kept k-mers are sorted and distinct.  They are entered
// into a table of indices (open addressing over 32-bit slots holding index+1;
// a probe compares the query with the kept key at that index, so one 32-bit
// compare-and-swap claims a slot whatever the key width).  A scan over every
// window then looks its canonical key up and, when the key is kept, emits the
// composite (k-mer index, global window start).  Sorting the composites (the
// LSD radix sort of k_sort.cu) puts each k-mer's occurrences together in
// position order, which is (read, position) order; a last pass turns the
// global start into (read, position in read) with a binary search over the
// read offsets.
//
// The payload codec (k_ext_encode / k_ext_decode) is the paper's encoding of
// extension information on its way to a destination: each item is
// (read, position); when both differ from the previous item of the stream by
// a value that fits an int8, the item is one flag byte plus the two int8
// differences, otherwise the flag byte plus the full uint32 read and uint32
// position.  Streams are cut into chunks of EXT_CHUNK items whose first item is
// always full, so chunks encode and decode independently.
#include "hsk_device.cuh"

namespace hsk {

constexpr uint32_t EXT_EMPTY = 0;

__device__ __forceinline__ uint32_t ext_hash(u64 k) { return (uint32_t)((k * 0x9E3779B97F4A7C15ULL) >> 32); }
__device__ __forceinline__ uint32_t ext_hash(const key128& k) {
    return (uint32_t)(((k.lo ^ (k.hi * 0xC2B2AE3D27D4EB4FULL)) * 0x9E3779B97F4A7C15ULL) >> 32);
}

template <typename K>
__global__ void __launch_bounds__(256) k_ext_insert(const K* __restrict__ keys, uint64_t n, uint32_t* table,
                                                    uint32_t mask, int* err) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const K key = keys[i];
        uint32_t h = ext_hash(key) & mask;
        for (uint32_t probe = 0;; ++probe) {
            if (probe > mask) {  // never: the table has twice as many slots as keys
                raise_error(err, HSK_DERR_BOUNDS);
                break;
            }
            if (atomicCAS(&table[h], EXT_EMPTY, (uint32_t)i + 1) == EXT_EMPTY) break;
            h = (h + 1) & mask;
        }
    }
}

// Index of `key` among the kept keys, or -1.
template <typename K>
__device__ __forceinline__ int64_t ext_find(const K& key, const K* __restrict__ kept, const uint32_t* __restrict__ table,
                                            uint32_t mask) {
    uint32_t h = ext_hash(key) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const uint32_t v = table[h];
        if (v == EXT_EMPTY) return -1;
        if (key_eq(kept[v - 1], key)) return (int64_t)(v - 1);
        h = (h + 1) & mask;
    }
    return -1;
}

// One thread per 64 window starts: validity from the invalid and read-start
// masks (no invalid base in the window, no read start after its first base),
// then each valid window's canonical key is looked up; kept ones emit
// (index << 40) | start into out[atomic cursor] (128-bit composites when the
// index needs more than 24 bits).
template <typename K>
__global__ void __launch_bounds__(256) k_ext_scan(const u64* __restrict__ packed, const u64* __restrict__ invalid,
                                                  const u64* __restrict__ start, uint64_t n_bases, int k,
                                                  const K* __restrict__ kept, const uint32_t* __restrict__ table,
                                                  uint32_t mask, bool wide_out, void* out, uint64_t out_cap,
                                                  unsigned long long* cursor, int* err) {
    const uint64_t words = (n_bases + 63) / 64;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (uint64_t)gridDim.x * blockDim.x) {
        // bad window starts: an invalid base in [p, p + k) or a read start in (p, p + k)
        u64 bad = 0;
        for (int j = 0; j < k; ++j) {
            const uint64_t g = w * 64 + j;  // bits of window starts w*64 .. w*64+63, shifted by j
            const uint64_t q = g >> 6;
            const int off = (int)(g & 63);
            const u64 a = q < words ? invalid[q] : ~0ULL;
            const u64 b = q + 1 < words ? invalid[q + 1] : ~0ULL;
            bad |= off ? (a << off) | (b >> (64 - off)) : a;
            if (j > 0) {
                const u64 sa = q < words ? start[q] : 0ULL;
                const u64 sb = q + 1 < words ? start[q + 1] : 0ULL;
                bad |= off ? (sa << off) | (sb >> (64 - off)) : sa;
            }
        }
        u64 good = ~bad;
        while (good) {
            const int t = __clzll(good);  // most significant first: window w*64 + t
            good &= ~(0x8000000000000000ULL >> t);
            const uint64_t p = w * 64 + (uint64_t)t;
            if (p + (uint64_t)k > n_bases) break;
            K key;
            if constexpr (std::is_same<K, u64>::value) key = canonical64(extract_k64(packed, p, k), k);
            else key = canonical128(extract_k128(packed, p, k), k);
            const int64_t idx = ext_find(key, kept, table, mask);
            if (idx < 0) continue;
            const unsigned long long at = atomicAdd(cursor, 1ULL);
            if (at >= out_cap) {
                raise_error(err, HSK_DERR_BOUNDS);
                continue;
            }
            if (!wide_out) {
                reinterpret_cast<u64*>(out)[at] = ((u64)idx << 40) | p;
            } else {
                key128 c;
                c.lo = p | ((u64)idx << 40);
                c.hi = (u64)idx >> 24;
                reinterpret_cast<key128*>(out)[at] = c;
            }
        }
    }
}

// Sorted composites -> (read, position in read): read = the last read whose
// offset is <= the global start.
__global__ void __launch_bounds__(256) k_ext_decode_pos(const void* comp, bool wide, uint64_t n,
                                                        const uint64_t* __restrict__ offsets, uint64_t n_reads,
                                                        uint32_t* __restrict__ occ_read, uint32_t* __restrict__ occ_pos) {
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x) {
        const u64 p = wide ? (reinterpret_cast<const key128*>(comp)[j].lo & ((1ULL << 40) - 1))
                           : (reinterpret_cast<const u64*>(comp)[j] & ((1ULL << 40) - 1));
        uint64_t lo = 0, hi = n_reads;  // offsets[lo] <= p < offsets[hi]
        while (hi - lo > 1) {
            const uint64_t mid = (lo + hi) >> 1;
            if (offsets[mid] <= p) lo = mid;
            else hi = mid;
        }
        occ_read[j] = (uint32_t)lo;
        occ_pos[j] = (uint32_t)(p - offsets[lo]);
    }
}

void launch_ext_insert(const void* keys, int key_words, uint64_t n, uint32_t* table, uint32_t mask, int* err,
                       cudaStream_t st) {
    if (n == 0) return;
    count_launch();
    const unsigned g = (unsigned)std::min<uint64_t>((n + 255) / 256, 65535);
    if (key_words == 1) k_ext_insert<u64><<<g, 256, 0, st>>>((const u64*)keys, n, table, mask, err);
    else k_ext_insert<key128><<<g, 256, 0, st>>>((const key128*)keys, n, table, mask, err);
}

void launch_ext_scan(const uint64_t* packed, const uint64_t* invalid, const uint64_t* start, uint64_t n_bases, int k,
                     const void* kept, const uint32_t* table, uint32_t mask, bool wide_out, void* out,
                     uint64_t out_cap, uint64_t* cursor, int* err, int grid, cudaStream_t st) {
    if (n_bases == 0) return;
    count_launch();
    const uint64_t words = (n_bases + 63) / 64;
    const unsigned g = (unsigned)std::min<uint64_t>((words + 255) / 256, (uint64_t)grid);
    if (k <= 32)
        k_ext_scan<u64><<<g, 256, 0, st>>>((const u64*)packed, (const u64*)invalid, (const u64*)start, n_bases, k,
                                           (const u64*)kept, table, mask, wide_out, out, out_cap,
                                           (unsigned long long*)cursor, err);
    else
        k_ext_scan<key128><<<g, 256, 0, st>>>((const u64*)packed, (const u64*)invalid, (const u64*)start, n_bases, k,
                                              (const key128*)kept, table, mask, wide_out, out, out_cap,
                                              (unsigned long long*)cursor, err);
}

void launch_ext_decode_pos(const void* comp, bool wide, uint64_t n, const uint64_t* offsets, uint64_t n_reads,
                           uint32_t* occ_read, uint32_t* occ_pos, int grid, cudaStream_t st) {
    if (n == 0) return;
    count_launch();
    const unsigned g = (unsigned)std::min<uint64_t>((n + 255) / 256, (uint64_t)grid);
    k_ext_decode_pos<<<g, 256, 0, st>>>(comp, wide, n, offsets, n_reads, occ_read, occ_pos);
}

// ---------------------------------------------------------------------------
// the extension-information codec (Sec. 3.3.2)
// ---------------------------------------------------------------------------
// Item i of a stream: (read[i], pos[i]).  Flag byte: 1 = deltas follow (two
// int8: read - previous read, pos - previous pos), 0 = full values follow
// (uint32 read, uint32 pos, little endian).  The first item of every chunk of
// EXT_CHUNK items is full.  Sizes: 3 or 9 bytes.
constexpr uint32_t EXT_CHUNK = 1024;

__device__ __forceinline__ bool ext_small(uint32_t r, uint32_t p, uint32_t pr, uint32_t pp) {
    const long long dr = (long long)r - (long long)pr, dp = (long long)p - (long long)pp;
    return dr >= -128 && dr <= 127 && dp >= -128 && dp <= 127;
}

// bytes of item i (pass 1)
__global__ void k_ext_sizes(const uint32_t* __restrict__ rd, const uint32_t* __restrict__ ps, uint64_t n,
                            uint32_t* __restrict__ size) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const bool delta = (i % EXT_CHUNK) != 0 && ext_small(rd[i], ps[i], rd[i - 1], ps[i - 1]);
        size[i] = delta ? 3u : 9u;
    }
}

// item i written at byte off[i] (pass 2, off = exclusive scan of the sizes)
__global__ void k_ext_encode(const uint32_t* __restrict__ rd, const uint32_t* __restrict__ ps, uint64_t n,
                             const uint64_t* __restrict__ off, uint8_t* __restrict__ out) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint8_t* o = out + off[i];
        const bool delta = (i % EXT_CHUNK) != 0 && ext_small(rd[i], ps[i], rd[i - 1], ps[i - 1]);
        if (delta) {
            o[0] = 1;
            o[1] = (uint8_t)(int8_t)((long long)rd[i] - (long long)rd[i - 1]);
            o[2] = (uint8_t)(int8_t)((long long)ps[i] - (long long)ps[i - 1]);
        } else {
            o[0] = 0;
            for (int b = 0; b < 4; ++b) {
                o[1 + b] = (uint8_t)(rd[i] >> (8 * b));
                o[5 + b] = (uint8_t)(ps[i] >> (8 * b));
            }
        }
    }
}

// One thread per chunk: walk the chunk's items from its first (full) item.
__global__ void k_ext_decode(const uint8_t* __restrict__ in, uint64_t n_bytes, uint64_t n,
                             const uint64_t* __restrict__ chunk_off, uint32_t* __restrict__ rd,
                             uint32_t* __restrict__ ps, int* err) {
    const uint64_t chunks = (n + EXT_CHUNK - 1) / EXT_CHUNK;
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < chunks;
         c += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t at = chunk_off[c];
        uint32_t r = 0, p = 0;
        const uint64_t i1 = (c + 1) * EXT_CHUNK < n ? (c + 1) * EXT_CHUNK : n;
        for (uint64_t i = c * EXT_CHUNK; i < i1; ++i) {
            if (at >= n_bytes) {
                raise_error(err, HSK_DERR_BOUNDS);
                return;
            }
            const uint8_t f = in[at];
            if (f == 1 && i != c * EXT_CHUNK && at + 3 <= n_bytes) {
                r = (uint32_t)((long long)r + (int8_t)in[at + 1]);
                p = (uint32_t)((long long)p + (int8_t)in[at + 2]);
                at += 3;
            } else if (f == 0 && at + 9 <= n_bytes) {
                r = p = 0;
                for (int b = 0; b < 4; ++b) {
                    r |= (uint32_t)in[at + 1 + b] << (8 * b);
                    p |= (uint32_t)in[at + 5 + b] << (8 * b);
                }
                at += 9;
            } else {
                raise_error(err, HSK_DERR_BOUNDS);
                return;
            }
            rd[i] = r;
            ps[i] = p;
        }
    }
}

// byte offset of each chunk's first item (from the item offsets)
__global__ void k_ext_chunk_off(const uint64_t* __restrict__ off, uint64_t n, uint64_t* __restrict__ chunk_off) {
    const uint64_t chunks = (n + EXT_CHUNK - 1) / EXT_CHUNK;
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < chunks;
         c += (uint64_t)gridDim.x * blockDim.x)
        chunk_off[c] = off[c * EXT_CHUNK];
}

uint64_t ext_chunk_items() { return EXT_CHUNK; }

void launch_ext_sizes(const uint32_t* rd, const uint32_t* ps, uint64_t n, uint32_t* size, int grid, cudaStream_t st) {
    if (n == 0) return;
    count_launch();
    k_ext_sizes<<<(unsigned)std::min<uint64_t>((n + 255) / 256, (uint64_t)grid), 256, 0, st>>>(rd, ps, n, size);
}
void launch_ext_encode(const uint32_t* rd, const uint32_t* ps, uint64_t n, const uint64_t* off, uint8_t* out,
                       int grid, cudaStream_t st) {
    if (n == 0) return;
    count_launch();
    k_ext_encode<<<(unsigned)std::min<uint64_t>((n + 255) / 256, (uint64_t)grid), 256, 0, st>>>(rd, ps, n,
                                                                                              off, out);
}
void launch_ext_chunk_off(const uint64_t* off, uint64_t n, uint64_t* chunk_off, int grid, cudaStream_t st) {
    if (n == 0) return;
    count_launch();
    const uint64_t chunks = (n + EXT_CHUNK - 1) / EXT_CHUNK;
    const unsigned g = (unsigned)std::min<uint64_t>((chunks + 255) / 256, (uint64_t)grid);
    k_ext_chunk_off<<<g, 256, 0, st>>>(off, n, chunk_off);
}
void launch_ext_decode(const uint8_t* in, uint64_t n_bytes, uint64_t n, const uint64_t* chunk_off, uint32_t* rd,
                       uint32_t* ps, int* err, int grid, cudaStream_t st) {
    if (n == 0) return;
    count_launch();
    const uint64_t chunks = (n + EXT_CHUNK - 1) / EXT_CHUNK;
    const unsigned g = (unsigned)std::min<uint64_t>((chunks + 255) / 256, (uint64_t)grid);
    k_ext_decode<<<g, 256, 0, st>>>(in, n_bytes, n, chunk_off, rd, ps, err);
}

}  // namespace hsk
