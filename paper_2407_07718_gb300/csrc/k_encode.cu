// k_encode.cu -- stage S1: 2-bit encoding of reads (Sec. 2.2: sequences are
// encoded before they are parsed into k-mers).
//
// One thread turns 64 ASCII bytes (four 128-bit loads) into two packed words
// (32 bases each, first base most significant) and one invalid-mask word.
// The kernel is bound by HBM: 1 byte read and 0.375 bytes written per base.
#include "hsk_device.cuh"

namespace hsk {

// 4 ASCII bytes (little-endian in x) -> 4 codes packed most significant first
// in 8 bits, plus a 4-bit invalid nibble (first byte in bit 3).
__device__ __forceinline__ void encode4(uint32_t x, uint32_t& code8, uint32_t& inv4) {
    uint32_t ok = __vcmpeq4(x, 0x41414141u) | __vcmpeq4(x, 0x43434343u) |
                  __vcmpeq4(x, 0x47474747u) | __vcmpeq4(x, 0x54545454u);
    // A 0x41 -> 0, C 0x43 -> 1, G 0x47 -> 2, T 0x54 -> 3: ((c >> 2) ^ (c >> 1)) & 3
    uint32_t c = ((x >> 2) ^ (x >> 1)) & 0x03030303u & ok;
    code8 = ((c & 3u) << 6) | (((c >> 8) & 3u) << 4) | (((c >> 16) & 3u) << 2) | ((c >> 24) & 3u);
    uint32_t bad = ~ok;
    inv4 = ((bad & 1u) << 3) | (((bad >> 8) & 1u) << 2) | (((bad >> 16) & 1u) << 1) | ((bad >> 24) & 1u);
}

__global__ void __launch_bounds__(256) k_encode(const char* __restrict__ reads, uint64_t n_bases,
                                                u64* __restrict__ packed, u64* __restrict__ invalid,
                                                uint64_t n_packed_words, uint64_t t0, uint64_t t1,
                                                bool aligned16) {
    uint64_t t = t0 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= t1) return;
    uint64_t b0 = t * 64;
    uint32_t x[16];
    if (aligned16 && b0 + 64 <= n_bases) {
        const uint4* src = reinterpret_cast<const uint4*>(reads + b0);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            uint4 q = __ldcs(src + v);  // streamed once: do not keep in L1/L2
            x[4 * v] = q.x;
            x[4 * v + 1] = q.y;
            x[4 * v + 2] = q.z;
            x[4 * v + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            uint32_t v = 0;
            for (int b = 0; b < 4; ++b) {
                uint64_t g = b0 + 4 * j + b;
                // bytes past the data read as 0 -> invalid
                uint32_t c = g < n_bases ? (uint32_t)(unsigned char)reads[g] : 0u;
                v |= c << (8 * b);
            }
            x[j] = v;
        }
    }
    u64 w0 = 0, w1 = 0, iv = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        uint32_t c8, i4;
        encode4(x[j], c8, i4);
        if (j < 8)
            w0 |= (u64)c8 << (56 - 8 * j);
        else
            w1 |= (u64)c8 << (56 - 8 * (j - 8));
        iv |= (u64)i4 << (60 - 4 * j);
    }
    if (2 * t < n_packed_words) packed[2 * t] = w0;
    if (2 * t + 1 < n_packed_words) packed[2 * t + 1] = w1;
    invalid[t] = iv;
}

// Marks the first base of every non-empty read and checks the offsets:
// offsets[0] = 0, offsets[n_reads] = n_bases, non-decreasing.
__global__ void k_mark_starts(const uint64_t* __restrict__ offsets, uint64_t n_reads,
                              uint64_t n_bases, u64* __restrict__ start, int* err) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_reads) return;
    uint64_t s = offsets[i], e = offsets[i + 1];
    if (e < s || e > n_bases || (i == 0 && s != 0) || (i + 1 == n_reads && e != n_bases)) {
        raise_error(err, HSK_DERR_OFFSETS);
        return;
    }
    if (e > s) atomicOr(start + (s >> 6), 1ULL << (63 - (s & 63)));
}

// Packed sets: set y's reads are offsets[off0[y] .. off0[y] + n_reads[y]]
// (its own offsets, starting at 0) placed at base[y] of the packed bases;
// the bytes from the set's last base to base[y + 1] are padding and are set
// to 0 here (an invalid byte, so no window reaches into them).  Marks the first
// base of every non-empty read; offsets that leave the set's range are an
// error.
__global__ void k_mark_starts_sets(const uint64_t* __restrict__ offsets, const uint64_t* __restrict__ off0,
                                   const uint64_t* __restrict__ n_reads, const uint64_t* __restrict__ base,
                                   char* reads, u64* __restrict__ start, int* err) {
    const uint32_t y = blockIdx.y;
    const uint64_t nr = n_reads[y], b0 = base[y], b1 = base[y + 1];
    const uint64_t* o = offsets + off0[y];
    const uint64_t nb = o[nr];
    if (o[0] != 0 || b0 + nb > b1) {  // every block checks: nothing is written outside the set
        if (blockIdx.x == 0 && threadIdx.x == 0) raise_error(err, HSK_DERR_OFFSETS);
        return;
    }
    if (blockIdx.x == 0)
        for (uint64_t p = b0 + nb + threadIdx.x; p < b1; p += blockDim.x) reads[p] = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t a = o[i], e = o[i + 1];
        if (e < a || e > nb) {
            raise_error(err, HSK_DERR_OFFSETS);
            return;
        }
        if (e > a) atomicOr(start + ((b0 + a) >> 6), 1ULL << (63 - ((b0 + a) & 63)));
    }
}

void launch_mark_starts_sets(const uint64_t* offsets, const uint64_t* off0, const uint64_t* n_reads,
                             const uint64_t* base, uint32_t n_sets, uint64_t max_reads, char* reads,
                             uint64_t* start_mask, int* err, cudaStream_t st) {
    if (n_sets == 0) return;
    count_launch();
    uint64_t bx = (max_reads + 255) / 256;
    if (bx < 1) bx = 1;
    if (bx > 1024) bx = 1024;
    k_mark_starts_sets<<<dim3((unsigned)bx, n_sets), 256, 0, st>>>(offsets, off0, n_reads, base, reads,
                                                                   (u64*)start_mask, err);
}

void launch_encode(const char* reads, uint64_t n_bases, uint64_t* packed, uint64_t* invalid,
                   uint64_t n_packed_words, uint64_t n_mask_words, cudaStream_t st) {
    uint64_t threads = (n_bases + 63) / 64;
    if (threads == 0) return;
    count_launch();
    bool al = (reinterpret_cast<uintptr_t>(reads) & 15) == 0;
    k_encode<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
        reads, n_bases, (u64*)packed, (u64*)invalid, n_packed_words, 0, threads, al);
}

void launch_encode_range(const char* reads, uint64_t n_bases, uint64_t b0, uint64_t b1, uint64_t* packed,
                         uint64_t* invalid, uint64_t n_packed_words, cudaStream_t st) {
    const uint64_t t0 = b0 / 64, t1 = (b1 + 63) / 64;
    if (t1 <= t0) return;
    count_launch();
    bool al = (reinterpret_cast<uintptr_t>(reads) & 15) == 0;
    k_encode<<<(unsigned)((t1 - t0 + 255) / 256), 256, 0, st>>>(reads, n_bases, (u64*)packed, (u64*)invalid,
                                                                n_packed_words, t0, t1, al);
}

void launch_mark_starts(const uint64_t* offsets, uint64_t n_reads, uint64_t n_bases,
                        uint64_t* start_mask, int* err, cudaStream_t st) {
    if (n_reads == 0) return;
    count_launch();
    k_mark_starts<<<(unsigned)((n_reads + 255) / 256), 256, 0, st>>>(offsets, n_reads, n_bases,
                                                                     (u64*)start_mask, err);
}

}  // namespace hsk
