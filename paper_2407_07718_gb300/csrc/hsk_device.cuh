// hsk_device.cuh -- device helpers shared by the k-mer counting kernels.
//
// Key types: k <= 32 uses uint64 (the 2k-bit canonical code, right aligned);
// 33 <= k <= 64 uses key128 {lo, hi}.  Bases are 2-bit codes A=0 C=1 G=2 T=3,
// the first base of a k-mer in its most significant bits, so numeric order is
// lexicographic order of the k-mer string (Sec. 2.1 defines k-mers; the code
// and the canonical form are this library's reading of it).
#pragma once

#include <type_traits>

#include <cstdint>

#include <cuda_runtime.h>

#include "hsk_internal.h"

namespace hsk {

typedef unsigned long long u64;

struct key128 {
    u64 lo, hi;
};

__device__ __forceinline__ bool key_lt(u64 a, u64 b) { return a < b; }
__device__ __forceinline__ bool key_lt(const key128& a, const key128& b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ bool key_eq(u64 a, u64 b) { return a == b; }
__device__ __forceinline__ bool key_eq(const key128& a, const key128& b) {
    return a.hi == b.hi && a.lo == b.lo;
}

// Radix digit of `bits` bits starting at bit `shift`.
__device__ __forceinline__ uint32_t key_digit(u64 k, int shift, uint32_t mask) {
    return (uint32_t)(k >> shift) & mask;
}
__device__ __forceinline__ uint32_t key_digit(const key128& k, int shift, uint32_t mask) {
    if (shift >= 64) return (uint32_t)(k.hi >> (shift - 64)) & mask;
    u64 v = k.lo >> shift;
    if (shift > 0) v |= k.hi << (64 - shift);
    return (uint32_t)v & mask;
}

// 64 bits of a most-significant-first bit stream starting `off` (0..63) bits
// into word a (b is the following word).
__device__ __forceinline__ u64 funnel64(u64 a, u64 b, uint32_t off) {
    return (a << off) | ((b >> 1) >> (63 - off));
}

// Reverse the order of 2-bit groups of x (complement applied by the caller).
__device__ __forceinline__ u64 reverse_pairs(u64 x) {
    x = __brevll(x);
    return ((x >> 1) & 0x5555555555555555ULL) | ((x & 0x5555555555555555ULL) << 1);
}

// Reverse complement of a right-aligned code of k <= 32 bases.
__device__ __forceinline__ u64 revcomp64(u64 fwd, int k) {
    return reverse_pairs(~fwd) >> (64 - 2 * k);
}

// Reverse complement of a right-aligned code of 33 <= k <= 64 bases.
__device__ __forceinline__ key128 revcomp128(const key128& f, int k) {
    u64 nh = reverse_pairs(~f.lo), nl = reverse_pairs(~f.hi);  // full 128-bit reversal
    int s = 128 - 2 * k;                                       // 0 .. 62
    key128 r;
    if (s == 0) {
        r.lo = nl;
        r.hi = nh;
    } else {
        r.lo = (nl >> s) | (nh << (64 - s));
        r.hi = nh >> s;
    }
    return r;
}

// Code of the k (<= 32) bases starting at base index p of a packed stream.
__device__ __forceinline__ u64 extract_k64(const u64* w, u64 p, int k) {
    u64 i = p >> 5;
    uint32_t off = (uint32_t)(p & 31) * 2;
    return funnel64(w[i], w[i + 1], off) >> (64 - 2 * k);
}

// Code of the k (33..64) bases starting at base index p of a packed stream.
__device__ __forceinline__ key128 extract_k128(const u64* w, u64 p, int k) {
    u64 i = p >> 5;
    uint32_t off = (uint32_t)(p & 31) * 2;
    u64 a = funnel64(w[i], w[i + 1], off);
    u64 b = funnel64(w[i + 1], w[i + 2], off);
    int s = 128 - 2 * k;  // 0..62
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

__device__ __forceinline__ u64 canonical64(u64 fwd, int k) {
    u64 rc = revcomp64(fwd, k);
    return fwd < rc ? fwd : rc;
}
__device__ __forceinline__ key128 canonical128(const key128& fwd, int k) {
    key128 rc = revcomp128(fwd, k);
    return key_lt(fwd, rc) ? fwd : rc;
}


// ---------------------------------------------------------------------------
// device error flag and bounded waits
// ---------------------------------------------------------------------------
__device__ __forceinline__ void raise_error(int* err, int code) {
    if (err) atomicCAS(err, 0, code);
}

__device__ __forceinline__ u64 ld_relaxed(const u64* p) {
    u64 v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(u64* p, u64 v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Look-back status word: [63:62] flag, [61:48] epoch, [47:0] value.
constexpr u64 LB_AGG = 1ULL << 62;
constexpr u64 LB_PREFIX = 2ULL << 62;
constexpr u64 LB_VALUE = (1ULL << 48) - 1;
// Words between the status words of consecutive tiles in one-value look-backs:
// one 32-byte L2 sector per tile, so neighbouring tiles never write the same sector.
constexpr int LB_PAD = 4;
__device__ __forceinline__ u64 lb_word(u64 flag, uint32_t epoch, u64 value) {
    return flag | ((u64)(epoch & 0x3FFF) << 48) | (value & LB_VALUE);
}

// Decoupled look-back for one value (Merrill & Garland, 2016): sum the values
// of tiles before `tile` until one carries an inclusive prefix.  Bounded: after
// LB_SPIN_LIMIT empty reads the wait gives up, raises HSK_DERR_TIMEOUT and
// returns what it has (the host then discards the result).
__device__ __forceinline__ u64 lookback_exclusive(u64* status, u64 stride, u64 tile,
                                                  uint32_t epoch, int* err,
                                                  uint32_t spin_limit = HSK_SPIN_LIMIT) {
    u64 excl = 0;
    long long j = (long long)tile - 1;
    uint32_t spins = 0;
    while (j >= 0) {
        u64 s = ld_relaxed(status + (u64)j * stride);
        uint32_t ep = (uint32_t)(s >> 48) & 0x3FFF;
        u64 fl = s & (3ULL << 62);
        if (fl == 0 || ep != (epoch & 0x3FFF)) {
            if (++spins > spin_limit) {
                raise_error(err, HSK_DERR_TIMEOUT);
                break;
            }
            if (spins > 64) __nanosleep(64);
            continue;
        }
        excl += s & LB_VALUE;
        if (fl == LB_PREFIX) break;
        --j;
    }
    return excl;
}

// The same look-back with WIN status words loaded per round trip: the WIN
// predecessors' words are read independently, then consumed in order until a
// word is not ready (re-read from there) or carries an inclusive prefix.  On
// this GPU a status word can sit in the far die's L2, so one dependent read
// costs ~1 us; reading WIN at a time divides the chain of waits by WIN.
template <int WIN>
__device__ __forceinline__ u64 lookback_exclusive_win(u64* status, u64 stride, u64 tile,
                                                      uint32_t epoch, int* err) {
    u64 excl = 0;
    long long j = (long long)tile - 1;
    uint32_t spins = 0;
    const uint32_t ep_want = epoch & 0x3FFF;
    while (j >= 0) {
        u64 s[WIN];
#pragma unroll
        for (int i = 0; i < WIN; ++i) s[i] = (j - i >= 0) ? ld_relaxed(status + (u64)(j - i) * stride) : 0ULL;
        int used = 0;
        bool done = false;
#pragma unroll
        for (int i = 0; i < WIN; ++i) {
            if (done || used != i) continue;  // stop at the first word not consumed
            if (j - i < 0) {
                done = true;
                continue;
            }
            u64 fl = s[i] & (3ULL << 62);
            if (fl == 0 || ((uint32_t)(s[i] >> 48) & 0x3FFF) != ep_want) continue;  // not ready
            excl += s[i] & LB_VALUE;
            used = i + 1;
            if (fl == LB_PREFIX) done = true;
        }
        if (done) break;
        if (used == 0) {
            if (++spins > HSK_SPIN_LIMIT) {
                raise_error(err, HSK_DERR_TIMEOUT);
                break;
            }
            if (spins > 64) __nanosleep(64);
        }
        j -= used;
    }
    return excl;
}

// ---------------------------------------------------------------------------
// TMA bulk copies (global -> shared) completed on an mbarrier
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(u64* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// make barrier initialisation visible to the async (TMA) proxy
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order earlier generic-proxy accesses of shared memory before later TMA writes
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// arrive once and expect `bytes` of transactions on the barrier's current phase
__device__ __forceinline__ void mbar_arrive_expect_tx(u64* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
__device__ __forceinline__ void tma_load_1d(void* smem_dst, const void* gmem_src, uint32_t bytes, u64* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(smem_dst)),
                 "l"(gmem_src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
// true once the barrier's phase with the given parity has completed
__device__ __forceinline__ bool mbar_try_wait(u64* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Bounded wait: false (and the error word set) if the phase never completes.
__device__ __forceinline__ bool mbar_wait(u64* bar, uint32_t parity, int* err) {
    for (uint32_t i = 0; i < HSK_SPIN_LIMIT; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 64) __nanosleep(64);
    }
    raise_error(err, HSK_DERR_TIMEOUT);
    return false;
}

template <typename T>
__device__ __forceinline__ T warp_incl_sum(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += o;
    }
    return v;
}

// Exclusive prefix sum over a block of NT threads (NT <= 1024, multiple of
// 32); `total` receives the block sum.  Uses NT/32 words of `scratch`.
template <int NT, typename T>
__device__ __forceinline__ T block_excl_sum(T v, T* scratch, T& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = warp_incl_sum(v);
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NT / 32 ? scratch[lane] : T(0);
        T wi = warp_incl_sum(w);
        if (lane < NT / 32) scratch[lane] = wi - w;
        if (lane == NT / 32 - 1) scratch[NT / 32] = wi;
    }
    __syncthreads();
    T r = scratch[warp] + inc - v;
    total = scratch[NT / 32];
    __syncthreads();
    return r;
}


// ---------------------------------------------------------------------------
// supermer records -> k-mers
// ---------------------------------------------------------------------------
constexpr int EXP_RPT = 4;                 // records per thread
constexpr int EXP_TILE = 256 * EXP_RPT;    // records per tile of the expanding kernels

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

// Calls f(j, key) for the canonical k-mers j = 0 .. n-1 of a supermer record
// (record words W, bases packed from the most significant bit of W[0]): the
// first k-mer is cut out of the words, every next one rolls the forward code
// one base left and the reverse complement one base right.
template <bool WIDE, typename F>
__device__ __forceinline__ void record_kmers(const u64 (&W)[4], uint32_t n, int k, F&& f) {
    if (n == 0) return;
    const int kk = 2 * k;
    if constexpr (!WIDE) {
        const u64 mask = kk == 64 ? ~0ULL : ((1ULL << kk) - 1);
        u64 fwd = W[0] >> (64 - kk);
        u64 rc = revcomp64(fwd, k);
        u64 h, l;  // the bases after the first k-mer, most significant first
        if (kk == 64) {
            h = W[1];
            l = 0;
        } else {
            h = (W[0] << kk) | (W[1] >> (64 - kk));
            l = W[1] << kk;
        }
        f(0u, fwd < rc ? fwd : rc);
        for (uint32_t j = 1; j < n; ++j) {
            const u64 b = h >> 62;
            h = (h << 2) | (l >> 62);
            l <<= 2;
            fwd = ((fwd << 2) | b) & mask;
            rc = (rc >> 2) | ((3ULL - b) << (kk - 2));
            f(j, fwd < rc ? fwd : rc);
        }
    } else {
        const int s = 128 - kk;  // 0 .. 62
        key128 fwd;
        if (s == 0) {
            fwd.hi = W[0];
            fwd.lo = W[1];
        } else {
            fwd.hi = W[0] >> s;
            fwd.lo = (W[1] >> s) | (W[0] << (64 - s));
        }
        key128 rc = revcomp128(fwd, k);
        const int q = kk - 64;  // 2 .. 64: bits of the codes' high words
        const u64 himask = q == 64 ? ~0ULL : ((1ULL << q) - 1);
        u64 h, m, l;
        if (q == 64) {
            h = W[2];
            m = W[3];
            l = 0;
        } else {
            h = (W[1] << q) | (W[2] >> (64 - q));
            m = (W[2] << q) | (W[3] >> (64 - q));
            l = W[3] << q;
        }
        f(0u, key_lt(fwd, rc) ? fwd : rc);
        for (uint32_t j = 1; j < n; ++j) {
            const u64 b = h >> 62;
            h = (h << 2) | (m >> 62);
            m = (m << 2) | (l >> 62);
            l <<= 2;
            fwd.hi = ((fwd.hi << 2) | (fwd.lo >> 62)) & himask;
            fwd.lo = (fwd.lo << 2) | b;
            rc.lo = (rc.lo >> 2) | (rc.hi << 62);
            rc.hi = (rc.hi >> 2) | ((3ULL - b) << (q - 2));
            f(j, key_lt(fwd, rc) ? fwd : rc);
        }
    }
}

}  // namespace hsk
