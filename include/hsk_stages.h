/* hsk_stages.h -- per-stage entry points of the k-mer counting pipeline.
 *
 * Each function runs ONE stage of the pipeline that hsk_count() runs end to
 * end, on device-resident inputs, so that each stage can be checked on its
 * own.  All pointers named d_* are device pointers; `stream` is a
 * cudaStream_t (NULL = legacy default stream).  Each function returns after
 * its work on `stream` is complete.  Caller-provided outputs must have the
 * sizes stated; context-owned outputs stay valid until the next call on the
 * same context.  Return codes are those of hsk.h.
 *
 * Device layouts (shared by all stages):
 *   packed 2-bit bases : uint64 words, 32 bases per word, base g in bits
 *                        [63-2(g%32)-1 .. 63-2(g%32)] of word g/32 (first
 *                        base most significant); A=0 C=1 G=2 T=3; invalid
 *                        bytes are stored as 0.
 *   bit masks          : uint64 words, 64 bases per word, base g at bit
 *                        63-(g%64) of word g/64.
 *   supermer record    : record_words uint64 words (2 for k <= 32, 4 for
 *                        k <= 64); the supermer's bases packed from the most
 *                        significant bit of word 0 onward, bases beyond the
 *                        supermer zero; the low 8 bits of the last word hold
 *                        the number of k-mers n; the record spans n + k - 1
 *                        bases.
 */
#ifndef HSK_STAGES_H
#define HSK_STAGES_H

#include "hsk.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Stage S1, 2-bit encoding (Sec. 2.2: reads are encoded before k-mers are
 * parsed).  d_reads holds n_bases ASCII bytes; d_offsets n_reads + 1 entries.
 * Outputs (caller-allocated): d_packed ceil(n_bases/32) + 4 words;
 * d_invalid and d_start ceil(n_bases/64) + 4 words each.  d_invalid marks
 * bytes other than upper-case A/C/G/T; d_start marks the first base of every
 * non-empty read.  Words past the data are zero. */
int hsk_stage_encode(hsk_ctx* ctx, const char* d_reads, uint64_t n_bases,
                     const uint64_t* d_offsets, uint64_t n_reads, uint64_t* d_packed,
                     uint64_t* d_invalid, uint64_t* d_start, void* stream);

/* Stage S2, canonical k-mers and hash-scored minimizers (Sec. 3.2).  For
 * every window start g in [0, n_bases): d_valid[g] = 1 if bases g..g+k-1 are
 * all ACGT and inside one read, else 0; for valid windows d_key[2g], d_key[2g+1]
 * = {lo, hi} of the canonical 2k-bit code and d_minhash[g] = the minimum over
 * the window's k-m+1 m-mers of their score, fmix32(lo32 ^ hi32 ^ seed32) with
 * lo32/hi32 the low and high 32-bit halves of the canonical m-mer code and
 * seed32 the low half of the context's seed (MurmurHash3's 32-bit
 * finalizer).  Entries of invalid windows are unspecified.  Outputs caller-allocated: n_bases,
 * 2*n_bases and n_bases elements. */
int hsk_stage_windows(hsk_ctx* ctx, const char* d_reads, const uint64_t* d_offsets,
                      uint64_t n_reads, uint64_t n_bases, int k, int m, uint8_t* d_valid,
                      uint64_t* d_key, uint64_t* d_minhash, void* stream);

/* Stage S3, supermers scattered into minimizer-hashed buckets (Sec. 2.4,
 * Sec. 3.2; the buckets are the tasks of Sec. 3.4).  A window's bucket is
 * minhash mod n_buckets (n_buckets a power of two, 1..8192); a supermer is a run of consecutive valid
 * windows of one read with equal buckets, cut at most every max_kmers windows
 * (and where the implementation's tiles end).  Outputs: d_bucket_kmers
 * (caller, n_buckets words) = k-mers per bucket; d_bucket_rec (caller,
 * n_buckets + 1 words) = first record of each bucket, last entry = total;
 * *d_records = context-owned device array of *n_records records of
 * *record_words words, grouped by bucket in ascending bucket order. */
int hsk_stage_supermers(hsk_ctx* ctx, const char* d_reads, const uint64_t* d_offsets,
                        uint64_t n_reads, uint64_t n_bases, int k, int m, uint32_t n_buckets,
                        uint64_t* d_bucket_kmers, uint64_t* d_bucket_rec,
                        const uint64_t** d_records, uint64_t* n_records, int* record_words,
                        int* max_kmers, void* stream);

/* Stage S4, LSD radix sort of packed keys (Sec. 3.1: equal k-mers become
 * adjacent).  Sorts n keys of key_words uint64 words (1, or 2 as {lo, hi})
 * in place, ascending, looking only at the low key_bits bits (1..128); the
 * other bits must be zero.  d_keys is 8-byte aligned (16-byte aligned for
 * key_words = 2), else HSK_EINVAL.  Scratch is context-owned. */
int hsk_stage_sort(hsk_ctx* ctx, uint64_t* d_keys, uint64_t n, int key_words, int key_bits,
                   void* stream);

/* Stage S5, linear scan of sorted keys (Sec. 3.1): run lengths, histogram
 * of all runs (as in hsk.h), filter lo <= count <= hi.  d_sorted holds n keys
 * of key_words words in ascending order.  *out receives context-owned device
 * arrays; n_windows = n. */
int hsk_stage_rle(hsk_ctx* ctx, const uint64_t* d_sorted, uint64_t n, int key_words,
                  uint32_t lo, uint32_t hi, void* stream, hsk_result* out);

/* Stage S6, output order: sort n (key, count) pairs by key, ascending, in
 * place (keys of key_words words with key_bits significant bits; counts move
 * with their keys).  Keys must be distinct for the order to be unique.
 * d_keys is 8-byte aligned (16-byte aligned for key_words = 2) and d_counts
 * 4-byte aligned, else HSK_EINVAL. */
int hsk_stage_order(hsk_ctx* ctx, uint64_t* d_keys, uint32_t* d_counts, uint64_t n,
                    int key_words, int key_bits, void* stream);

/* The paper's compact encoding of extension information (Sec. 3.3.2: an
 * item whose read ID and position both differ from the previous item's by
 * a value that fits an int8 is sent as the two differences, else in full;
 * a flag byte per item says which).  The stream of n items (d_read[i],
 * d_pos[i]) becomes bytes at d_out (out_cap >= 9 n): per item a flag byte
 * (1 = deltas, 0 = full), then either two int8 differences from the previous
 * item, or the uint32 read and uint32 position, little endian.  Items are
 * cut into chunks of HSK_EXT_CHUNK; a chunk's first item is always full and
 * d_chunk_off[c] (ceil(n / HSK_EXT_CHUNK) entries, written) is its byte
 * offset, so chunks decode independently.  *n_bytes receives the stream's
 * length.  hsk_stage_ext_decode is the inverse; HSK_EINVAL for a malformed
 * stream.  Device pointers; ordered on `stream`, complete on return. */
#define HSK_EXT_CHUNK 1024
int hsk_stage_ext_encode(hsk_ctx* ctx, const uint32_t* d_read, const uint32_t* d_pos, uint64_t n, uint8_t* d_out,
                         uint64_t out_cap, uint64_t* d_chunk_off, uint64_t* n_bytes, void* stream);
int hsk_stage_ext_decode(hsk_ctx* ctx, const uint8_t* d_in, uint64_t n_bytes, const uint64_t* d_chunk_off, uint64_t n,
                         uint32_t* d_read, uint32_t* d_pos, void* stream);

/* Stage S4's key sort for callers that cannot allocate device memory (the
 * paper has no counterpart: this serves callers of this library, not the
 * method).  Such callers are, for example, processes whose device memory is
 * all reserved up front by another allocator (a framework's caching allocator,
 * a fixed arena), or code that must not take the device-wide synchronization
 * cudaMalloc/cudaFree can imply.  Sorts n keys of key_words words (1, or 2 as
 * {lo, hi}) in place, ascending, on the low key_bits bits (the others must be
 * zero), with the same result as hsk_stage_sort, and calls no allocating
 * routine.  Its scratch is one fixed array of about 9.2 MB that every GPU
 * loading this library holds until the process exits; n may be at most
 * HSK_NOALLOC_MAX_KEYS_U64 (key_words = 1) or HSK_NOALLOC_MAX_KEYS_U128
 * (key_words = 2), larger n returns HSK_EOVERFLOW and does nothing.  The
 * first call on a device (with that device current) looks up the array's
 * device address and keeps it for the life of the process; after a
 * cudaDeviceReset that address is stale, so the entry point must not be
 * called again.  All calls share the array, so calls that overlap on the GPU
 * (other streams, other host threads) race.  No context is needed.  The call
 * is synchronous: the work is ordered on `stream` and the call reads the
 * result status back and synchronizes `stream` before it returns, so it
 * cannot be called while `stream` is being captured into a CUDA graph.
 * d_keys must be 8-byte aligned for key_words = 1 (it need not be 16-byte
 * aligned) and 16-byte aligned for key_words = 2.  Returns HSK_EINVAL for bad
 * arguments (a misaligned d_keys included), HSK_ETIMEOUT as elsewhere, and HSK_ECUDA when a CUDA call or
 * launch of this call fails -- or, without doing anything, when a launch
 * error from the caller's earlier work is still pending (it is not
 * cleared). */
#define HSK_NOALLOC_MAX_KEYS_U64 (1u << 20)
#define HSK_NOALLOC_MAX_KEYS_U128 (1u << 19)
int hsk_sort_keys_noalloc(uint64_t* d_keys, uint64_t n, int key_words, int key_bits, void* stream);

/* Test and diagnostic hooks.  hsk_debug_fail_alloc_after(ctx, n): the n-th following device
 * allocation of the context fails as if the budget were exhausted (-1 turns
 * this off), to check that every caller returns HSK_ENOMEM cleanly.
 * hsk_debug_allocated: bytes of device memory the context holds now. */
int hsk_debug_fail_alloc_after(hsk_ctx* ctx, int n);
uint64_t hsk_debug_allocated(hsk_ctx* ctx);
/* Keys of the context's last counting call that did not fit the on-chip
 * sort and went through the global radix passes instead (0 when none). */
uint64_t hsk_debug_last_overflow(hsk_ctx* ctx);
/* Failure detection without a GPU fault: runs the decoupled look-back wait
 * that the scans and radix passes use, on a predecessor status word that
 * nothing ever publishes, giving up after spin_limit polls (1 .. 2^24).
 * Returns HSK_ETIMEOUT once the wait has given up and the kernel returned;
 * the context stays usable. */
int hsk_debug_wait_timeout(hsk_ctx* ctx, uint32_t spin_limit);

/* Packing of the batched and served forms: *passes = packed passes run so
 * far on this context (each counts several small jobs of one k, m and
 * filter together), *sets = jobs they held, *alone = jobs among those that a
 * pass could not finish (a sub-segment too large for the on-chip sort) and
 * that were then counted alone.  NULL outputs are skipped. */
int hsk_debug_pack_stats(hsk_ctx* ctx, uint64_t* passes, uint64_t* sets, uint64_t* alone);
/* Packed passes that failed as a whole (their jobs were then counted alone,
 * so results are unaffected): *failed_passes (may be NULL) receives their
 * number, the return value the last one's reason ("" if none; owned by the
 * context, valid until the next failure). */
const char* hsk_debug_pack_failure(hsk_ctx* ctx, uint64_t* failed_passes);

/* Self-check of the host block pool that holds the batched and served forms'
 * results (size classes, best-fit reuse, the cap on kept blocks, arrays
 * returning their blocks).  Host memory only: no device call is made.
 * Returns 0, or the number of the first check that failed. */
int hsk_debug_host_pool_check(void);

/* Profiling hooks.  When enabled, each counting call on the context records
 * CUDA events on its own stream at the boundaries of its stages and adds the
 * device time between them to per-stage totals:
 *   0 S1 encode, 1 S2 k-mers/minimizers + supermer count + bucket scan,
 *   2 S3 supermer scatter, 3 S4 record expansion + digit histograms,
 *   4 S4 radix passes, 5 S5 run-length count/filter/histogram, 6 S6 order.
 * hsk_profile_read copies HSK_N_STAGES totals (ms) and the number of radix-pass
 * launches they include, then clears them when reset != 0.
 * hsk_launch_count: kernels launched by this library in this process so far. */
#define HSK_N_STAGES 7
int hsk_profile_enable(hsk_ctx* ctx, int on);
int hsk_profile_read(hsk_ctx* ctx, double* stage_ms, uint64_t* radix_pass_launches, int reset);
uint64_t hsk_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* HSK_STAGES_H */
