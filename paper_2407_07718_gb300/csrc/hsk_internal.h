// hsk_internal.h -- launch wrappers and parameter blocks shared between the
// kernel translation units and the host runtime.  Not part of the public ABI.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

// Device-side error codes written to the context's error word.
#define HSK_DERR_TIMEOUT 1  // a bounded spin gave up
#define HSK_DERR_BOUNDS 2   // an index check failed (inconsistent counts)
#define HSK_DERR_OFFSETS 3  // read offsets are not monotone / do not match n_bases

// Empty reads of a look-back status word before a wait gives up (with a
// 64 ns back-off after the first 64 reads this bounds a wait to ~1 s).
#define HSK_SPIN_LIMIT (1u << 24)

namespace hsk {

// Kernels launched by this library (all launch_* wrappers add to it).
void count_launch(unsigned n = 1);

// ---- S1 encode ----------------------------------------------------------
void launch_encode(const char* reads, uint64_t n_bases, uint64_t* packed, uint64_t* invalid,
                   uint64_t n_packed_words, uint64_t n_mask_words, cudaStream_t st);
// bases [b0, b1) only (b0 a multiple of 64)
void launch_encode_range(const char* reads, uint64_t n_bases, uint64_t b0, uint64_t b1, uint64_t* packed,
                         uint64_t* invalid, uint64_t n_packed_words, cudaStream_t st);
constexpr uint64_t SM_TILE_BASES = 1024;   // windows per S2 warp tile
constexpr uint64_t SM_TILE_REACH = 1280;   // bases past a tile's start that its walk reads
// warps per CTA of the walk; one bucket-counter table per CTA in shared
// memory, so more warps share it (16: short-read S2 17.9 -> 16.1 ms against 8)
constexpr int SM_CTA_WARPS = 16;
void launch_mark_starts(const uint64_t* offsets, uint64_t n_reads, uint64_t n_bases,
                        uint64_t* start_mask, int* err, cudaStream_t st);

// packed sets: read starts of every set, padding between sets zeroed
void launch_mark_starts_sets(const uint64_t* offsets, const uint64_t* off0, const uint64_t* n_reads,
                             const uint64_t* base, uint32_t n_sets, uint64_t max_reads, char* reads,
                             uint64_t* start_mask, int* err, cudaStream_t st);

// ---- S2/S3 canonical k-mers, minimizers, supermers -------------------------
enum { SM_DESC = 0, SM_DUMP = 2 };

struct SmParams {
    const uint64_t* packed;
    const uint64_t* invalid;
    const uint64_t* start;
    uint64_t n_bases;
    uint64_t n_packed_words, n_mask_words;
    int k, m, w;
    uint32_t seed32;
    int lexical;              // 1: m-mers ordered by their code (lexical), 0: by hash
    uint32_t n_buckets;       // a power of two (one set), or the buckets of all packed sets
    int nmax;                 // k-mers per supermer record at most
    uint32_t nmax_magic;      // ceil(2^32 / nmax): q = umulhi(x, magic) = x / nmax for x < 2^24
    int rec_words;            // 2 (k <= 32) or 4 (k <= 64)
    uint32_t grid;
    uint64_t tile_begin, tile_end;     // warp tiles [begin, end) of 1024 windows (end 0 = all)
    uint64_t* desc;                    // supermer descriptors (DESC)
    uint64_t desc_cap;
    unsigned long long* desc_count;    // descriptors produced (may exceed desc_cap)
    uint32_t* bucket_rec;              // [n_buckets] records per bucket (atomic adds)
    uint64_t* bucket_kmers;            // [n_buckets] k-mers per bucket (atomic adds)
    // Packed sets (n_sets > 0): set s owns warp tiles [set_tile0[s],
    // set_tile0[s + 1]) and buckets set_bucket[s] + (score & set_bmask[s]);
    // every set starts on a tile boundary, so a tile belongs to one set.
    const uint32_t* set_tile0;         // n_sets + 1 entries
    const uint32_t* set_bucket;        // n_sets entries
    const uint32_t* set_bmask;         // n_sets entries (buckets of the set - 1)
    uint32_t n_sets;
    uint8_t* dump_valid;               // (DUMP)
    uint64_t* dump_key;
    uint64_t* dump_minhash;
    int* err;
};

size_t supermer_smem_bytes(int mode, uint32_t n_buckets);
int supermer_max_ctas_per_sm(int mode, bool wide, int nreg, uint32_t n_buckets);
void launch_supermer(int mode, const SmParams& p, cudaStream_t st);
// records from descriptors: bucket_off[B+1] record offsets; cursor[b *
// SCATTER_CURSOR_STRIDE] zeroed for every bucket b.  The cursors take every
// descriptor's atomic: packed into 16 KB they fell into a few L2 slices, and
// 128 bytes apart they spread over all of them (S3 took 6.2 ms packed, 5.35 ms
// spread, on the long-read workload)
constexpr uint32_t SCATTER_CURSOR_STRIDE = 32;
void launch_scatter_desc(const uint64_t* desc, uint64_t n_desc, const uint64_t* packed, int k,
                         const uint64_t* bucket_off, uint32_t* cursor, uint64_t* records, uint64_t n_records,
                         int* err, int grid, cudaStream_t st);

// exclusive scan of n uint32 counts into uint64 offsets; offsets[n] = total.
// Scratch: scan_status_words(n) uint64 words.
uint64_t scan_status_words(uint64_t n);
void launch_scan_u32(const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* status,
                     uint32_t* tile_ctr, uint32_t epoch, int* err, cudaStream_t st);

// ---- S4 sort ---------------------------------------------------------------
// Segment c: records [rec_base[c], rec_base[c+1]) expand to keys
// [key_base[c], key_base[c+1]); hist[c][p][256] receives the segment's digit
// histograms.  tile_ctrs: C zeroed counters; status: C * (max_tiles + 1) words.
uint64_t expand_tiles(uint64_t n_rec);
int expand_grid(int num_sms);
void launch_expand_seg(const uint64_t* records, const uint64_t* rec_base, const uint64_t* key_base,
                       uint32_t C, uint64_t max_tiles, int k, void* keys, uint64_t* status,
                       uint32_t* tile_ctrs, uint32_t epoch, uint64_t* hist, int n_pass, int* err,
                       int grid, cudaStream_t st);

// Digit histograms of plain keys (one segment): hist[p][256].
void launch_digit_hist(const void* keys, int key_words, uint64_t n, uint64_t* hist, int n_pass,
                       int grid, cudaStream_t st);
// Digit histograms of C consecutive segments of plain keys (keys
// [key_base[c], key_base[c+1]) of n): hist[c][p][256], accumulated.
void launch_digit_hist_seg(const void* keys, int key_words, const uint64_t* key_base, uint32_t C, uint64_t n,
                           uint64_t* hist, int n_pass, cudaStream_t st, int shift0 = 0);
// dst[i] = src[idx[i]] for i < n
void launch_gather_u64(const uint64_t* src, const uint64_t* idx, uint32_t n, uint64_t* dst, cudaStream_t st);
// doff[p][c][d] = key_base[c] + exclusive prefix over d of hist[c][p][d]
void launch_digit_offsets_seg(const uint64_t* hist, const uint64_t* key_base, uint64_t* doff, int n_pass,
                              uint32_t C, cudaStream_t st);

// One LSD pass over C segments, optionally carrying uint32 values; doff: this
// pass's [C][256].  Interleaved segments (tile_start == nullptr): tmax = most
// tiles of any segment, status C * tmax * 256 words.  Listed segments:
// segment c owns global tiles [tile_start[c], tile_start[c + 1]), tmax = all
// tiles (tile_start[C]), status tmax * 256 words.
uint64_t onesweep_tile_keys(int key_words);
// S6: counts into / out of the keys' bits from cshift up (cshift = 8 * passes)
void launch_pack_pairs(void* keys, uint32_t* counts, uint64_t n, int key_words, int cshift, bool unpack, int grid,
                       cudaStream_t st);
// status: >= 2 * LB_PAD zeroed words
void launch_debug_wait(uint64_t* status, uint32_t spin_limit, int* err, cudaStream_t st);
void launch_onesweep_seg(const void* kin, void* kout, const uint32_t* vin, uint32_t* vout,
                         const uint64_t* key_base, uint32_t C, uint32_t tmax, const uint32_t* tile_start,
                         int key_words, int shift, const uint64_t* doff, uint64_t* status, uint32_t* tile_ctr,
                         uint32_t epoch, int* err, cudaStream_t st);

// ---- S5 run-length count, filter, histogram -------------------------------
// on-chip sort of sub-segments (k_local.cu)
size_t part_smem_bytes(int mode, int k);
void launch_part(int mode, const uint64_t* records, const uint64_t* rec_base, const uint64_t* tile_base,
                 const uint32_t* tile_seg, uint32_t n_tiles, int k, int shift, uint32_t* tile_ctr,
                 uint32_t* sub_cnt, uint64_t* cursor, const uint64_t* sub_end, void* keys, int* err, int grid,
                 cudaStream_t st);
uint32_t local_cap(int key_words);
uint32_t local_cap_big(int key_words);
// keys a sub-segment may hold in on-chip tier 0 (first pass), 1 or 2
uint32_t local_cap_tier(int key_words, int tier);
// grp_set: set of each group (packed sets; nullptr = one set), statistics
// per set at hist + set * hist_len, max_count[set], n_distinct[set]
void launch_local_sort(const uint64_t* sub_off, const uint32_t* only, uint32_t n_sub, int tier, int shift0,
                       int key_words, void* keys, uint32_t* kcount, uint32_t* kc, uint32_t* ov_list,
                       uint64_t* ov_stats, uint32_t lo, uint32_t hi, uint64_t* hist, uint32_t hist_len,
                       uint32_t* max_count, uint64_t* n_distinct, const uint32_t* grp_set, uint32_t* claim,
                       int* err, int num_sms, cudaStream_t st);
// heavy-hitter sub-segments of 64-bit keys (listed by the first on-chip pass):
// each folded into a shared-memory (k-mer, count) table; too many distinct
// keys -> listed again in ov_list for the global path
void launch_heavy_count(const uint64_t* sub_off, const uint32_t* list, uint32_t n_list, void* keys,
                        uint32_t* kcount, uint32_t* kc, uint32_t* ov_list, uint64_t* ov_stats, uint32_t lo,
                        uint32_t hi, uint64_t* hist, uint32_t hist_len, uint32_t* max_count, uint64_t* n_distinct,
                        const uint32_t* grp_set, uint32_t* claim, int* err, int num_sms, cudaStream_t st);
// n_groups > 0: digit-major output (out_off indexed d * n_groups + g)
void launch_compact(const uint64_t* sub_off, const uint32_t* kc, const uint64_t* out_off, uint32_t n_sub,
                    uint32_t n_groups, int key_words, const void* keys, const uint32_t* kcount, void* out_keys,
                    uint32_t* out_counts, uint64_t out_cap, int* err, int grid, cudaStream_t st);
void launch_transpose_kc(const uint32_t* kc, uint32_t n_groups, uint32_t* kc_t, int grid, cudaStream_t st);
// S6 on chip: sub-range r holds pairs [bounds[r], bounds[r+1]) of (kin, vin)
// that share their key bits from shift up; each is sorted by its key and
// written to the same range of (kout, vout).  A sub-range over
// range_sort_cap() sets *too_big and is skipped.
uint32_t range_sort_cap(int key_words);
void launch_range_sort(const void* kin, const uint32_t* vin, void* kout, uint32_t* vout, const uint64_t* bounds,
                       uint32_t n_ranges, int key_words, int shift, int* too_big, uint32_t* claim, int num_sms,
                       cudaStream_t st);
void launch_ov_gather(const uint64_t* sub_off, const uint32_t* ov_list, uint32_t n_ov, uint64_t* ov_pre,
                      int key_words, const void* keys, void* dst, uint64_t dst_cap, int* err, int grid,
                      cudaStream_t st);

uint64_t rle_tiles(uint64_t n, int key_words);
uint64_t rle_bits_words(uint64_t n);
// Pass 1: head bitmask, per-tile first/last head and kept count of the runs
// closing inside the tile; histogram, max and head count (added into n_heads).
void launch_rle_mark(const void* keys, uint64_t n, int key_words, uint32_t* bits, uint64_t* tile_first,
                     uint64_t* tile_last, uint32_t* tile_keep, uint32_t lo, uint32_t hi, uint64_t* hist,
                     uint32_t hist_len, uint32_t* max_count, uint64_t* n_heads, int grid, cudaStream_t st);
// Pass 2: next[t] = first head after tile t (or n); closes each tile's last run.
void launch_rle_close(const uint64_t* tile_first, const uint64_t* tile_last, uint64_t* next, uint64_t* block_min,
                      uint64_t n_tiles, uint64_t n, uint32_t* tile_keep, uint32_t lo, uint32_t hi, uint64_t* hist,
                      uint32_t hist_len, uint32_t* max_count, cudaStream_t st);
// Pass 3: kept (key, count) pairs at out_off[t] (exclusive scan of tile_keep).
void launch_rle_write(const void* keys, uint64_t n, int key_words, const uint32_t* bits, const uint64_t* next,
                      const uint64_t* out_off, uint32_t lo, uint32_t hi, void* out_keys, uint32_t* out_counts,
                      uint64_t out_cap, int* err, int grid, cudaStream_t st);

// ---- extension information (k_ext.cu) ---------------------------------------
void launch_ext_insert(const void* keys, int key_words, uint64_t n, uint32_t* table, uint32_t mask, int* err,
                       cudaStream_t st);
void launch_ext_scan(const uint64_t* packed, const uint64_t* invalid, const uint64_t* start, uint64_t n_bases, int k,
                     const void* kept, const uint32_t* table, uint32_t mask, bool wide_out, void* out,
                     uint64_t out_cap, uint64_t* cursor, int* err, int grid, cudaStream_t st);
void launch_ext_decode_pos(const void* comp, bool wide, uint64_t n, const uint64_t* offsets, uint64_t n_reads,
                           uint32_t* occ_read, uint32_t* occ_pos, int grid, cudaStream_t st);
uint64_t ext_chunk_items();
void launch_ext_sizes(const uint32_t* rd, const uint32_t* ps, uint64_t n, uint32_t* size, int grid, cudaStream_t st);
void launch_ext_encode(const uint32_t* rd, const uint32_t* ps, uint64_t n, const uint64_t* off, uint8_t* out,
                       int grid, cudaStream_t st);
void launch_ext_chunk_off(const uint64_t* off, uint64_t n, uint64_t* chunk_off, int grid, cudaStream_t st);
void launch_ext_decode(const uint8_t* in, uint64_t n_bytes, uint64_t n, const uint64_t* chunk_off, uint32_t* rd,
                       uint32_t* ps, int* err, int grid, cudaStream_t st);

}  // namespace hsk
