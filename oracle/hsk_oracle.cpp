// hsk_oracle.cpp -- CPU oracle for sorting-based k-mer counting (HySortK,
// arXiv 2407.07718).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the library path may include, link or
// call this file.  It is used by tests/, by the smoke check and by the
// benchmark's CPU-baseline leg.  It shares no code, header or constant table
// with the CUDA path.
//
// Everything here is written for a reader who checks it against the paper by
// eye: no blocking, no fusion, no rolling updates.  Each k-mer and m-mer code
// is recomputed from its bases, one base at a time.
//
//   * oracle_count      -- the plain definition of the counted result
//                          (Sec. 2.1 k-mer counting; Sec. 3.1 sort + linear
//                          scan + frequency filter + histogram).
//   * oracle_count_keys -- count chosen canonical k-mers by direct scan, for
//                          sampled parity at sizes the full oracle cannot hold.
//   * oracle_encode     -- stage reference for the 2-bit encoding (Sec. 2.2).
//   * oracle_windows    -- stage reference for canonical k-mers and hashed
//                          minimizers found by the monotone deque (Sec. 3.2).
//   * oracle_supermers  -- stage reference for supermers and buckets (Sec. 2.4,
//                          Sec. 3.2, Sec. 3.4 tasks).
//   * oracle_sort_u64   -- stage reference for the sort: std::sort (Sec. 3.1).
//   * oracle_count_ext  -- extension information of the kept k-mers: every
//                          occurrence's read and position (Sec. 3.3.2).
//
// Readings of the paper that these functions fix (the paper is silent on them):
//   base code A=0 C=1 G=2 T=3, first base in the most significant bits;
//   canonical = numeric min(forward, reverse complement); any byte other than
//   upper-case A/C/G/T breaks the window; the histogram counts every distinct
//   k-mer before the filter, with bin H-1 collecting counts >= H-1; the filter
//   is inclusive [lo, hi]; output is in ascending key order; the m-mer score is
//   MurmurHash3's 32-bit finalizer applied to (low 32 bits XOR high 32 bits of
//   the canonical m-mer, XOR the low 32 bits of the seed); the bucket of a
//   window is minhash mod B, the remainder rule of Sec. 3.2.

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

typedef unsigned __int128 u128;

struct u128_hasher {
    size_t operator()(const u128& v) const noexcept {
        return std::hash<uint64_t>()((uint64_t)v) ^ (std::hash<uint64_t>()((uint64_t)(v >> 64)) * 31);
    }
};

// ---------------------------------------------------------------------------
// Base code.  Sec. 2.1 names the four nucleotides; the numeric code is this
// library's reading (A=0, C=1, G=2, T=3; complement of c is 3-c).
// ---------------------------------------------------------------------------
static int base_code(char c) {
    switch (c) {
        case 'A': return 0;
        case 'C': return 1;
        case 'G': return 2;
        case 'T': return 3;
        default: return -1;  // N, lower case, IUPAC, anything else: invalid
    }
}

// Forward code of the len bases at s: sum_j code(s[j]) * 4^(len-1-j).
static u128 forward_code(const char* s, int len) {
    u128 v = 0;
    for (int j = 0; j < len; ++j) v = v * 4 + (u128)base_code(s[j]);
    return v;
}

// Reverse-complement code: sum_j (3 - code(s[len-1-j])) * 4^(len-1-j).
static u128 revcomp_code(const char* s, int len) {
    u128 v = 0;
    for (int j = 0; j < len; ++j) v = v * 4 + (u128)(3 - base_code(s[len - 1 - j]));
    return v;
}

static bool all_acgt(const char* s, int len) {
    for (int j = 0; j < len; ++j)
        if (base_code(s[j]) < 0) return false;
    return true;
}

static u128 canonical_code(const char* s, int len) {
    u128 f = forward_code(s, len), r = revcomp_code(s, len);
    return f < r ? f : r;
}

// MurmurHash3 64-bit finalizer ("fmix64", A. Appleby, public domain), the
// hash-based m-mer score of Sec. 3.2.
static uint64_t fmix64(uint64_t h) {
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdULL;
    h ^= h >> 33;
    h *= 0xc4ceb9fe1a85ec53ULL;
    h ^= h >> 33;
    return h;
}

// MurmurHash3 32-bit finalizer ("fmix32", A. Appleby, public domain).
static uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// Score of an m-mer (Sec. 3.2: a hash value; the lowest score is the
// minimizer): fmix32 of the canonical code folded to 32 bits, XOR the seed.
static uint64_t mmer_score(const char* s, int m, uint64_t seed) {
    uint64_t c = (uint64_t)canonical_code(s, m);
    return fmix32((uint32_t)c ^ (uint32_t)(c >> 32) ^ (uint32_t)seed);
}

// Target of a minimizer (Sec. 3.2): the remainder of its hash value divided
// by the number of targets.
static uint32_t bucket_of(uint64_t minhash, uint32_t n_buckets) {
    return (uint32_t)(minhash % n_buckets);
}

extern "C" {

uint64_t oracle_n_windows(const char* reads, const uint64_t* offsets, uint64_t n_reads, int k);

// Result of oracle_count.  Arrays are malloc'ed here; release with oracle_free.
typedef struct {
    uint64_t n_windows;   // valid k-mer windows (instances counted)
    uint64_t n_distinct;  // distinct canonical k-mers
    uint64_t n_pairs;     // distinct k-mers whose count lies in [lo, hi]
    uint32_t max_count;
    int key_words;        // 1 for k <= 32, 2 for 33 <= k <= 64
    uint64_t* kmers;      // n_pairs * key_words words; 2 words = {lo, hi}
    uint32_t* counts;     // n_pairs
    uint64_t* hist;       // hist_len bins
    uint32_t hist_len;
} oracle_result;

void oracle_free(oracle_result* r) {
    if (!r) return;
    free(r->kmers);
    free(r->counts);
    free(r->hist);
    r->kmers = nullptr;
    r->counts = nullptr;
    r->hist = nullptr;
}

// The counted result, written out as its definition (Sec. 2.1; Sec. 3.1):
// every window of k upper-case ACGT bases inside one read yields its canonical
// code; the codes are sorted so equal k-mers are adjacent; one linear scan
// counts each run, records the histogram of run lengths over all distinct
// k-mers, and keeps (k-mer, count) for lo <= count <= hi.
// Returns 0, or -1 on bad arguments / allocation failure.
int oracle_count(const char* reads, const uint64_t* offsets, uint64_t n_reads, int k,
                 uint32_t lo, uint32_t hi, uint32_t hist_len, oracle_result* out) {
    if (!out || k < 1 || k > 64 || hist_len < 2 || lo > hi) return -1;
    memset(out, 0, sizeof(*out));
    out->key_words = k <= 32 ? 1 : 2;
    out->hist_len = hist_len;

    // 1. enumerate every valid window of every read
    // (storage only: the exact number of windows is reserved up front, so a
    // large input holds 16 bytes per window instead of the up-to-3x of a
    // vector grown by doubling)
    std::vector<u128> keys;
    keys.reserve(oracle_n_windows(reads, offsets, n_reads, k));
    for (uint64_t r = 0; r < n_reads; ++r) {
        const char* s = reads + offsets[r];
        uint64_t len = offsets[r + 1] - offsets[r];
        for (uint64_t i = 0; i + (uint64_t)k <= len; ++i)
            if (all_acgt(s + i, k)) keys.push_back(canonical_code(s + i, k));
    }
    out->n_windows = keys.size();

    // 2. sort: equal k-mers become adjacent
    std::sort(keys.begin(), keys.end());

    // 3. linear scan: run lengths -> histogram, filter, output
    out->hist = (uint64_t*)calloc(hist_len, sizeof(uint64_t));
    if (!out->hist) return -1;
    std::vector<u128> kept;
    std::vector<uint32_t> kept_counts;
    size_t i = 0;
    while (i < keys.size()) {
        size_t j = i;
        while (j < keys.size() && keys[j] == keys[i]) ++j;
        uint64_t c = j - i;
        out->n_distinct += 1;
        if (c > out->max_count) out->max_count = (uint32_t)c;
        out->hist[c < hist_len - 1 ? c : hist_len - 1] += 1;
        if (c >= lo && c <= hi) {
            kept.push_back(keys[i]);
            kept_counts.push_back((uint32_t)c);
        }
        i = j;
    }
    out->n_pairs = kept.size();
    size_t nw = kept.size() * (size_t)out->key_words;
    out->kmers = (uint64_t*)malloc((nw ? nw : 1) * sizeof(uint64_t));
    out->counts = (uint32_t*)malloc((kept.size() ? kept.size() : 1) * sizeof(uint32_t));
    if (!out->kmers || !out->counts) return -1;
    for (size_t p = 0; p < kept.size(); ++p) {
        out->counts[p] = kept_counts[p];
        if (out->key_words == 1) {
            out->kmers[p] = (uint64_t)kept[p];
        } else {
            out->kmers[2 * p] = (uint64_t)kept[p];
            out->kmers[2 * p + 1] = (uint64_t)(kept[p] >> 64);
        }
    }
    return 0;
}

// Count the occurrences of n_query given canonical k-mers (key_words words
// each, ascending, distinct) by scanning every window of every read; also
// returns the number of valid windows.  Same definition as oracle_count, for
// sampled parity on inputs too large to sort on the host.  The scan is split
// over n_threads host threads by read ranges; each thread writes its own
// count array, and the arrays are summed.
int oracle_count_keys(const char* reads, const uint64_t* offsets, uint64_t n_reads, int k,
                      const uint64_t* query, uint64_t n_query, int n_threads,
                      uint64_t* counts_out, uint64_t* n_windows_out) {
    if (k < 1 || k > 64 || n_threads < 1) return -1;
    int kw = k <= 32 ? 1 : 2;
    std::unordered_map<u128, uint64_t, u128_hasher> index;
    index.reserve(n_query * 2 + 1);
    for (uint64_t q = 0; q < n_query; ++q) {
        u128 v = query[q * kw];
        if (kw == 2) v |= (u128)query[q * kw + 1] << 64;
        index[v] = q;
    }
    std::vector<std::vector<uint64_t>> part(n_threads, std::vector<uint64_t>(n_query, 0));
    std::vector<uint64_t> part_windows(n_threads, 0);
    std::vector<std::thread> pool;
    for (int t = 0; t < n_threads; ++t) {
        pool.emplace_back([&, t]() {
            uint64_t r0 = n_reads * t / n_threads, r1 = n_reads * (t + 1) / n_threads;
            for (uint64_t r = r0; r < r1; ++r) {
                const char* s = reads + offsets[r];
                uint64_t len = offsets[r + 1] - offsets[r];
                for (uint64_t i = 0; i + (uint64_t)k <= len; ++i) {
                    if (!all_acgt(s + i, k)) continue;
                    part_windows[t] += 1;
                    auto it = index.find(canonical_code(s + i, k));
                    if (it != index.end()) part[t][it->second] += 1;
                }
            }
        });
    }
    for (auto& th : pool) th.join();
    uint64_t nw = 0;
    for (int t = 0; t < n_threads; ++t) nw += part_windows[t];
    for (uint64_t q = 0; q < n_query; ++q) {
        uint64_t c = 0;
        for (int t = 0; t < n_threads; ++t) c += part[t][q];
        counts_out[q] = c;
    }
    if (n_windows_out) *n_windows_out = nw;
    return 0;
}

// Stage reference, 2-bit encoding (Sec. 2.2 "encode the sequences"): per base
// its code (invalid bases read as 0) and an invalid flag.
void oracle_encode(const char* reads, uint64_t n_bases, uint8_t* code_out, uint8_t* invalid_out) {
    for (uint64_t i = 0; i < n_bases; ++i) {
        int c = base_code(reads[i]);
        code_out[i] = (uint8_t)(c < 0 ? 0 : c);
        invalid_out[i] = (uint8_t)(c < 0);
    }
}

// Number of valid windows (the size oracle_windows will fill).
uint64_t oracle_n_windows(const char* reads, const uint64_t* offsets, uint64_t n_reads, int k) {
    uint64_t n = 0;
    for (uint64_t r = 0; r < n_reads; ++r) {
        const char* s = reads + offsets[r];
        uint64_t len = offsets[r + 1] - offsets[r];
        for (uint64_t i = 0; i + (uint64_t)k <= len; ++i)
            if (all_acgt(s + i, k)) ++n;
    }
    return n;
}

// Hash-scored minimizers of one read (Sec. 3.2).  For every valid window of
// the read, in position order, appends its start (relative to the read), its
// canonical key and the minimum m-mer score over its k-m+1 m-mers, with the
// m-mer position that holds it.  The minimum is found with the paper's
// monotone deque, run over each maximal stretch of ACGT bases: when the
// window slides, (a) an entry whose m-mer has left the window is removed from
// the front, and (b) before a new m-mer is appended, entries at the back whose
// score is not lower than the new score are removed; the front then holds the
// window's minimizer.  Ties keep the right-most m-mer, as rule (b) implies.
struct window_rec {
    uint64_t pos;
    u128 key;
    uint64_t minhash;
    uint64_t minpos;
};

static void windows_of_read(const char* s, uint64_t len, int k, int m, uint64_t seed,
                            std::vector<window_rec>& out) {
    int w = k - m + 1;
    uint64_t a = 0;
    while (a < len) {
        while (a < len && base_code(s[a]) < 0) ++a;  // skip invalid bases
        uint64_t b = a;
        while (b < len && base_code(s[b]) >= 0) ++b;  // [a, b) is all ACGT
        if (b - a >= (uint64_t)k) {
            std::deque<std::pair<uint64_t, uint64_t>> dq;  // (score, m-mer position)
            for (uint64_t q = a; q + (uint64_t)m <= b; ++q) {
                uint64_t sc = mmer_score(s + q, m, seed);
                while (!dq.empty() && dq.back().first >= sc) dq.pop_back();  // rule (b)
                dq.emplace_back(sc, q);
                if (q + 1 < a + (uint64_t)w) continue;  // first window not complete yet
                uint64_t p = q + 1 - (uint64_t)w;        // window start
                if (p + (uint64_t)k > b) break;
                while (dq.front().second < p) dq.pop_front();  // rule (a)
                out.push_back({p, canonical_code(s + p, k), dq.front().first, dq.front().second});
            }
        }
        a = b;
    }
}

// Stage reference for canonical k-mers and minimizers over all reads.  Writes,
// per valid window in read order then position order: global start position,
// canonical key as 2 words {lo, hi} (hi = 0 for k <= 32), minimum m-mer score
// and the global position of the m-mer holding it.  Returns the window count.
uint64_t oracle_windows(const char* reads, const uint64_t* offsets, uint64_t n_reads, int k,
                        int m, uint64_t seed, uint64_t* pos_out, uint64_t* key_out,
                        uint64_t* minhash_out, uint64_t* minpos_out) {
    uint64_t n = 0;
    std::vector<window_rec> ws;
    for (uint64_t r = 0; r < n_reads; ++r) {
        ws.clear();
        windows_of_read(reads + offsets[r], offsets[r + 1] - offsets[r], k, m, seed, ws);
        for (const window_rec& x : ws) {
            pos_out[n] = offsets[r] + x.pos;
            key_out[2 * n] = (uint64_t)x.key;
            key_out[2 * n + 1] = (uint64_t)(x.key >> 64);
            minhash_out[n] = x.minhash;
            if (minpos_out) minpos_out[n] = offsets[r] + x.minpos;
            ++n;
        }
    }
    return n;
}

// Stage reference, supermers and buckets (Sec. 2.4; Sec. 3.2; tasks of
// Sec. 3.4).  A window's bucket is minhash mod n_buckets, the remainder of the
// minimizer's hash divided by the number of targets (Sec. 3.2).  A supermer is a maximal run of windows of one read that start at consecutive
// positions and have equal buckets; its overlapping bases are stored once.
// Writes, per supermer in read order: global start position, number of
// k-mers, bucket; and per bucket its number of k-mers.  Returns the number of
// supermers.
uint64_t oracle_supermers(const char* reads, const uint64_t* offsets, uint64_t n_reads, int k,
                          int m, uint64_t seed, uint32_t n_buckets, uint64_t* sm_pos_out,
                          uint32_t* sm_nkmers_out, uint32_t* sm_bucket_out,
                          uint64_t* bucket_kmers_out) {
    for (uint32_t b = 0; b < n_buckets; ++b) bucket_kmers_out[b] = 0;
    uint64_t ns = 0;
    std::vector<window_rec> ws;
    for (uint64_t r = 0; r < n_reads; ++r) {
        ws.clear();
        windows_of_read(reads + offsets[r], offsets[r + 1] - offsets[r], k, m, seed, ws);
        size_t i = 0;
        while (i < ws.size()) {
            uint32_t bk = bucket_of(ws[i].minhash, n_buckets);
            size_t j = i + 1;
            while (j < ws.size() && ws[j].pos == ws[j - 1].pos + 1 &&
                   bucket_of(ws[j].minhash, n_buckets) == bk)
                ++j;
            sm_pos_out[ns] = offsets[r] + ws[i].pos;
            sm_nkmers_out[ns] = (uint32_t)(j - i);
            sm_bucket_out[ns] = bk;
            bucket_kmers_out[bk] += j - i;
            ++ns;
            i = j;
        }
    }
    return ns;
}

// Extension information (Sec. 3.3.2): for every kept k-mer, the ID of each
// read it occurs in and its position in that read.  Written out as its
// definition: every valid window yields (canonical key, read, position);
// the triples are sorted, so the occurrences of one k-mer are adjacent and in
// (read, position) order; each run whose length lies in [lo, hi] is kept.
// Outputs (caller-allocated, sized by a first call with out arrays NULL that
// returns the counts): *n_pairs kept k-mers with their counts as in
// oracle_count, occ_read/occ_pos the kept k-mers' occurrences k-mer after
// k-mer (the count of a k-mer is the length of its list).  Returns the
// number of occurrences of kept k-mers, or -1 on bad arguments.
int64_t oracle_count_ext(const char* reads, const uint64_t* offsets, uint64_t n_reads, int k, uint32_t lo,
                         uint32_t hi, uint64_t* n_pairs, uint64_t* kmers_out, uint32_t* counts_out,
                         uint32_t* occ_read, uint32_t* occ_pos) {
    if (k < 1 || k > 64 || lo > hi || !n_pairs) return -1;
    struct occ {
        u128 key;
        uint64_t read, pos;
    };
    std::vector<occ> all;
    all.reserve(oracle_n_windows(reads, offsets, n_reads, k));
    for (uint64_t r = 0; r < n_reads; ++r) {
        const char* s = reads + offsets[r];
        uint64_t len = offsets[r + 1] - offsets[r];
        for (uint64_t i = 0; i + (uint64_t)k <= len; ++i)
            if (all_acgt(s + i, k)) all.push_back({canonical_code(s + i, k), r, i});
    }
    std::sort(all.begin(), all.end(), [](const occ& a, const occ& b) {
        if (a.key != b.key) return a.key < b.key;
        if (a.read != b.read) return a.read < b.read;
        return a.pos < b.pos;
    });
    const int kw = k <= 32 ? 1 : 2;
    uint64_t np = 0, no = 0;
    size_t i = 0;
    while (i < all.size()) {
        size_t j = i;
        while (j < all.size() && all[j].key == all[i].key) ++j;
        const uint64_t c = j - i;
        if (c >= lo && c <= hi) {
            if (kmers_out) {
                kmers_out[np * kw] = (uint64_t)all[i].key;
                if (kw == 2) kmers_out[np * kw + 1] = (uint64_t)(all[i].key >> 64);
                counts_out[np] = (uint32_t)c;
                for (size_t q = i; q < j; ++q) {
                    occ_read[no + (q - i)] = (uint32_t)all[q].read;
                    occ_pos[no + (q - i)] = (uint32_t)all[q].pos;
                }
            }
            ++np;
            no += c;
        }
        i = j;
    }
    *n_pairs = np;
    return (int64_t)no;
}

// Stage reference for the sort alone: std::sort (Sec. 3.1).
void oracle_sort_u64(uint64_t* keys, uint64_t n) { std::sort(keys, keys + n); }

// The finalizers exposed for the tests that pin the score function.
uint64_t oracle_fmix64(uint64_t h) { return fmix64(h); }
uint32_t oracle_fmix32(uint32_t h) { return fmix32(h); }

}  // extern "C"
