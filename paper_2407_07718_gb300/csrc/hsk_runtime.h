// hsk_runtime.h -- host-side state of a context (not part of the public ABI).
#pragma once

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/hsk.h"

#define HSK_N_COUNTERS 16384
#define HSK_SMALL_BYTES (256 + HSK_N_COUNTERS * 4)
#define HSK_MAX_BUCKETS 8192
#ifndef HSK_SEGMENTS
#define HSK_SEGMENTS 256            // bucket groups sorted side by side
#endif
#define HSK_MIN_SEGMENT_KMERS 16384 // smaller jobs use fewer segments

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

struct Encoded {
    const uint64_t* packed = nullptr;
    const uint64_t* invalid = nullptr;
    const uint64_t* start = nullptr;
    uint64_t n_bases = 0, n_pw = 0, n_mw = 0;
};

struct Supermers {
    uint32_t B = 0;
    std::vector<uint64_t> h_bucket_kmers;  // k-mers per bucket
    std::vector<uint64_t> h_bucket_rec;    // first record of each bucket (+ total)
    uint64_t n_records = 0, n_kmers = 0;
    int rec_words = 2, nmax = 0;
    const uint64_t* records = nullptr;
};

struct Output {
    uint64_t n_pairs = 0;
    uint64_t n_distinct = 0;
};

struct DevResult {
    uint64_t n_pairs;
    const uint64_t* kmers;
    const uint32_t* counts;
    const uint64_t* hist;
    uint32_t hist_len;
    int key_words;
    uint64_t n_windows, n_distinct;
    uint32_t max_count, n_chunks;
    uint64_t n_supermers;
    double device_ms;
};

// Host blocks for the results the batched and served forms hand out.  Each
// job's arrays are filled by device copies and held by the caller until its
// ticket is released (or the next batch); freshly allocated pageable memory
// would be faulted in page by page during that copy, and a new pinned block
// costs a slow pinning call, so released blocks are kept and reused by later
// jobs.  Blocks are pinned up to pin_cap bytes in total, pageable beyond;
// at most keep_cap bytes of free blocks are kept.
struct HostPool {
    size_t pin_cap = (size_t)8 << 30;
    size_t keep_cap = (size_t)16 << 30;
    struct Block {
        void* p;
        bool pinned;
    };
    std::mutex mu;
    std::multimap<size_t, Block> free_blocks;  // capacity (bytes) -> block
    size_t pinned_total = 0, free_total = 0;
    // size classes: multiples of the smallest power of two (>= 64 KiB) above
    // b / 16, so a block exceeds the request by less than b / 8
    static size_t round_up(size_t b) {
        size_t step = (size_t)64 << 10;
        while (step * 16 <= b) step *= 2;
        return (b + step - 1) / step * step;
    }
    // the smallest free block of at least `bytes`, else a new one
    void* get(size_t bytes, size_t* cap, bool* pinned) {
        const size_t want = round_up(bytes);
        {
            std::lock_guard<std::mutex> g(mu);
            auto it = free_blocks.lower_bound(want);
            if (it != free_blocks.end()) {
                *cap = it->first;
                *pinned = it->second.pinned;
                void* p = it->second.p;
                free_total -= it->first;
                free_blocks.erase(it);
                return p;
            }
        }
        bool pin = false;
        {
            std::lock_guard<std::mutex> g(mu);
            if (pinned_total + want <= pin_cap) {
                pinned_total += want;
                pin = true;
            }
        }
        void* p = nullptr;
        if (pin && cudaMallocHost(&p, want) != cudaSuccess) {
            cudaGetLastError();  // a failed pin is not an error of the call
            p = nullptr;
            std::lock_guard<std::mutex> g(mu);
            pinned_total -= want;
            pin = false;
        }
        if (!p) p = new unsigned char[want];
        *cap = want;
        *pinned = pin;
        return p;
    }
    void put(void* p, size_t cap, bool pinned) {
        {
            std::lock_guard<std::mutex> g(mu);
            if (free_total + cap <= keep_cap) {
                free_blocks.emplace(cap, Block{p, pinned});
                free_total += cap;
                return;
            }
            if (pinned) pinned_total -= cap;
        }
        if (pinned) cudaFreeHost(p);
        else delete[] static_cast<unsigned char*>(p);
    }
    ~HostPool() {
        for (auto& kv : free_blocks) {
            if (kv.second.pinned) cudaFreeHost(kv.second.p);
            else delete[] static_cast<unsigned char*>(kv.second.p);
        }
    }
};

// Host array whose elements are left uninitialised on resize: a device copy
// fills them at once, so zero-filling hundreds of MB first would be wasted.
// A pinned array (page-locked, grown only) takes device copies at link speed
// and keeps its pages from call to call; if pinning fails it falls back to
// ordinary memory.  An array with a pool takes its block from the pool and
// gives it back when released.
template <class T>
struct HostArr {
    T* p = nullptr;
    size_t n = 0, cap = 0;
    bool pinned = false, is_pinned = false;
    HostPool* pool = nullptr;
    HostArr() = default;
    HostArr(const HostArr&) = delete;
    HostArr& operator=(const HostArr&) = delete;
    HostArr(HostArr&& o) noexcept { take(o); }
    HostArr& operator=(HostArr&& o) noexcept {
        if (this != &o) {
            release();
            take(o);
        }
        return *this;
    }
    ~HostArr() { release(); }
    void take(HostArr& o) {
        p = o.p;
        n = o.n;
        cap = o.cap;
        pinned = o.pinned;
        is_pinned = o.is_pinned;
        pool = o.pool;
        o.p = nullptr;
        o.n = o.cap = 0;
    }
    void release() {
        if (p) {
            if (pool) pool->put(p, cap * sizeof(T), is_pinned);
            else if (is_pinned) cudaFreeHost(p);
            else delete[] p;
        }
        p = nullptr;
        cap = 0;
        is_pinned = false;
    }
    void resize(size_t m) {
        if (m > cap) {
            release();
            if (pool) {
                size_t bytes = 0;
                bool pin = false;
                p = static_cast<T*>(pool->get(m * sizeof(T), &bytes, &pin));
                is_pinned = pin;
                cap = bytes / sizeof(T);
                n = m;
                return;
            }
            void* q = nullptr;
            if (pinned && cudaMallocHost(&q, m * sizeof(T)) == cudaSuccess) {
                p = static_cast<T*>(q);
                is_pinned = true;
            } else {
                cudaGetLastError();  // a failed pin is not an error of the call
                p = new T[m];
            }
            cap = m;
        }
        n = m;
    }
    T* data() { return p; }
    const T* data() const { return p; }
    size_t size() const { return n; }
};

struct HostResult {
    DevResult R{};
    HostArr<uint64_t> kmers;
    HostArr<uint32_t> counts;
    HostArr<uint64_t> hist;
    void set_pinned(bool on) { kmers.pinned = counts.pinned = hist.pinned = on; }
    void set_pool(HostPool* p) { kmers.pool = counts.pool = hist.pool = p; }
};

struct ServeState;  // served form (hsk_serve.cu)

// Input copied to the device in chunks on a copy stream while S1/S2 run on
// the chunks already there (host-input counting).  issue(i) enqueues chunk
// i's copy and records ev[i]; chunk bounds are multiples of 65536 bases.
#define HSK_MAX_PIPE 8
struct InputPipe {
    int n = 0, issued = 0;
    uint64_t bound[HSK_MAX_PIPE + 1] = {0};
    cudaEvent_t ev[HSK_MAX_PIPE] = {};
    const char* h_reads = nullptr;
    char* d_reads = nullptr;
    cudaStream_t cs = nullptr;
    cudaError_t issue(int i) {
        cudaError_t e = cudaMemcpyAsync(d_reads + bound[i], h_reads + bound[i], bound[i + 1] - bound[i],
                                        cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ev[i], cs);
        return e;
    }
};

struct hsk_ctx {
    hsk_config cfg{};
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cstream = nullptr;  // input copies of host-input counting
    cudaStream_t hstream = nullptr;  // highest priority: a serving slot's jobs too large to pack
    cudaEvent_t pipe_ev[HSK_MAX_PIPE] = {};
    cudaStream_t zst = nullptr;  // stream of the call in progress (orders zero-fills)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::string err_msg;
    size_t budget = 0, allocated = 0;
    int fail_alloc_after = -1;

    // small device scalars: error word, max count, run count, kept count, tile counters
    void* small = nullptr;
    int* d_err = nullptr;
    uint32_t* d_max = nullptr;
    uint64_t* d_nheads = nullptr;
    uint64_t* d_nout = nullptr;
    uint64_t* d_ndesc = nullptr;
    uint64_t* d_nlocal = nullptr;   // distinct k-mers counted on chip
    uint64_t* d_ovstats = nullptr;  // per on-chip step: [2i] low half = sub-segments it listed, [2i+1] their keys
    int* d_flag = nullptr;          // S6: a sub-range was over the on-chip capacity
    uint32_t* counters = nullptr;
    uint32_t ctr_used = 0;
    uint32_t epoch = 0;

    // device arena
    DevBuf in_reads, in_offsets;     // staged host inputs
    DevBuf pk, iv, rs;               // S1 packed bases, invalid mask, read-start mask
    DevBuf cta_cnt, cta_off, bucket_kmers, bucket_rec, records;  // S2/S3
    DevBuf keys, alt, pass_hist, digit_off, lb_status, seg;        // S4
    DevBuf heads, rle_tiles, out_keys, out_counts, hist;           // S5
    DevBuf pair_alt_keys, pair_alt_counts;                         // S6
    DevBuf loc_tab;                                                // on-chip path: sub-segment tables
    DevBuf batch_a, batch_b, batch_c, batch_d;                     // on-chip path: overflow keys, tile map
    DevBuf pack_tab, pack_stat;                                    // packed sets: set tables, per-set statistics
    DevBuf ext_tab, ext_occ;                                       // extension information: key table, occurrence arrays
    DevBuf s6_bounds;                                              // S6: where each top digit's kept pairs start
    bool s6_digit_major = false;                                   // the output holds only digit-major pairs

    // tuned parameters (0 = built-in default); see hsk_tune.cu
    struct Tune {
        uint32_t group_div = 0;          // bucket-group keys = 256 x on-chip capacity / group_div (default 3)
        uint32_t plain_bucket_shift = 0; // large plain jobs use (4096 or 8192) >> shift buckets
        uint64_t pack_bases = 0;         // bases of one pack at most (default 2^28)
        uint64_t pack_small = 0;         // sets with more bases run alone (default 2^28)
        int slots = 0;                   // serving slots (default 4)
    } tune;
    std::mutex tune_mu;
    std::string tune_path;               // cache file of tuned parameters ("" = none)
    std::vector<std::pair<std::string, Tune>> tuned;  // (class key, parameters)
    bool tuning = false;                 // hsk_autotune is running its trials

    void* h_pin = nullptr;
    size_t h_pin_cap = 0;

    HostPool result_pool;                // host blocks of batched and served results (outlives them)
    HostResult host_res;                 // result of the last hsk_count
    HostArr<uint64_t> ext_off;           // occurrence lists of the last hsk_count_ext
    HostArr<uint32_t> ext_read, ext_pos;
    std::vector<HostResult> batch_res;   // results of the last hsk_count_batch

    ServeState* serve = nullptr;
    // packed passes run for this context's batched and served jobs, the sets
    // they held, and the sets among them counted again alone
    std::atomic<uint64_t> pack_passes{0}, pack_sets{0}, pack_redo{0};
    std::atomic<uint64_t> pack_fail{0};  // passes that failed as a whole (their sets were counted alone)
    std::string pack_fail_msg;           // the last such failure's reason (under tune_mu)

    // profiling: events at stage boundaries (stage id of the span that ends there)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, int>> marks;  // (event index, stage id; -1 = start)
    double prof_ms[8] = {0};
    uint64_t prof_passes = 0;
    uint64_t last_ov_keys = 0;  // keys of the last job that did not fit the on-chip sort

    std::vector<DevBuf*> all_bufs() {
        return {&in_reads, &in_offsets, &pk, &iv, &rs, &cta_cnt, &cta_off, &bucket_kmers,
                &bucket_rec, &records, &keys, &alt, &pass_hist, &digit_off, &lb_status, &seg, &heads, &rle_tiles,
                &out_keys, &out_counts, &hist, &pair_alt_keys, &pair_alt_counts, &loc_tab, &batch_a,
                &batch_b, &batch_c, &batch_d, &pack_tab, &pack_stat, &ext_tab, &ext_occ, &s6_bounds};
    }
};

// Packed sets of one pass (device arrays; see SmParams): set s owns warp
// tiles [tile0[s], tile0[s + 1]) and buckets bucket[s] .. bucket[s] + bmask[s].
struct SetMap {
    const uint32_t* tile0 = nullptr;
    const uint32_t* bucket = nullptr;
    const uint32_t* bmask = nullptr;
    uint32_t n = 0;
};

void hsk_set_error(hsk_ctx* c, const char* fmt, ...);

// CUDA call / library call checks for functions with an hsk_ctx* c in scope
#define CK(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            hsk_set_error(c, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),        \
                          __FILE__, __LINE__);                                              \
            return HSK_ECUDA;                                                               \
        }                                                                                   \
    } while (0)

#define TRY(x)                      \
    do {                            \
        int rc_ = (x);              \
        if (rc_ != HSK_OK) return rc_; \
    } while (0)

// A named NVTX range over a scope (a profiler groups the scope's launches
// under the name; without a profiler attached the calls do nothing).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Runs the body of a C entry point so that no C++ exception crosses the C
// boundary: a failed host allocation returns HSK_ENOMEM, anything else
// HSK_ECUDA, with the reason in the context's error text (when there is one).
template <class F>
int hsk_guarded(hsk_ctx* c, F&& body) {
    try {
        return body();
    } catch (const std::bad_alloc&) {
        if (c) hsk_set_error(c, "host memory allocation failed");
        return HSK_ENOMEM;
    } catch (const std::exception& e) {
        if (c) hsk_set_error(c, "host exception: %s", e.what());
        return HSK_ECUDA;
    } catch (...) {
        if (c) hsk_set_error(c, "unknown host exception");
        return HSK_ECUDA;
    }
}
int hsk_ensure(hsk_ctx* c, DevBuf& b, size_t bytes, bool zero_new);
int hsk_ensure_status(hsk_ctx* c, uint64_t words, cudaStream_t st);
int hsk_next_epoch(hsk_ctx* c, cudaStream_t st, uint32_t* epoch);
int hsk_next_counter(hsk_ctx* c, cudaStream_t st, uint32_t** ctr);
int hsk_next_counters(hsk_ctx* c, cudaStream_t st, uint32_t n, uint32_t** ctr);
int hsk_read_device_error(hsk_ctx* c, cudaStream_t st, uint32_t* max_count = nullptr);
int hsk_upload_segments(hsk_ctx* c, const std::vector<uint64_t>& key_base, const std::vector<uint64_t>* rec_base,
                        cudaStream_t st);
int hsk_grow_output(hsk_ctx* c, const Output& O, uint64_t need, int key_words, cudaStream_t st);
std::vector<uint32_t> hsk_group_buckets(const Supermers& S, uint32_t b0, uint32_t b1, uint32_t C_want);
int hsk_plan_chunks(hsk_ctx* c, const Supermers& S, int key_words, std::vector<std::pair<uint32_t, uint32_t>>& chunks);
int hsk_supermers(hsk_ctx* c, const Encoded& E, int k, int m, uint32_t B, Supermers& S, cudaStream_t st,
                  InputPipe* pipe, const SetMap* sets = nullptr);
uint32_t hsk_pick_buckets(hsk_ctx* c, uint64_t n_bases, int k);
int hsk_plain_sort(hsk_ctx* c, void* keys, uint32_t* vals, uint64_t n, int key_words, int key_bits, DevBuf& alt_keys,
                   DevBuf* alt_vals, cudaStream_t st);
int hsk_local_overflow(hsk_ctx* c, const uint64_t* sub_off, uint32_t n_ov1, uint32_t* ov_list, uint32_t* ov_list_m,
                       uint32_t* ov_list2, uint32_t* ov_list3, int kw, int shift0, void* keys, uint32_t* kcount,
                       uint32_t* kcv, uint32_t lo, uint32_t hi, uint64_t* hist, uint32_t H, uint32_t* d_max,
                       uint64_t* d_distinct, const uint32_t* grp_set, cudaStream_t st, uint32_t** left,
                       uint32_t* n_left, uint64_t* left_keys);
int hsk_run_count(hsk_ctx* c, const char* d_reads, const uint64_t* d_offsets, uint64_t n_reads,
                  uint64_t n_bases, int k, int m, uint32_t lo, uint32_t hi, cudaStream_t st,
                  DevResult& R, InputPipe* pipe = nullptr);
int hsk_count_host_on(hsk_ctx* c, const char* reads, const uint64_t* offsets, uint64_t n_reads,
                      int k, int m, uint32_t lo, uint32_t hi, cudaStream_t st, DevBuf& d_reads,
                      DevBuf& d_offsets, HostResult& HR);
void hsk_serve_shutdown(hsk_ctx* c);
void hsk_serve_set_tune(hsk_ctx* c);  // the context's parameters to its serving slots
// autotuner (hsk_tune.cu)
std::string hsk_tune_class(const hsk_job* jobs, uint32_t n);
void hsk_tune_load(hsk_ctx* c);
bool hsk_tune_lookup(hsk_ctx* c, const std::string& key, hsk_ctx::Tune* out);
void hsk_tune_apply(hsk_ctx* c, const hsk_ctx::Tune& t);
