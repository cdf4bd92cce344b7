// hsk_runtime.cu -- host runtime and C ABI of the k-mer counter.
//
// The context owns a device arena (named buffers grown on demand, all counted
// against an HBM budget), a compute stream and a copy stream, a device error
// word and the look-back bookkeeping (epoch-tagged status words, tile
// counters).  hsk_count_device runs the whole pipeline on one stream:
//
//   S1 encode -> S2 supermer walk (descriptors, per-bucket counts) -> scan
//   -> S3 scatter records into buckets -> plan chunks of buckets under the
//   budget -> per chunk: group buckets, S4 count + scatter keys into
//   (group, top digit) sub-segments, S4/S5 sort and count each sub-segment
//   on chip (k_local.cu; the ones that do not fit go through the 8-bit LSD
//   passes of k_sort.cu and the run scan of k_rle.cu) -> S6 order the kept
//   pairs.  With local_sort = 0 every chunk takes the LSD passes and the run
//   scan.  hsk_count copies large inputs in chunks on the copy stream while
//   S1/S2 run on the chunks already there.
//
// Buckets are the paper's tasks (Sec. 3.4): a k-mer value never lands in two
// of them, so chunks and groups of buckets are sorted and counted
// independently, the way the paper's workers count tasks.  The chunk planner
// plays the role of the paper's memory-aware choice between an out-of-place
// and an in-place sort (Sec. 3.1): it sizes each chunk so its buffers fit the
// budget.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hsk.h"
#include "../../include/hsk_stages.h"
#include "hsk_internal.h"
#include "hsk_runtime.h"

using namespace hsk;

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
void hsk_set_error(hsk_ctx* c, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err_msg = buf;
}


int hsk_ensure(hsk_ctx* c, DevBuf& b, size_t bytes, bool zero_new) {
    if (bytes == 0) bytes = 256;
    if (b.cap >= bytes) return HSK_OK;
    size_t want = (bytes + (2u << 20) - 1) & ~size_t((2u << 20) - 1);  // 2 MiB granules
    if (c->allocated - b.cap + want > c->budget) {
        hsk_set_error(c, "device memory budget exceeded: need %zu more bytes, budget %zu, held %zu",
                      want - b.cap, c->budget, c->allocated);
        return HSK_ENOMEM;
    }
    if (b.p) {
        cudaError_t e = cudaFree(b.p);
        if (e != cudaSuccess) {
            hsk_set_error(c, "cudaFree: %s", cudaGetErrorString(e));
            return HSK_ECUDA;
        }
        c->allocated -= b.cap;
        b.p = nullptr;
        b.cap = 0;
    }
    if (c->fail_alloc_after >= 0 && c->fail_alloc_after-- == 0) {
        hsk_set_error(c, "injected allocation failure");
        return HSK_ENOMEM;
    }
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        hsk_set_error(c, "cudaMalloc(%zu): %s", want, cudaGetErrorString(e));
        b.p = nullptr;
        return HSK_ENOMEM;
    }
    b.cap = want;
    c->allocated += want;
    if (zero_new) {  // ordered before every later kernel on the call's stream
        e = cudaMemsetAsync(b.p, 0, want, c->zst);
        if (e != cudaSuccess) {
            hsk_set_error(c, "cudaMemsetAsync: %s", cudaGetErrorString(e));
            return HSK_ECUDA;
        }
    }
    return HSK_OK;
}

static void free_buf(hsk_ctx* c, DevBuf& b) {
    if (b.p) {
        cudaFree(b.p);
        c->allocated -= b.cap;
    }
    b.p = nullptr;
    b.cap = 0;
}

// A fresh epoch for a look-back launch (status words of other launches never
// match).  Epochs run 1..16383; on wrap-around the status buffer is cleared.
int hsk_next_epoch(hsk_ctx* c, cudaStream_t st, uint32_t* epoch) {
    if (++c->epoch > 0x3FFF) {
        c->epoch = 1;
        if (c->lb_status.p) CK(cudaMemsetAsync(c->lb_status.p, 0, c->lb_status.cap, st));
    }
    *epoch = c->epoch;
    return HSK_OK;
}

// A zeroed tile counter for a look-back launch.
int hsk_next_counter(hsk_ctx* c, cudaStream_t st, uint32_t** ctr) {
    if (c->ctr_used >= HSK_N_COUNTERS) {
        CK(cudaMemsetAsync(c->counters, 0, HSK_N_COUNTERS * sizeof(uint32_t), st));
        c->ctr_used = 0;
    }
    *ctr = c->counters + c->ctr_used++;
    return HSK_OK;
}

// Grow the shared look-back status buffer (new memory is zeroed: stale bytes
// could otherwise look like a status word of the current epoch).
int hsk_ensure_status(hsk_ctx* c, uint64_t words, cudaStream_t st) {
    if (c->lb_status.cap >= words * 8) return HSK_OK;
    CK(cudaStreamSynchronize(st));
    return hsk_ensure(c, c->lb_status, words * 8, true);
}

extern "C" int hsk_config_default(hsk_config* cfg) {
    if (!cfg) return HSK_EINVAL;
    memset(cfg, 0, sizeof(*cfg));
    cfg->device = 0;
    cfg->hbm_budget = 0;
    cfg->hist_len = 65536;
    cfg->n_buckets = 0;
    cfg->radix_bits = 8;
    cfg->max_chunk_kmers = 0;
    cfg->seed = 0x9E3779B97F4A7C15ULL;
    cfg->autotune = 1;
    cfg->local_sort = 1;
    return HSK_OK;
}

extern "C" int hsk_create(hsk_ctx** out, const hsk_config* cfg_in) {
    return hsk_guarded(nullptr, [&]() -> int {
        if (!out) return HSK_EINVAL;
        *out = nullptr;
        hsk_config cfg;
        if (cfg_in) cfg = *cfg_in;
        else hsk_config_default(&cfg);
        if (cfg.hist_len < 2 || (cfg.radix_bits != 0 && cfg.radix_bits != 8) || cfg.minimizer_order < 0 ||
            cfg.minimizer_order > 1)
            return HSK_EINVAL;
        if (cfg.n_buckets && (cfg.n_buckets > HSK_MAX_BUCKETS || (cfg.n_buckets & (cfg.n_buckets - 1))))
            return HSK_EINVAL;  // a power of two: the bucket is a mask of the hash
        hsk_ctx* c = new hsk_ctx();
        c->cfg = cfg;
        cudaError_t e = cudaSetDevice(cfg.device);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, cfg.device);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking);
        int prio_least = 0, prio_greatest = 0;
        if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->hstream, cudaStreamNonBlocking, prio_greatest);
        for (int i = 0; i < HSK_MAX_PIPE && e == cudaSuccess; ++i)
            e = cudaEventCreateWithFlags(&c->pipe_ev[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
        size_t free_b = 0, total_b = 0;
        if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
        if (e == cudaSuccess) e = cudaMalloc(&c->small, HSK_SMALL_BYTES);
        if (e == cudaSuccess) e = cudaMemset(c->small, 0, HSK_SMALL_BYTES);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return HSK_ECUDA;
        }
        c->budget = cfg.hbm_budget ? cfg.hbm_budget : (size_t)(free_b * 0.9);
        if (cfg.tune_cache) {
            c->tune_path = cfg.tune_cache;
            c->cfg.tune_cache = nullptr;  // the caller's string is not kept
            hsk_tune_load(c);
        }
        c->host_res.set_pinned(true);  // hsk_count's results: reused from call to call
        c->allocated = HSK_SMALL_BYTES;
        char* s = (char*)c->small;
        c->d_err = (int*)(s + 0);
        c->d_max = (uint32_t*)(s + 8);
        c->d_nheads = (uint64_t*)(s + 16);
        c->d_nout = (uint64_t*)(s + 24);
        c->d_ndesc = (uint64_t*)(s + 32);
        c->d_nlocal = (uint64_t*)(s + 40);
        c->d_ovstats = (uint64_t*)(s + 48);
        c->d_flag = (int*)(s + 112);
        c->counters = (uint32_t*)(s + 256);
        *out = c;
        return HSK_OK;
    });
}

extern "C" void hsk_destroy(hsk_ctx* c) {
    if (!c) return;
    hsk_serve_shutdown(c);
    cudaSetDevice(c->cfg.device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (DevBuf* b : c->all_bufs()) free_buf(c, *b);
    if (c->small) cudaFree(c->small);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->stream) cudaStreamDestroy(c->stream);
    if (c->cstream) {
        cudaStreamSynchronize(c->cstream);
        cudaStreamDestroy(c->cstream);
    }
    if (c->hstream) {
        cudaStreamSynchronize(c->hstream);
        cudaStreamDestroy(c->hstream);
    }
    for (int i = 0; i < HSK_MAX_PIPE; ++i)
        if (c->pipe_ev[i]) cudaEventDestroy(c->pipe_ev[i]);
    if (c->h_pin) cudaFreeHost(c->h_pin);
    delete c;
}

extern "C" const char* hsk_last_error(hsk_ctx* c) { return c ? c->err_msg.c_str() : "null context"; }

extern "C" int hsk_host_pin(void* p, uint64_t bytes) {
    if (!p || bytes == 0) return HSK_EINVAL;
    if (cudaHostRegister(p, (size_t)bytes, cudaHostRegisterDefault) != cudaSuccess) {
        cudaGetLastError();
        return HSK_ECUDA;
    }
    return HSK_OK;
}

extern "C" int hsk_host_unpin(void* p) {
    if (!p) return HSK_EINVAL;
    if (cudaHostUnregister(p) != cudaSuccess) {
        cudaGetLastError();
        return HSK_ECUDA;
    }
    return HSK_OK;
}

// test hook: make the n-th following device allocation fail (-1 = never)
extern "C" int hsk_debug_fail_alloc_after(hsk_ctx* c, int n) {
    if (!c) return HSK_EINVAL;
    c->fail_alloc_after = n;
    return HSK_OK;
}

extern "C" uint64_t hsk_debug_allocated(hsk_ctx* c) { return c ? c->allocated : 0; }
extern "C" uint64_t hsk_debug_last_overflow(hsk_ctx* c) { return c ? c->last_ov_keys : 0; }


// ---------------------------------------------------------------------------
// launch counter and stage profiling
// ---------------------------------------------------------------------------
static std::atomic<uint64_t> g_launches{0};
namespace hsk {
void count_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace hsk

extern "C" uint64_t hsk_launch_count(void) { return g_launches.load(); }

static void prof_mark(hsk_ctx* c, cudaStream_t st, int stage) {
    if (!c->prof) return;
    size_t i = c->marks.size();
    if (i >= c->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        c->ev_pool.push_back(e);
    }
    cudaEventRecord(c->ev_pool[i], st);
    c->marks.emplace_back((int)i, stage);
}

// after the stream is synchronized: add the spans between marks to their stages
static void prof_collect(hsk_ctx* c) {
    if (!c->prof) return;
    for (size_t i = 1; i < c->marks.size(); ++i) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, c->ev_pool[c->marks[i - 1].first], c->ev_pool[c->marks[i].first]) ==
                cudaSuccess &&
            c->marks[i].second >= 0)
            c->prof_ms[c->marks[i].second] += ms;
    }
    c->marks.clear();
}

extern "C" int hsk_profile_enable(hsk_ctx* c, int on) {
    if (!c) return HSK_EINVAL;
    c->prof = on != 0;
    c->marks.clear();
    return HSK_OK;
}

extern "C" int hsk_profile_read(hsk_ctx* c, double* stage_ms, uint64_t* passes, int reset) {
    if (!c) return HSK_EINVAL;
    for (int i = 0; i < HSK_N_STAGES; ++i) {
        if (stage_ms) stage_ms[i] = c->prof_ms[i];
        if (reset) c->prof_ms[i] = 0;
    }
    if (passes) *passes = c->prof_passes;
    if (reset) c->prof_passes = 0;
    return HSK_OK;
}

// ---------------------------------------------------------------------------
// argument checks
// ---------------------------------------------------------------------------
static int check_args(hsk_ctx* c, const void* reads, const void* offsets, uint64_t n_reads, int k,
                      int m, uint32_t lo, uint32_t hi) {
    if (!c) return HSK_EINVAL;
    if (k < 1 || k > 64) {
        hsk_set_error(c, "k=%d outside [1, 64]", k);
        return HSK_EINVAL;
    }
    if (m < 1 || m > k || m > 32) {
        hsk_set_error(c, "m=%d outside [1, min(k, 32)]", m);
        return HSK_EINVAL;
    }
    if (lo > hi) {
        hsk_set_error(c, "filter bounds lo=%u > hi=%u", lo, hi);
        return HSK_EINVAL;
    }
    if (n_reads > 0 && (!reads && !offsets)) {
        hsk_set_error(c, "NULL reads/offsets with n_reads=%llu", (unsigned long long)n_reads);
        return HSK_EINVAL;
    }
    if (n_reads > 0 && !offsets) {
        hsk_set_error(c, "NULL offsets with n_reads=%llu", (unsigned long long)n_reads);
        return HSK_EINVAL;
    }
    return HSK_OK;
}

// Reads the device error word (and the largest count, stored 8 bytes after it)
// once the stream's work is done.
int hsk_read_device_error(hsk_ctx* c, cudaStream_t st, uint32_t* max_count) {
    uint32_t w[3] = {0, 0, 0};
    CK(cudaMemcpyAsync(w, c->d_err, sizeof(w), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int derr = (int)w[0];
    if (max_count) *max_count = w[2];
    if (derr == HSK_DERR_OFFSETS) {
        hsk_set_error(c, "offsets must start at 0, be non-decreasing and end at n_bases");
        return HSK_EINVAL;
    }
    if (derr == HSK_DERR_TIMEOUT) {
        hsk_set_error(c, "a bounded device wait gave up (look-back status never arrived)");
        return HSK_ETIMEOUT;
    }
    if (derr != 0) {
        hsk_set_error(c, "device consistency check failed (code %d)", derr);
        return HSK_ECUDA;
    }
    return HSK_OK;
}

// ---------------------------------------------------------------------------
// pipeline pieces
// ---------------------------------------------------------------------------
int hsk_encode_into(hsk_ctx* c, const char* d_reads, uint64_t n_bases, const uint64_t* d_offsets,
                    uint64_t n_reads, DevBuf& pk, DevBuf& iv, DevBuf& rs, Encoded& E,
                    cudaStream_t st, bool defer_bases) {
    E.n_bases = n_bases;
    E.n_pw = (n_bases + 31) / 32;
    E.n_mw = (n_bases + 63) / 64;
    TRY(hsk_ensure(c, pk, (E.n_pw + 8) * 8, false));
    TRY(hsk_ensure(c, iv, (E.n_mw + 8) * 8, false));
    TRY(hsk_ensure(c, rs, (E.n_mw + 8) * 8, false));
    CK(cudaMemsetAsync((uint64_t*)pk.p + E.n_pw, 0, 8 * 8, st));
    CK(cudaMemsetAsync((uint64_t*)iv.p + E.n_mw, 0, 8 * 8, st));
    CK(cudaMemsetAsync(rs.p, 0, (E.n_mw + 8) * 8, st));
    launch_mark_starts(d_offsets, n_reads, n_bases, (uint64_t*)rs.p, c->d_err, st);
    // with defer_bases the bases are encoded chunk by chunk as they arrive (hsk_supermers)
    if (!defer_bases) launch_encode(d_reads, n_bases, (uint64_t*)pk.p, (uint64_t*)iv.p, E.n_pw, E.n_mw, st);
    CK(cudaGetLastError());
    E.packed = (const uint64_t*)pk.p;
    E.invalid = (const uint64_t*)iv.p;
    E.start = (const uint64_t*)rs.p;
    return HSK_OK;
}

uint32_t hsk_pick_buckets(hsk_ctx* c, uint64_t n_bases, int k) {
    if (c->cfg.n_buckets) return c->cfg.n_buckets;
    // small jobs: fewer buckets keep the per-CTA tables cheap
    if (n_bases < (1ull << 22)) return 256;
    // 4096 buckets for both key widths.  128-bit keys fit half as many per
    // sub-segment, but twice the groups (8192 buckets) measured about 1 ms
    // slower on the short-read workload once the middle on-chip tier took
    // the sub-segments over the first tier's capacity
    (void)k;
    const uint32_t B = 4096;
    return c->tune.plain_bucket_shift ? std::max<uint32_t>(256, B >> c->tune.plain_bucket_shift) : B;
}

static void fill_sm_params(hsk_ctx* c, const Encoded& E, int k, int m, uint32_t B, SmParams& P) {
    memset(&P, 0, sizeof(P));
    P.packed = E.packed;
    P.invalid = E.invalid;
    P.start = E.start;
    P.n_bases = E.n_bases;
    P.n_packed_words = E.n_pw;
    P.n_mask_words = E.n_mw;
    P.k = k;
    P.m = m;
    P.w = k - m + 1;
    P.seed32 = (uint32_t)c->cfg.seed;
    P.lexical = c->cfg.minimizer_order == 1;
    P.n_buckets = B;
    P.rec_words = k <= 32 ? 2 : 4;
    P.nmax = (P.rec_words * 32 - 4) - k + 1;  // bases per record minus (k - 1)
    if (P.nmax > 255) P.nmax = 255;
    P.nmax_magic = (uint32_t)(((1ull << 32) + P.nmax - 1) / P.nmax);
    P.err = c->d_err;
}

// Count supermers per (bucket, CTA), scan to record offsets, scatter records.
// With a set map the bases hold packed sets and B is the buckets of all sets.
static_assert(HSK_MAX_BUCKETS == 8192, "the S2 walk's shared-memory limit is sized for 8192 buckets");
int hsk_supermers(hsk_ctx* c, const Encoded& E, int k, int m, uint32_t B, Supermers& S, cudaStream_t st,
                  InputPipe* pipe, const SetMap* sets) {
    SmParams P;
    fill_sm_params(c, E, k, m, B, P);
    if (sets) {
        P.set_tile0 = sets->tile0;
        P.set_bucket = sets->bucket;
        P.set_bmask = sets->bmask;
        P.n_sets = sets->n;
    }
    const bool wide = k > 32;
    const int nreg = P.w <= 33 ? 2 : 3;
    const int occ = supermer_max_ctas_per_sm(SM_DESC, wide, nreg, B);
    const uint64_t warp_tiles = (E.n_bases + 1023) / 1024;
    uint64_t g = std::min<uint64_t>((uint64_t)c->num_sms * occ, (warp_tiles + SM_CTA_WARPS - 1) / SM_CTA_WARPS);
    P.grid = (uint32_t)std::max<uint64_t>(g, 1);
    TRY(hsk_ensure(c, c->bucket_kmers, (uint64_t)B * 8, false));
    TRY(hsk_ensure(c, c->bucket_rec, ((uint64_t)B + 1) * 8, false));
    // records per bucket, then the bucket cursors of the scatter (spread out)
    const size_t cnt_bytes = (size_t)B * 4 * (1 + SCATTER_CURSOR_STRIDE);
    TRY(hsk_ensure(c, c->cta_cnt, cnt_bytes, false));
    uint32_t* d_rec_cnt = (uint32_t*)c->cta_cnt.p;
    uint32_t* d_cursor = d_rec_cnt + B;
    // descriptors: about 2/(w+1) supermers per window (random minimizers), plus
    // cuts at invalid bases, tile ends and the record cap; re-run if short
    uint64_t cap = std::min<uint64_t>(E.n_bases + 1, (uint64_t)((double)E.n_bases *
                                       (3.0 / (P.w + 1) + 1.0 / P.nmax + 1.0 / 256)) + (1u << 16));
    uint64_t n_desc = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        TRY(hsk_ensure(c, c->cta_off, cap * 8, false));
        CK(cudaMemsetAsync(c->bucket_kmers.p, 0, (size_t)B * 8, st));
        CK(cudaMemsetAsync(d_rec_cnt, 0, cnt_bytes, st));
        CK(cudaMemsetAsync(c->d_ndesc, 0, 8, st));
        P.desc = (uint64_t*)c->cta_off.p;
        P.desc_cap = cap;
        P.desc_count = (unsigned long long*)c->d_ndesc;
        P.bucket_rec = d_rec_cnt;
        P.bucket_kmers = (uint64_t*)c->bucket_kmers.p;
        if (pipe && attempt == 0) {
            // chunk i's bytes arrive on the copy stream: encode them, then walk
            // every tile whose staged bases are now encoded; the next copy is
            // issued before this chunk's work is queued (a pageable copy
            // returns only once staged, and the GPU works meanwhile)
            const uint64_t n_tiles = (E.n_bases + SM_TILE_BASES - 1) / SM_TILE_BASES;
            uint64_t t_done = 0;
            const uint32_t grid = P.grid;
            for (int i = 0; i < pipe->n; ++i) {
                while (pipe->issued < pipe->n && pipe->issued <= i + 1) CK(pipe->issue(pipe->issued++));
                CK(cudaStreamWaitEvent(st, pipe->ev[i], 0));
                launch_encode_range(pipe->d_reads, E.n_bases, pipe->bound[i], pipe->bound[i + 1],
                                    (uint64_t*)E.packed, (uint64_t*)E.invalid, E.n_pw, st);
                const uint64_t b = pipe->bound[i + 1];
                uint64_t t_end = i + 1 == pipe->n ? n_tiles
                                 : (b >= SM_TILE_REACH ? (b - SM_TILE_REACH) / SM_TILE_BASES + 1 : 0);
                if (t_end > n_tiles) t_end = n_tiles;
                if (t_end > t_done) {
                    P.tile_begin = t_done;
                    P.tile_end = t_end;
                    P.grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(grid, (t_end - t_done + SM_CTA_WARPS - 1) / SM_CTA_WARPS));
                    launch_supermer(SM_DESC, P, st);
                    t_done = t_end;
                }
            }
            P.tile_begin = P.tile_end = 0;
            P.grid = grid;
        } else {
            launch_supermer(SM_DESC, P, st);
        }
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&n_desc, c->d_ndesc, 8, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (n_desc <= cap) break;
        cap = n_desc;  // the walk counted every supermer: one more run fits them all
    }
    // record offsets of the buckets
    TRY(hsk_ensure_status(c, scan_status_words(B), st));
    uint32_t ep, *ctr;
    TRY(hsk_next_epoch(c, st, &ep));
    TRY(hsk_next_counter(c, st, &ctr));
    launch_scan_u32(d_rec_cnt, B, (uint64_t*)c->bucket_rec.p, (uint64_t*)c->lb_status.p, ctr, ep, c->d_err, st);
    CK(cudaGetLastError());
    // bucket statistics to the host (needed to size records and plan chunks)
    S.B = B;
    S.h_bucket_kmers.resize(B);
    S.h_bucket_rec.resize((size_t)B + 1);
    CK(cudaMemcpyAsync(S.h_bucket_kmers.data(), c->bucket_kmers.p, (size_t)B * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(S.h_bucket_rec.data(), c->bucket_rec.p, ((size_t)B + 1) * 8, cudaMemcpyDeviceToHost, st));
    TRY(hsk_read_device_error(c, st));
    S.n_records = S.h_bucket_rec[B];
    if (S.n_records != n_desc) {
        hsk_set_error(c, "supermer count mismatch: %llu descriptors, %llu records",
                      (unsigned long long)n_desc, (unsigned long long)S.n_records);
        return HSK_ECUDA;
    }
    S.n_kmers = 0;
    for (uint64_t v : S.h_bucket_kmers) S.n_kmers += v;
    S.rec_words = P.rec_words;
    S.nmax = P.nmax;
    TRY(hsk_ensure(c, c->records, std::max<uint64_t>(S.n_records, 1) * P.rec_words * 8, false));
    prof_mark(c, st, 1);
    launch_scatter_desc((const uint64_t*)c->cta_off.p, n_desc, E.packed, k, (const uint64_t*)c->bucket_rec.p,
                        d_cursor, (uint64_t*)c->records.p, S.n_records, c->d_err, c->num_sms * 8, st);
    CK(cudaGetLastError());
    S.records = (const uint64_t*)c->records.p;
    return HSK_OK;
}

static int n_passes_for(int key_bits) { return (key_bits + 7) / 8; }

// Output capacity for `need` pairs; the pairs already there are kept.
int hsk_grow_output(hsk_ctx* c, const Output& O, uint64_t need, int key_words, cudaStream_t st) {
    const size_t kb = (size_t)key_words * 8;
    if (c->out_keys.cap >= need * kb && c->out_counts.cap >= need * 4) return HSK_OK;
    DevBuf nk, ncn;
    TRY(hsk_ensure(c, nk, need * kb + need * kb / 4, false));
    TRY(hsk_ensure(c, ncn, need * 4 + need, false));
    if (O.n_pairs) {
        CK(cudaMemcpyAsync(nk.p, c->out_keys.p, O.n_pairs * kb, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(ncn.p, c->out_counts.p, O.n_pairs * 4, cudaMemcpyDeviceToDevice, st));
        CK(cudaStreamSynchronize(st));
    }
    free_buf(c, c->out_keys);
    free_buf(c, c->out_counts);
    c->out_keys = nk;
    c->out_counts = ncn;
    return HSK_OK;
}

// C zeroed tile counters in a row for one launch.
int hsk_next_counters(hsk_ctx* c, cudaStream_t st, uint32_t n, uint32_t** ctr) {
    if (n > HSK_N_COUNTERS) {
        hsk_set_error(c, "%u tile counters requested", n);
        return HSK_EINVAL;
    }
    if (c->ctr_used + n > HSK_N_COUNTERS) {
        CK(cudaMemsetAsync(c->counters, 0, HSK_N_COUNTERS * sizeof(uint32_t), st));
        c->ctr_used = 0;
    }
    *ctr = c->counters + c->ctr_used;
    c->ctr_used += n;
    return HSK_OK;
}

// Segment boundaries (C + 1 key offsets, and record offsets when given) to
// the device; the host arrays are copied before the call returns.
int hsk_upload_segments(hsk_ctx* c, const std::vector<uint64_t>& key_base,
                           const std::vector<uint64_t>* rec_base, cudaStream_t st) {
    size_t n = key_base.size();
    TRY(hsk_ensure(c, c->seg, 2 * n * 8, false));
    CK(cudaMemcpyAsync(c->seg.p, key_base.data(), n * 8, cudaMemcpyHostToDevice, st));
    if (rec_base)
        CK(cudaMemcpyAsync((uint64_t*)c->seg.p + n, rec_base->data(), n * 8, cudaMemcpyHostToDevice, st));
    return HSK_OK;
}

// LSD passes over C segments of keys in a (b is scratch of the same size);
// the digit offsets doff[P][C][256] must be ready.  *sorted_in_b tells where
// the result ended.
static int sort_segments(hsk_ctx* c, void* a, void* b, uint32_t* va, uint32_t* vb, const uint64_t* d_key_base,
                         uint32_t C, uint32_t tmax, int key_words, int n_pass, const uint64_t* doff,
                         bool* sorted_in_b, cudaStream_t st) {
    *sorted_in_b = false;
    if (tmax == 0 || n_pass == 0) return HSK_OK;
    TRY(hsk_ensure_status(c, (uint64_t)C * tmax * 256 + 1, st));
    void *src = a, *dst = b;
    uint32_t *vs = va, *vd = vb;
    for (int p = 0; p < n_pass; ++p) {
        uint32_t ep, *ctr;
        TRY(hsk_next_epoch(c, st, &ep));
        TRY(hsk_next_counter(c, st, &ctr));
        launch_onesweep_seg(src, dst, vs, vd, d_key_base, C, tmax, nullptr, key_words, 8 * p, doff + (size_t)p * C * 256,
                            (uint64_t*)c->lb_status.p, ctr, ep, c->d_err, st);
        std::swap(src, dst);
        std::swap(vs, vd);
    }
    CK(cudaGetLastError());
    *sorted_in_b = (n_pass % 2) == 1;
    return HSK_OK;
}

// A plain (one-segment) sort of n keys (with optional values) in place.
int hsk_plain_sort(hsk_ctx* c, void* keys, uint32_t* vals, uint64_t n, int key_words, int key_bits,
                      DevBuf& alt_keys, DevBuf* alt_vals, cudaStream_t st) {
    if (n <= 1) return HSK_OK;
    size_t kb = (size_t)key_words * 8;
    int P = (key_bits + 7) / 8;
    TRY(hsk_ensure(c, alt_keys, n * kb, false));
    if (vals) TRY(hsk_ensure(c, *alt_vals, n * 4, false));
    TRY(hsk_ensure(c, c->pass_hist, 16 * 256 * 8, false));
    TRY(hsk_ensure(c, c->digit_off, 16 * 256 * 8, false));
    std::vector<uint64_t> kb0 = {0, n};
    TRY(hsk_upload_segments(c, kb0, nullptr, st));
    CK(cudaMemsetAsync(c->pass_hist.p, 0, (size_t)P * 256 * 8, st));
    launch_digit_hist(keys, key_words, n, (uint64_t*)c->pass_hist.p, P, c->num_sms * 4, st);
    launch_digit_offsets_seg((uint64_t*)c->pass_hist.p, (const uint64_t*)c->seg.p, (uint64_t*)c->digit_off.p, P,
                             1, st);
    uint32_t tmax = (uint32_t)((n + onesweep_tile_keys(key_words) - 1) / onesweep_tile_keys(key_words));
    bool in_b = false;
    TRY(sort_segments(c, keys, alt_keys.p, vals, vals ? (uint32_t*)alt_vals->p : nullptr,
                      (const uint64_t*)c->seg.p, 1, tmax, key_words, P, (const uint64_t*)c->digit_off.p, &in_b,
                      st));
    if (in_b) {
        CK(cudaMemcpyAsync(keys, alt_keys.p, n * kb, cudaMemcpyDeviceToDevice, st));
        if (vals) CK(cudaMemcpyAsync(vals, alt_vals->p, n * 4, cudaMemcpyDeviceToDevice, st));
    }
    return HSK_OK;
}

// Run-length count, histogram and filter of one sorted chunk; appends the
// kept pairs to the context's output.
int hsk_rle_chunk(hsk_ctx* c, const void* sorted, uint64_t n, int key_words, uint32_t lo,
                  uint32_t hi, uint32_t hist_len, uint64_t* d_hist, Output& O, cudaStream_t st) {
    if (n == 0) return HSK_OK;
    if (n >= 0xFFFFFFFFull) {
        hsk_set_error(c, "a sort chunk of %llu keys exceeds 2^32-1", (unsigned long long)n);
        return HSK_EOVERFLOW;
    }
    const uint64_t nt = rle_tiles(n, key_words), nb = (nt + 1023) / 1024;
    TRY(hsk_ensure(c, c->heads, rle_bits_words(n) * 4, false));
    TRY(hsk_ensure(c, c->rle_tiles, (nt * 8 * 4 + 8) + nt * 4 + nb * 8 + 64, false));
    uint64_t* t_first = (uint64_t*)c->rle_tiles.p;
    uint64_t* t_last = t_first + nt;
    uint64_t* t_next = t_last + nt;
    uint64_t* t_off = t_next + nt;  // nt + 1 entries
    uint32_t* t_keep = (uint32_t*)(t_off + nt + 1);
    uint64_t* b_min = (uint64_t*)(t_keep + ((nt + 1) & ~1ull));
    CK(cudaMemsetAsync(c->d_nheads, 0, 8, st));
    launch_rle_mark(sorted, n, key_words, (uint32_t*)c->heads.p, t_first, t_last, t_keep, lo, hi, d_hist,
                    hist_len, c->d_max, c->d_nheads, c->num_sms * (key_words == 1 ? 4 : 2), st);
    launch_rle_close(t_first, t_last, t_next, b_min, nt, n, t_keep, lo, hi, d_hist, hist_len, c->d_max, st);
    TRY(hsk_ensure_status(c, scan_status_words(nt), st));
    uint32_t ep, *ctr;
    TRY(hsk_next_epoch(c, st, &ep));
    TRY(hsk_next_counter(c, st, &ctr));
    launch_scan_u32(t_keep, nt, t_off, (uint64_t*)c->lb_status.p, ctr, ep, c->d_err, st);
    CK(cudaGetLastError());
    uint64_t D = 0, kept = 0;
    CK(cudaMemcpyAsync(&D, c->d_nheads, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&kept, t_off + nt, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    O.n_distinct += D;
    const size_t kb = (size_t)key_words * 8;
    TRY(hsk_grow_output(c, O, O.n_pairs + kept, key_words, st));
    launch_rle_write(sorted, n, key_words, (const uint32_t*)c->heads.p, t_next, t_off, lo, hi,
                     (char*)c->out_keys.p + O.n_pairs * kb, (uint32_t*)c->out_counts.p + O.n_pairs, kept,
                     c->d_err, c->num_sms * 4, st);
    CK(cudaGetLastError());
    O.n_pairs += kept;
    return HSK_OK;
}

// Order the output pairs by key (stage S6): segments and chunks are groups
// of minimizer buckets, so their pairs come out in bucket order.
// When every count is at most count_max (> 0) and fits the key bits above the
// sort's top digit, the counts ride in those bits and the pairs are sorted as
// keys alone; otherwise the counts move as values.
int hsk_order_pairs(hsk_ctx* c, void* keys, uint32_t* counts, uint64_t n, int key_words,
                    int key_bits, cudaStream_t st, uint32_t count_max) {
    const int cshift = 8 * ((key_bits + 7) / 8);
    const int spare = 64 * key_words - cshift;
    if (n > 1 && count_max > 0 && spare > 0 && spare < 64 && (uint64_t)count_max < (1ULL << spare)) {
        launch_pack_pairs(keys, counts, n, key_words, cshift, false, c->num_sms * 8, st);
        TRY(hsk_plain_sort(c, keys, nullptr, n, key_words, key_bits, c->pair_alt_keys, nullptr, st));
        launch_pack_pairs(keys, counts, n, key_words, cshift, true, c->num_sms * 8, st);
        CK(cudaGetLastError());
        return HSK_OK;
    }
    return hsk_plain_sort(c, keys, counts, n, key_words, key_bits, c->pair_alt_keys, &c->pair_alt_counts, st);
}

// Stage S6 for kept pairs laid out by their top digit (c->s6_bounds holds
// the 257 digit starts): one segmented LSD pass on the second digit groups
// every top-digit range into 256 sub-ranges, then each of the 65,536
// sub-ranges is sorted on chip (k_range_sort).  *done = false leaves the
// pairs for the general path (keys of fewer than 24 bits, or a sub-range over
// the on-chip capacity; the pairs are then back in place, unsorted).
static int order_pairs_msd(hsk_ctx* c, uint64_t n, int kw, int key_bits, cudaStream_t st, bool* done) {
    *done = false;
    const int shift1 = key_bits - 16, shift2 = key_bits - 24;
    if (shift2 < 0 || n < 2) return HSK_OK;
    const size_t kb = (size_t)kw * 8;
    const uint64_t* d_bounds = (const uint64_t*)c->s6_bounds.p;
    std::vector<uint64_t> hb(257);
    CK(cudaMemcpyAsync(hb.data(), d_bounds, 257 * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hb[256] != n) {
        hsk_set_error(c, "S6: %llu pairs laid out by digit, %llu expected", (unsigned long long)hb[256],
                      (unsigned long long)n);
        return HSK_ECUDA;
    }
    const uint64_t TILE = onesweep_tile_keys(kw);
    std::vector<uint32_t> ts(257);
    uint64_t tiles = 0;
    for (int d = 0; d < 256; ++d) {
        ts[d] = (uint32_t)tiles;
        tiles += (hb[d + 1] - hb[d] + TILE - 1) / TILE;
    }
    ts[256] = (uint32_t)tiles;
    TRY(hsk_ensure(c, c->seg, 257 * 4, false));
    CK(cudaMemcpyAsync(c->seg.p, ts.data(), 257 * 4, cudaMemcpyHostToDevice, st));
    TRY(hsk_ensure(c, c->pass_hist, 256 * 256 * 8, false));
    TRY(hsk_ensure(c, c->digit_off, (256 * 256 + 1) * 8, false));
    TRY(hsk_ensure(c, c->pair_alt_keys, n * kb, false));
    TRY(hsk_ensure(c, c->pair_alt_counts, n * 4, false));
    TRY(hsk_ensure_status(c, tiles * 256 + 1, st));
    uint64_t* doff = (uint64_t*)c->digit_off.p;
    CK(cudaMemsetAsync(c->pass_hist.p, 0, 256 * 256 * 8, st));
    launch_digit_hist_seg(c->out_keys.p, kw, d_bounds, 256, n, (uint64_t*)c->pass_hist.p, 1, st, shift1);
    launch_digit_offsets_seg((const uint64_t*)c->pass_hist.p, d_bounds, doff, 1, 256, st);
    CK(cudaMemcpyAsync(doff + 256 * 256, &hb[256], 8, cudaMemcpyHostToDevice, st));
    uint32_t ep, *ctr;
    TRY(hsk_next_epoch(c, st, &ep));
    TRY(hsk_next_counter(c, st, &ctr));
    launch_onesweep_seg(c->out_keys.p, c->pair_alt_keys.p, (const uint32_t*)c->out_counts.p,
                        (uint32_t*)c->pair_alt_counts.p, d_bounds, 256, (uint32_t)tiles, (const uint32_t*)c->seg.p, kw,
                        shift1, doff, (uint64_t*)c->lb_status.p, ctr, ep, c->d_err, st);
    CK(cudaMemsetAsync(c->d_flag, 0, sizeof(int), st));
    TRY(hsk_next_counter(c, st, &ctr));
    launch_range_sort(c->pair_alt_keys.p, (const uint32_t*)c->pair_alt_counts.p, c->out_keys.p,
                      (uint32_t*)c->out_counts.p, doff, 256 * 256, kw, shift2, c->d_flag, ctr, c->num_sms, st);
    CK(cudaGetLastError());
    int too_big = 0;
    CK(cudaMemcpyAsync(&too_big, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (too_big) {  // a sub-range over the on-chip capacity: the general path sorts all pairs
        CK(cudaMemcpyAsync(c->out_keys.p, c->pair_alt_keys.p, n * kb, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(c->out_counts.p, c->pair_alt_counts.p, n * 4, cudaMemcpyDeviceToDevice, st));
        return HSK_OK;
    }
    *done = true;
    return HSK_OK;
}

// Split buckets [b0, b1) into at most C_want groups of roughly equal k-mer
// counts; returns the first bucket of every group and b1.
std::vector<uint32_t> hsk_group_buckets(const Supermers& S, uint32_t b0, uint32_t b1, uint32_t C_want) {
    uint64_t total = 0;
    for (uint32_t b = b0; b < b1; ++b) total += S.h_bucket_kmers[b];
    std::vector<uint32_t> cut = {b0};
    uint64_t acc = 0;
    uint32_t made = 1;
    for (uint32_t b = b0; b < b1; ++b) {
        acc += S.h_bucket_kmers[b];
        if (b + 1 < b1 && made < C_want && acc * C_want >= total * made) {
            cut.push_back(b + 1);
            ++made;
        }
    }
    cut.push_back(b1);
    return cut;
}

// Plan chunks of consecutive buckets whose keys fit the sort budget.
int hsk_plan_chunks(hsk_ctx* c, const Supermers& S, int key_words,
                    std::vector<std::pair<uint32_t, uint32_t>>& chunks) {
    chunks.clear();
    size_t kb = (size_t)key_words * 8;
    // per key: keys + alt keys + heads + look-back status + worst-case output pair
    double per_key = 2.0 * kb + 4 + (key_words == 1 ? 0.5 : 1.0) + kb + 4;
    size_t held_sort = c->keys.cap + c->alt.cap + c->heads.cap + c->lb_status.cap + c->out_keys.cap +
                       c->out_counts.cap;
    size_t other = c->allocated - held_sort;
    size_t avail = c->budget > other + (64u << 20) ? c->budget - other - (64u << 20) : 0;
    uint64_t cap = (uint64_t)(avail / per_key);
    if (cap > 0xF0000000ull) cap = 0xF0000000ull;  // run heads are 32-bit indices
    if (c->cfg.max_chunk_kmers && cap > c->cfg.max_chunk_kmers) cap = c->cfg.max_chunk_kmers;
    uint32_t b0 = 0;
    uint64_t acc = 0;
    for (uint32_t b = 0; b < S.B; ++b) {
        uint64_t v = S.h_bucket_kmers[b];
        if (v > cap) {
            hsk_set_error(c, "bucket %u holds %llu k-mers, more than a sort chunk can hold (%llu)", b,
                          (unsigned long long)v, (unsigned long long)cap);
            return HSK_ENOMEM;
        }
        if (acc + v > cap && b > b0) {
            chunks.emplace_back(b0, b);
            b0 = b;
            acc = 0;
        }
        acc += v;
    }
    if (S.B > b0) chunks.emplace_back(b0, S.B);
    return HSK_OK;
}

// The first on-chip pass listed n_ov1 sub-segments over its capacity in
// ov_list.  They take a second sort pass with 1.5 times the capacity (tier 1,
// two CTAs per SM), what still does not fit a third with three times it
// (tier 2); what is larger still -- tasks about nine times the mean
// sub-segment or more, made of heavy hitters (Sec. 3.5) -- is folded into
// on-chip k-mer lists (64-bit keys).  *left, *n_left, *left_keys receive the
// sub-segments none of these could take (for the global radix passes) and
// their key count.  The statistics words d_ovstats[0..7] hold {listed, keys}
// of the four steps; ov_list_m receives tier 1's list.
int hsk_local_overflow(hsk_ctx* c, const uint64_t* sub_off, uint32_t n_ov1, uint32_t* ov_list, uint32_t* ov_list_m,
                       uint32_t* ov_list2, uint32_t* ov_list3, int kw, int shift0, void* keys, uint32_t* kcount,
                       uint32_t* kcv, uint32_t lo, uint32_t hi, uint64_t* hist, uint32_t H, uint32_t* d_max,
                       uint64_t* d_distinct, const uint32_t* grp_set, cudaStream_t st, uint32_t** left,
                       uint32_t* n_left, uint64_t* left_keys) {
    uint64_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    *left = ov_list2;
    *n_left = 0;
    *left_keys = 0;
    if (!n_ov1) return HSK_OK;
    uint32_t* ctr;
    TRY(hsk_next_counter(c, st, &ctr));
    launch_local_sort(sub_off, ov_list, n_ov1, 1, shift0, kw, keys, kcount, kcv, ov_list_m, c->d_ovstats + 2, lo,
                      hi, hist, H, d_max, d_distinct, grp_set, ctr, c->d_err, c->num_sms, st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(w, c->d_ovstats, sizeof(w), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const uint32_t n_ovm = (uint32_t)(w[2] & 0xFFFFFFFFull);
    *left = ov_list_m;
    *n_left = n_ovm;
    *left_keys = w[3];
    if (!n_ovm) return HSK_OK;
    TRY(hsk_next_counter(c, st, &ctr));
    launch_local_sort(sub_off, ov_list_m, n_ovm, 2, shift0, kw, keys, kcount, kcv, ov_list2, c->d_ovstats + 4, lo,
                      hi, hist, H, d_max, d_distinct, grp_set, ctr, c->d_err, c->num_sms, st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(w, c->d_ovstats, sizeof(w), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const uint32_t n_ov2 = (uint32_t)(w[4] & 0xFFFFFFFFull);
    *left = ov_list2;
    *n_left = n_ov2;
    *left_keys = w[5];
    if (n_ov2 && kw == 1) {
        TRY(hsk_next_counter(c, st, &ctr));
        launch_heavy_count(sub_off, ov_list2, n_ov2, keys, kcount, kcv, ov_list3, c->d_ovstats + 6, lo, hi, hist, H,
                           d_max, d_distinct, grp_set, ctr, c->d_err, c->num_sms, st);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(w, c->d_ovstats, sizeof(w), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        *left = ov_list3;
        *n_left = (uint32_t)(w[6] & 0xFFFFFFFFull);
        *left_keys = w[7];
    }
    return HSK_OK;
}

// One chunk of buckets through the on-chip path.  The buckets are cut into C
// groups (cut[0..C]); every group's keys are split by their top digit into
// 256 sub-segments, each sorted and counted in shared memory (k_local.cu);
// sub-segments over capacity go through the global radix passes and S5.  The
// kept pairs are appended to the output unordered (stage S6 orders them).
static int local_chunk(hsk_ctx* c, const Supermers& S, const std::vector<uint32_t>& cut, uint64_t nk, int k,
                       uint32_t lo, uint32_t hi, uint32_t H, Output& O, cudaStream_t st) {
    const int kw = k <= 32 ? 1 : 2;
    const size_t kb = (size_t)kw * 8;
    const uint32_t C = (uint32_t)cut.size() - 1;
    const uint64_t NS = (uint64_t)C * 256;
    const int key_bits = 2 * k;
    const int shift0 = key_bits > 8 ? key_bits - 8 : 0;
    // record range and record tiles of each group; the tile -> group map
    std::vector<uint64_t> rbase(C + 1), tbase(C + 1);
    uint64_t nt = 0;
    for (uint32_t i = 0; i <= C; ++i) rbase[i] = S.h_bucket_rec[cut[i]];
    for (uint32_t i = 0; i < C; ++i) {
        tbase[i] = nt;
        nt += expand_tiles(rbase[i + 1] - rbase[i]);
    }
    tbase[C] = nt;
    if (nt >= 0xFFFFFFFFull) {
        hsk_set_error(c, "%llu record tiles in one chunk", (unsigned long long)nt);
        return HSK_EOVERFLOW;
    }
    std::vector<uint32_t> tseg(nt);
    for (uint32_t i = 0; i < C; ++i)
        for (uint64_t t = tbase[i]; t < tbase[i + 1]; ++t) tseg[t] = i;
    TRY(hsk_ensure(c, c->keys, nk * kb, false));
    TRY(hsk_ensure(c, c->alt, nk * 4, false));  // counts of the kept pairs
    // sub-segment tables: sub_cnt | kc | ov_list | ov_list2 | ov_list3 |
    // ov_list_m (u32[NS] each), then sub_off (NS + 1) | cursor (NS) | kc_off
    // (NS + 1) (u64)
    const size_t t32 = (6 * NS * 4 + 7) & ~(size_t)7;
    TRY(hsk_ensure(c, c->loc_tab, t32 + (3 * NS + 2) * 8, false));
    uint32_t* sub_cnt = (uint32_t*)c->loc_tab.p;
    uint32_t* kcv = sub_cnt + NS;
    uint32_t* ov_list = kcv + NS;
    uint32_t* ov_list2 = ov_list + NS;
    uint32_t* ov_list3 = ov_list2 + NS;
    uint32_t* ov_list_m = ov_list3 + NS;
    uint64_t* sub_off = (uint64_t*)((char*)c->loc_tab.p + t32);
    uint64_t* cursor = sub_off + NS + 1;
    uint64_t* kc_off = cursor + NS;
    TRY(hsk_ensure(c, c->batch_d, std::max<uint64_t>(nt, 1) * 4, false));
    TRY(hsk_upload_segments(c, rbase, &tbase, st));
    if (nt) CK(cudaMemcpyAsync(c->batch_d.p, tseg.data(), nt * 4, cudaMemcpyHostToDevice, st));
    const uint64_t* d_rbase = (const uint64_t*)c->seg.p;
    const uint64_t* d_tbase = d_rbase + (C + 1);
    const uint32_t* d_tseg = (const uint32_t*)c->batch_d.p;
    // count keys per (group, top digit), offsets, scatter
    CK(cudaMemsetAsync(sub_cnt, 0, NS * 4, st));
    uint32_t *ctr, ep;
    TRY(hsk_next_counter(c, st, &ctr));
    launch_part(0, S.records, d_rbase, d_tbase, d_tseg, (uint32_t)nt, k, shift0, ctr, sub_cnt, nullptr, nullptr,
                nullptr, c->d_err, expand_grid(c->num_sms), st);
    TRY(hsk_ensure_status(c, scan_status_words(NS), st));
    TRY(hsk_next_epoch(c, st, &ep));
    TRY(hsk_next_counter(c, st, &ctr));
    launch_scan_u32(sub_cnt, NS, sub_off, (uint64_t*)c->lb_status.p, ctr, ep, c->d_err, st);
    CK(cudaMemcpyAsync(cursor, sub_off, NS * 8, cudaMemcpyDeviceToDevice, st));
    TRY(hsk_next_counter(c, st, &ctr));
    launch_part(1, S.records, d_rbase, d_tbase, d_tseg, (uint32_t)nt, k, shift0, ctr, nullptr, cursor,
                sub_off + 1, c->keys.p, c->d_err, expand_grid(c->num_sms), st);
    CK(cudaGetLastError());
    prof_mark(c, st, 3);
    // sort and count on chip; the sub-segments that do not fit go to the
    // larger tiers (1.5 and 3 times the capacity), then to heavy-hitter k-mer
    // lists, and what none of these takes to the global radix passes
    CK(cudaMemsetAsync(c->d_nlocal, 0, 72, st));  // distinct, then {listed, keys} of the four steps
    TRY(hsk_next_counter(c, st, &ctr));
    launch_local_sort(sub_off, nullptr, (uint32_t)NS, 0, shift0, kw, c->keys.p, (uint32_t*)c->alt.p, kcv,
                      ov_list, c->d_ovstats, lo, hi, (uint64_t*)c->hist.p, H, c->d_max, c->d_nlocal, nullptr, ctr, c->d_err,
                      c->num_sms, st);
    CK(cudaGetLastError());
    uint64_t st3[3] = {0, 0, 0};  // distinct, first pass {listed, keys}
    CK(cudaMemcpyAsync(st3, c->d_nlocal, sizeof(st3), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    uint32_t* left = nullptr;
    uint32_t n_ov = 0;
    uint64_t ov_keys = 0;
    TRY(hsk_local_overflow(c, sub_off, (uint32_t)(st3[1] & 0xFFFFFFFFull), ov_list, ov_list_m, ov_list2, ov_list3, kw, shift0,
                           c->keys.p, (uint32_t*)c->alt.p, kcv, lo, hi, (uint64_t*)c->hist.p, H, c->d_max,
                           c->d_nlocal, nullptr, st, &left, &n_ov, &ov_keys));
    // kept pairs in digit-major order (all groups' top digit 0, then 1, ...):
    // the output is then partitioned by the top digit for stage S6
    uint32_t* kc_t = ov_list;  // free again: the later steps list into ov_list_m / ov_list2 / ov_list3
    launch_transpose_kc(kcv, C, kc_t, c->num_sms * 8, st);
    TRY(hsk_next_epoch(c, st, &ep));
    TRY(hsk_next_counter(c, st, &ctr));
    launch_scan_u32(kc_t, NS, kc_off, (uint64_t*)c->lb_status.p, ctr, ep, c->d_err, st);
    CK(cudaGetLastError());
    prof_mark(c, st, 4);
    uint64_t kept = 0;
    CK(cudaMemcpyAsync(st3, c->d_nlocal, sizeof(st3), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&kept, kc_off + NS, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    O.n_distinct += st3[0];
    TRY(hsk_grow_output(c, O, O.n_pairs + kept, kw, st));
    launch_compact(sub_off, kcv, kc_off, (uint32_t)NS, C, kw, c->keys.p, (const uint32_t*)c->alt.p,
                   (char*)c->out_keys.p + O.n_pairs * kb, (uint32_t*)c->out_counts.p + O.n_pairs, kept, c->d_err,
                   c->num_sms * 8, st);
    CK(cudaGetLastError());
    // where each top digit's pairs start (S6), valid while they are the only pairs
    {
        std::vector<uint64_t> at(257);
        for (uint32_t d = 0; d <= 256; ++d) at[d] = (uint64_t)d * C;
        TRY(hsk_ensure(c, c->s6_bounds, 2 * 257 * 8, false));
        uint64_t* d_at = (uint64_t*)c->s6_bounds.p + 257;
        CK(cudaMemcpyAsync(d_at, at.data(), 257 * 8, cudaMemcpyHostToDevice, st));
        launch_gather_u64(kc_off, d_at, 257, (uint64_t*)c->s6_bounds.p, st);
        CK(cudaGetLastError());
        c->s6_digit_major = O.n_pairs == 0;
    }
    O.n_pairs += kept;
    if (n_ov) {  // the sub-segments that did not fit: global radix passes, then S5
        TRY(hsk_ensure(c, c->batch_a, ov_keys * kb, false));
        TRY(hsk_ensure(c, c->batch_c, ((uint64_t)n_ov + 1) * 8, false));
        launch_ov_gather(sub_off, left, n_ov, (uint64_t*)c->batch_c.p, kw, c->keys.p, c->batch_a.p, ov_keys,
                         c->d_err, c->num_sms * 4, st);
        CK(cudaGetLastError());
        TRY(hsk_plain_sort(c, c->batch_a.p, nullptr, ov_keys, kw, key_bits, c->batch_b, nullptr, st));
        TRY(hsk_rle_chunk(c, c->batch_a.p, ov_keys, kw, lo, hi, H, (uint64_t*)c->hist.p, O, st));
        c->s6_digit_major = false;  // pairs appended after the digit-major ones
    }
    c->last_ov_keys += ov_keys;
    prof_mark(c, st, 5);
    return HSK_OK;
}

int hsk_run_count(hsk_ctx* c, const char* d_reads, const uint64_t* d_offsets, uint64_t n_reads,
                  uint64_t n_bases, int k, int m, uint32_t lo, uint32_t hi, cudaStream_t st,
                  DevResult& R, InputPipe* pipe) {
    memset(&R, 0, sizeof(R));
    c->zst = st;
    if (n_bases >= (1ull << 40)) {
        hsk_set_error(c, "n_bases %llu exceeds 2^40", (unsigned long long)n_bases);
        return HSK_EOVERFLOW;
    }
    const int kw = k <= 32 ? 1 : 2;
    const size_t kb = (size_t)kw * 8;
    const uint32_t H = c->cfg.hist_len;
    TRY(hsk_ensure(c, c->hist, (size_t)H * 8, false));
    CK(cudaEventRecord(c->ev0, st));
    CK(cudaMemsetAsync(c->hist.p, 0, (size_t)H * 8, st));
    CK(cudaMemsetAsync(c->small, 0, 64, st));  // err, max, n_heads, n_out
    CK(cudaMemsetAsync(c->counters, 0, HSK_N_COUNTERS * sizeof(uint32_t), st));
    c->ctr_used = 0;
    c->marks.clear();
    prof_mark(c, st, -1);
    Output O;
    Encoded E;
    {
        NvtxRange r("S1 encode");
        TRY(hsk_encode_into(c, d_reads, n_bases, d_offsets, n_reads, c->pk, c->iv, c->rs, E, st, pipe != nullptr));
    }
    prof_mark(c, st, 0);
    Supermers S;
    uint32_t B = hsk_pick_buckets(c, n_bases, k);
    {
        NvtxRange r("S2-S3 supermers");
        TRY(hsk_supermers(c, E, k, m, B, S, st, pipe));
    }
    prof_mark(c, st, 2);
    R.n_windows = S.n_kmers;
    R.n_supermers = S.n_records;
    std::vector<std::pair<uint32_t, uint32_t>> chunks;
    if (S.n_kmers > 0) TRY(hsk_plan_chunks(c, S, kw, chunks));
    c->s6_digit_major = false;
    const int P = n_passes_for(2 * k);
    uint32_t total_segments = 0;
    bool unordered = false;
    c->last_ov_keys = 0;
    for (auto& ch : chunks) {
        uint64_t nk = 0;
        for (uint32_t b = ch.first; b < ch.second; ++b) nk += S.h_bucket_kmers[b];
        if (nk == 0) continue;
        if (c->cfg.local_sort) {
            // groups of about a third of the on-chip capacity per top digit
            const uint64_t per_group = 256ull * local_cap(kw) / (c->tune.group_div ? c->tune.group_div : 3);
            const uint32_t C_want = (uint32_t)std::min<uint64_t>(ch.second - ch.first,
                                                                 std::max<uint64_t>(1, nk / per_group));
            NvtxRange r("S4-S5 on-chip sort and count");
            TRY(local_chunk(c, S, hsk_group_buckets(S, ch.first, ch.second, C_want), nk, k, lo, hi, H, O, st));
            unordered = true;
            continue;
        }
        // segments: groups of buckets sorted independently, tiles interleaved
        NvtxRange r("S4-S5 global radix sort and count");
        uint32_t C_want = (uint32_t)std::min<uint64_t>({(uint64_t)HSK_SEGMENTS, ch.second - ch.first,
                                                        std::max<uint64_t>(1, nk / HSK_MIN_SEGMENT_KMERS)});
        std::vector<uint32_t> cut = hsk_group_buckets(S, ch.first, ch.second, C_want);
        const uint32_t C = (uint32_t)cut.size() - 1;
        total_segments += C;
        std::vector<uint64_t> kbase(C + 1), rbase(C + 1);
        uint64_t acc = 0, max_rt = 0, max_kt = 0;
        const uint64_t tk = onesweep_tile_keys(kw);
        for (uint32_t sgi = 0; sgi < C; ++sgi) {
            kbase[sgi] = acc;
            rbase[sgi] = S.h_bucket_rec[cut[sgi]];
            uint64_t sk = 0;
            for (uint32_t b = cut[sgi]; b < cut[sgi + 1]; ++b) sk += S.h_bucket_kmers[b];
            acc += sk;
            max_rt = std::max<uint64_t>(max_rt, expand_tiles(S.h_bucket_rec[cut[sgi + 1]] - rbase[sgi]));
            max_kt = std::max<uint64_t>(max_kt, (sk + tk - 1) / tk);
        }
        kbase[C] = acc;
        rbase[C] = S.h_bucket_rec[cut[C]];
        TRY(hsk_ensure(c, c->keys, nk * kb, false));
        TRY(hsk_ensure(c, c->alt, nk * kb, false));
        TRY(hsk_ensure(c, c->pass_hist, (size_t)C * P * 256 * 8, false));
        TRY(hsk_ensure(c, c->digit_off, (size_t)C * P * 256 * 8, false));
        TRY(hsk_ensure_status(c, (uint64_t)C * (max_rt + 1) * 4 + 4, st));
        TRY(hsk_upload_segments(c, kbase, &rbase, st));
        const uint64_t* d_kbase = (const uint64_t*)c->seg.p;
        const uint64_t* d_rbase = d_kbase + (C + 1);
        CK(cudaMemsetAsync(c->pass_hist.p, 0, (size_t)C * P * 256 * 8, st));
        uint32_t ep, *ctrs;
        TRY(hsk_next_epoch(c, st, &ep));
        TRY(hsk_next_counters(c, st, C, &ctrs));
        launch_expand_seg(S.records, d_rbase, d_kbase, C, max_rt, k, c->keys.p, (uint64_t*)c->lb_status.p, ctrs,
                          ep, (uint64_t*)c->pass_hist.p, P, c->d_err, expand_grid(c->num_sms), st);
        launch_digit_offsets_seg((uint64_t*)c->pass_hist.p, d_kbase, (uint64_t*)c->digit_off.p, P, C, st);
        CK(cudaGetLastError());
        prof_mark(c, st, 3);
        bool in_b = false;
        TRY(sort_segments(c, c->keys.p, c->alt.p, nullptr, nullptr, d_kbase, C, (uint32_t)max_kt, kw, P,
                          (const uint64_t*)c->digit_off.p, &in_b, st));
        if (c->prof) c->prof_passes += P;
        prof_mark(c, st, 4);
        const void* sorted = in_b ? c->alt.p : c->keys.p;
        TRY(hsk_rle_chunk(c, sorted, nk, kw, lo, hi, H, (uint64_t*)c->hist.p, O, st));
        prof_mark(c, st, 5);
    }
    if (total_segments > 1 || unordered) {
        NvtxRange r("S6 order");
        bool done = false;
        if (chunks.size() == 1 && c->cfg.local_sort && c->s6_digit_major)
            TRY(order_pairs_msd(c, O.n_pairs, kw, 2 * k, st, &done));
        if (!done) TRY(hsk_order_pairs(c, c->out_keys.p, (uint32_t*)c->out_counts.p, O.n_pairs, kw, 2 * k, st, hi));
    }
    prof_mark(c, st, 6);
    CK(cudaEventRecord(c->ev1, st));
    uint32_t mx = 0;
    TRY(hsk_read_device_error(c, st, &mx));
    prof_collect(c);
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    R.n_pairs = O.n_pairs;
    R.n_distinct = O.n_distinct;
    R.max_count = mx;
    R.n_chunks = (uint32_t)chunks.size();
    R.key_words = kw;
    R.kmers = (const uint64_t*)c->out_keys.p;
    R.counts = (const uint32_t*)c->out_counts.p;
    R.hist = (const uint64_t*)c->hist.p;
    R.hist_len = H;
    R.device_ms = ms;
    return HSK_OK;
}

static void to_public(const DevResult& R, hsk_result* out) {
    memset(out, 0, sizeof(*out));
    out->n_pairs = R.n_pairs;
    out->kmers = R.kmers;
    out->counts = R.counts;
    out->hist = R.hist;
    out->hist_len = R.hist_len;
    out->key_words = R.key_words;
    out->n_windows = R.n_windows;
    out->n_distinct = R.n_distinct;
    out->max_count = R.max_count;
    out->n_chunks = R.n_chunks;
    out->n_supermers = R.n_supermers;
    out->device_ms = R.device_ms;
}

// ---------------------------------------------------------------------------
// C ABI: plain counting
// ---------------------------------------------------------------------------
extern "C" int hsk_count_device(hsk_ctx* c, const char* d_reads, const uint64_t* d_offsets,
                                uint64_t n_reads, uint64_t n_bases, int k, int m, uint32_t lo,
                                uint32_t hi, void* stream, hsk_result* out) {
    return hsk_guarded(c, [&]() -> int {
        TRY(check_args(c, d_reads, d_offsets, n_reads, k, m, lo, hi));
        if (!out) return HSK_EINVAL;
        if (n_bases > 0 && !d_reads) {
            hsk_set_error(c, "NULL reads with n_bases > 0");
            return HSK_EINVAL;
        }
        CK(cudaSetDevice(c->cfg.device));
        cudaStream_t st = (cudaStream_t)stream;
        DevResult R;
        int rc = hsk_run_count(c, d_reads, d_offsets, n_reads, n_bases, k, m, lo, hi, st, R);
        if (rc != HSK_OK) return rc;
        to_public(R, out);
        return HSK_OK;
    });
}

// Stage host buffers into context device memory, count, copy results back.
int hsk_count_host_on(hsk_ctx* c, const char* reads, const uint64_t* offsets, uint64_t n_reads,
                      int k, int m, uint32_t lo, uint32_t hi, cudaStream_t st, DevBuf& d_reads,
                      DevBuf& d_offsets, HostResult& HR) {
    uint64_t n_bases = 0;
    if (n_reads > 0) {
        if (offsets[0] != 0) {
            hsk_set_error(c, "offsets[0] must be 0");
            return HSK_EINVAL;
        }
        for (uint64_t i = 0; i < n_reads; ++i)
            if (offsets[i + 1] < offsets[i]) {
                hsk_set_error(c, "offsets not monotone at read %llu", (unsigned long long)i);
                return HSK_EINVAL;
            }
        n_bases = offsets[n_reads];
        if (n_bases > 0 && !reads) {
            hsk_set_error(c, "NULL reads with bases present");
            return HSK_EINVAL;
        }
    }
    TRY(hsk_ensure(c, d_reads, n_bases + 16, false));
    TRY(hsk_ensure(c, d_offsets, (n_reads + 1) * 8, false));
    if (n_reads) CK(cudaMemcpyAsync(d_offsets.p, offsets, (n_reads + 1) * 8, cudaMemcpyHostToDevice, st));
    else CK(cudaMemsetAsync(d_offsets.p, 0, 8, st));
    // large inputs: the read bytes arrive in chunks on the copy stream while
    // S1/S2 work on the chunks already there
    InputPipe pipe;
    InputPipe* pp = nullptr;
    if (n_bases >= (64ull << 20) && c->cstream) {
        const int n = (int)std::min<uint64_t>(HSK_MAX_PIPE, std::max<uint64_t>(2, n_bases >> 27));
        pipe.n = n;
        // a short first chunk, so that S1/S2 start soon after the call, then
        // equal chunks (bounds on 64 K-base multiples)
        const uint64_t first = std::max<uint64_t>(1ull << 20, n_bases / (4 * (uint64_t)n));
        pipe.bound[0] = 0;
        for (int i = 1; i < n; ++i)
            pipe.bound[i] = (first + (uint64_t)(i - 1) * (n_bases - first) / (uint64_t)(n - 1)) & ~0xFFFFull;
        pipe.bound[n] = n_bases;
        for (int i = 0; i < n; ++i) pipe.ev[i] = c->pipe_ev[i];
        pipe.h_reads = reads;
        pipe.d_reads = (char*)d_reads.p;
        pipe.cs = c->cstream;
        pp = &pipe;
    } else if (n_bases) {
        CK(cudaMemcpyAsync(d_reads.p, reads, n_bases, cudaMemcpyHostToDevice, st));
    }
    DevResult R;
    int rc_run = hsk_run_count(c, (const char*)d_reads.p, (const uint64_t*)d_offsets.p, n_reads, n_bases, k, m,
                               lo, hi, st, R, pp);
    if (pp) {
        // every chunk copy is issued (an early error return may have left some)
        // and finished before the buffers can be reused
        for (; pipe.issued < pipe.n; ++pipe.issued) CK(pipe.issue(pipe.issued));
        CK(cudaStreamSynchronize(c->cstream));
    }
    TRY(rc_run);
    size_t kb = (size_t)R.key_words * 8;
    HR.kmers.resize(R.n_pairs * R.key_words);
    HR.counts.resize(R.n_pairs);
    HR.hist.resize(R.hist_len);
    if (R.n_pairs) {
        CK(cudaMemcpyAsync(HR.kmers.data(), R.kmers, R.n_pairs * kb, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(HR.counts.data(), R.counts, R.n_pairs * 4, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaMemcpyAsync(HR.hist.data(), R.hist, (size_t)R.hist_len * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    HR.R = R;
    HR.R.kmers = HR.kmers.data();
    HR.R.counts = HR.counts.data();
    HR.R.hist = HR.hist.data();
    return HSK_OK;
}

extern "C" int hsk_count(hsk_ctx* c, const char* reads, const uint64_t* offsets, uint64_t n_reads,
                         int k, int m, uint32_t lo, uint32_t hi, hsk_result* out) {
    return hsk_guarded(c, [&]() -> int {
        TRY(check_args(c, reads, offsets, n_reads, k, m, lo, hi));
        if (!out) return HSK_EINVAL;
        CK(cudaSetDevice(c->cfg.device));
        TRY(hsk_count_host_on(c, reads, offsets, n_reads, k, m, lo, hi, c->stream, c->in_reads,
                              c->in_offsets, c->host_res));
        to_public(c->host_res.R, out);
        return HSK_OK;
    });
}

extern "C" int hsk_result_copy(hsk_ctx* c, const hsk_result* r, uint64_t* kmers_dst,
                               uint32_t* counts_dst, uint64_t* hist_dst, int dst_on_device,
                               void* stream) {
    if (!c || !r) return HSK_EINVAL;
    CK(cudaSetDevice(c->cfg.device));
    cudaStream_t st = (cudaStream_t)stream;
    size_t kb = (size_t)r->key_words * 8;
    if (kmers_dst && r->n_pairs)
        CK(cudaMemcpyAsync(kmers_dst, r->kmers, r->n_pairs * kb, cudaMemcpyDefault, st));
    if (counts_dst && r->n_pairs)
        CK(cudaMemcpyAsync(counts_dst, r->counts, r->n_pairs * 4, cudaMemcpyDefault, st));
    if (hist_dst && r->hist_len)
        CK(cudaMemcpyAsync(hist_dst, r->hist, (size_t)r->hist_len * 8, cudaMemcpyDefault, st));
    (void)dst_on_device;  // unified addressing: the runtime infers the direction
    CK(cudaStreamSynchronize(st));
    return HSK_OK;
}

// ---------------------------------------------------------------------------
// C ABI: stages
// ---------------------------------------------------------------------------
extern "C" int hsk_stage_encode(hsk_ctx* c, const char* d_reads, uint64_t n_bases,
                                const uint64_t* d_offsets, uint64_t n_reads, uint64_t* d_packed,
                                uint64_t* d_invalid, uint64_t* d_start, void* stream) {
    return hsk_guarded(c, [&]() -> int {
        if (!c || !d_packed || !d_invalid || !d_start) return HSK_EINVAL;
        CK(cudaSetDevice(c->cfg.device));
        cudaStream_t st = (cudaStream_t)stream;
        c->zst = st;
        uint64_t n_pw = (n_bases + 31) / 32, n_mw = (n_bases + 63) / 64;
        CK(cudaMemsetAsync(c->small, 0, 64, st));
        CK(cudaMemsetAsync(d_packed, 0, (n_pw + 4) * 8, st));
        CK(cudaMemsetAsync(d_invalid, 0, (n_mw + 4) * 8, st));
        CK(cudaMemsetAsync(d_start, 0, (n_mw + 4) * 8, st));
        launch_mark_starts(d_offsets, n_reads, n_bases, d_start, c->d_err, st);
        launch_encode(d_reads, n_bases, d_packed, d_invalid, n_pw, n_mw, st);
        CK(cudaGetLastError());
        return hsk_read_device_error(c, st);
    });
}

extern "C" int hsk_stage_windows(hsk_ctx* c, const char* d_reads, const uint64_t* d_offsets,
                                 uint64_t n_reads, uint64_t n_bases, int k, int m, uint8_t* d_valid,
                                 uint64_t* d_key, uint64_t* d_minhash, void* stream) {
    return hsk_guarded(c, [&]() -> int {
        TRY(check_args(c, d_reads, d_offsets, n_reads, k, m, 0, 0));
        CK(cudaSetDevice(c->cfg.device));
        cudaStream_t st = (cudaStream_t)stream;
        c->zst = st;
        CK(cudaMemsetAsync(c->small, 0, 64, st));
        Encoded E;
        TRY(hsk_encode_into(c, d_reads, n_bases, d_offsets, n_reads, c->pk, c->iv, c->rs, E, st, false));
        SmParams P;
        fill_sm_params(c, E, k, m, 1, P);
        uint64_t warp_tiles = (n_bases + 1023) / 1024;
        P.grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)c->num_sms * 4, (warp_tiles + SM_CTA_WARPS - 1) / SM_CTA_WARPS));
        P.dump_valid = d_valid;
        P.dump_key = d_key;
        P.dump_minhash = d_minhash;
        launch_supermer(SM_DUMP, P, st);
        CK(cudaGetLastError());
        return hsk_read_device_error(c, st);
    });
}

extern "C" int hsk_stage_supermers(hsk_ctx* c, const char* d_reads, const uint64_t* d_offsets,
                                   uint64_t n_reads, uint64_t n_bases, int k, int m,
                                   uint32_t n_buckets, uint64_t* d_bucket_kmers,
                                   uint64_t* d_bucket_rec, const uint64_t** d_records,
                                   uint64_t* n_records, int* record_words, int* max_kmers,
                                   void* stream) {
    return hsk_guarded(c, [&]() -> int {
        TRY(check_args(c, d_reads, d_offsets, n_reads, k, m, 0, 0));
        if (n_buckets < 1 || n_buckets > HSK_MAX_BUCKETS || (n_buckets & (n_buckets - 1)) || !d_bucket_kmers || !d_bucket_rec || !d_records ||
            !n_records || !record_words)
            return HSK_EINVAL;
        CK(cudaSetDevice(c->cfg.device));
        cudaStream_t st = (cudaStream_t)stream;
        c->zst = st;
        CK(cudaMemsetAsync(c->small, 0, 64, st));
        CK(cudaMemsetAsync(c->counters, 0, HSK_N_COUNTERS * sizeof(uint32_t), st));
        c->ctr_used = 0;
        Encoded E;
        TRY(hsk_encode_into(c, d_reads, n_bases, d_offsets, n_reads, c->pk, c->iv, c->rs, E, st, false));
        Supermers S;
        TRY(hsk_supermers(c, E, k, m, n_buckets, S, st, nullptr));
        CK(cudaMemcpyAsync(d_bucket_kmers, c->bucket_kmers.p, (size_t)n_buckets * 8, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(d_bucket_rec, c->bucket_rec.p, ((size_t)n_buckets + 1) * 8, cudaMemcpyDeviceToDevice, st));
        *d_records = S.records;
        *n_records = S.n_records;
        *record_words = S.rec_words;
        if (max_kmers) *max_kmers = S.nmax;
        return hsk_read_device_error(c, st);
    });
}

extern "C" int hsk_stage_sort(hsk_ctx* c, uint64_t* d_keys, uint64_t n, int key_words, int key_bits,
                              void* stream) {
    return hsk_guarded(c, [&]() -> int {
        if (!c || (n && !d_keys) || (key_words != 1 && key_words != 2) || key_bits < 1 ||
            key_bits > 64 * key_words || reinterpret_cast<uintptr_t>(d_keys) % (8u * (unsigned)key_words))
            return HSK_EINVAL;
        CK(cudaSetDevice(c->cfg.device));
        cudaStream_t st = (cudaStream_t)stream;
        c->zst = st;
        CK(cudaMemsetAsync(c->small, 0, 64, st));
        CK(cudaMemsetAsync(c->counters, 0, HSK_N_COUNTERS * sizeof(uint32_t), st));
        c->ctr_used = 0;
        if (n <= 1) return HSK_OK;
        TRY(hsk_plain_sort(c, d_keys, nullptr, n, key_words, key_bits, c->alt, nullptr, st));
        return hsk_read_device_error(c, st);
    });
}

extern "C" int hsk_stage_rle(hsk_ctx* c, const uint64_t* d_sorted, uint64_t n, int key_words,
                             uint32_t lo, uint32_t hi, void* stream, hsk_result* out) {
    return hsk_guarded(c, [&]() -> int {
        if (!c || !out || (n && !d_sorted) || (key_words != 1 && key_words != 2) || lo > hi) return HSK_EINVAL;
        CK(cudaSetDevice(c->cfg.device));
        cudaStream_t st = (cudaStream_t)stream;
        c->zst = st;
        const uint32_t H = c->cfg.hist_len;
        TRY(hsk_ensure(c, c->hist, (size_t)H * 8, false));
        CK(cudaMemsetAsync(c->hist.p, 0, (size_t)H * 8, st));
        CK(cudaMemsetAsync(c->small, 0, 64, st));
        CK(cudaMemsetAsync(c->counters, 0, HSK_N_COUNTERS * sizeof(uint32_t), st));
        c->ctr_used = 0;
        Output O;
        TRY(hsk_rle_chunk(c, d_sorted, n, key_words, lo, hi, H, (uint64_t*)c->hist.p, O, st));
        uint32_t mx = 0;
        TRY(hsk_read_device_error(c, st, &mx));
        DevResult R;
        memset(&R, 0, sizeof R);
        R.n_pairs = O.n_pairs;
        R.n_distinct = O.n_distinct;
        R.n_windows = n;
        R.max_count = mx;
        R.key_words = key_words;
        R.kmers = (const uint64_t*)c->out_keys.p;
        R.counts = (const uint32_t*)c->out_counts.p;
        R.hist = (const uint64_t*)c->hist.p;
        R.hist_len = H;
        R.n_chunks = 1;
        to_public(R, out);
        return HSK_OK;
    });
}

extern "C" int hsk_stage_order(hsk_ctx* c, uint64_t* d_keys, uint32_t* d_counts, uint64_t n,
                               int key_words, int key_bits, void* stream) {
    return hsk_guarded(c, [&]() -> int {
        if (!c || (n && (!d_keys || !d_counts)) || (key_words != 1 && key_words != 2) || key_bits < 1 ||
            key_bits > 64 * key_words || reinterpret_cast<uintptr_t>(d_keys) % (8u * (unsigned)key_words) ||
            reinterpret_cast<uintptr_t>(d_counts) % 4u)
            return HSK_EINVAL;
        CK(cudaSetDevice(c->cfg.device));
        cudaStream_t st = (cudaStream_t)stream;
        c->zst = st;
        CK(cudaMemsetAsync(c->small, 0, 64, st));
        CK(cudaMemsetAsync(c->counters, 0, HSK_N_COUNTERS * sizeof(uint32_t), st));
        c->ctr_used = 0;
        TRY(hsk_order_pairs(c, d_keys, d_counts, n, key_words, key_bits, st, 0));
        return hsk_read_device_error(c, st);
    });
}

extern "C" int hsk_debug_wait_timeout(hsk_ctx* c, uint32_t spin_limit) {
    if (!c || spin_limit < 1 || spin_limit > HSK_SPIN_LIMIT) return HSK_EINVAL;
    CK(cudaSetDevice(c->cfg.device));
    cudaStream_t st = c->stream;
    c->zst = st;
    TRY(hsk_ensure(c, c->batch_c, 256, false));  // two padded status words
    CK(cudaMemsetAsync(c->batch_c.p, 0, 256, st));
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
    launch_debug_wait((uint64_t*)c->batch_c.p, spin_limit, c->d_err, st);
    CK(cudaGetLastError());
    const int rc = hsk_read_device_error(c, st);
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
    CK(cudaStreamSynchronize(st));
    return rc;
}

// host block pool self-check (see hsk_stages.h); pinning is off (pin_cap = 0)
// so that no device call is made
extern "C" int hsk_debug_host_pool_check(void) {
    HostPool pool;
    pool.pin_cap = 0;
    pool.keep_cap = (size_t)8 << 20;
    // 1-3: size classes
    if (HostPool::round_up(1) != ((size_t)64 << 10)) return 1;
    if (HostPool::round_up((size_t)1 << 20) != ((size_t)1 << 20)) return 2;
    const size_t b = ((size_t)3 << 20) + 1, r = HostPool::round_up(b);
    if (r < b || (r - b) * 8 >= b) return 3;
    // 4-6: a released block is reused by a request it fits, the smallest first
    size_t c1 = 0, c4 = 0, c = 0;
    bool pin = true;
    void* p1 = pool.get((size_t)1 << 20, &c1, &pin);
    if (!p1 || pin || c1 != ((size_t)1 << 20)) return 4;
    void* p4 = pool.get((size_t)4 << 20, &c4, &pin);
    pool.put(p1, c1, false);
    pool.put(p4, c4, false);
    void* q = pool.get((size_t)600 << 10, &c, &pin);
    if (q != p1 || c != c1) return 5;
    void* q2 = pool.get((size_t)2 << 20, &c, &pin);
    if (q2 != p4 || c != c4) return 6;
    // 7: past keep_cap a released block is freed, not kept
    pool.put(q, c1, false);
    pool.put(q2, c4, false);
    size_t c16 = 0;
    void* p16 = pool.get((size_t)16 << 20, &c16, &pin);
    pool.put(p16, c16, false);
    if (pool.free_total > pool.keep_cap || pool.free_total != c1 + c4) return 7;
    // 8-10: arrays take blocks from the pool and give them back (moves included)
    {
        HostArr<uint64_t> a;
        a.pool = &pool;
        a.resize(100000);
        if (!a.data() || a.size() != 100000 || a.cap < 100000) return 8;
        uint64_t* d = a.data();
        a.resize(50000);
        if (a.data() != d) return 9;
        HostArr<uint64_t> m(std::move(a));
        if (m.data() != d || a.data() != nullptr || m.pool != &pool) return 10;
    }
    if (pool.free_total != c1 + c4) return 11;  // the array's block went back (it was one of the two)
    return 0;
}
