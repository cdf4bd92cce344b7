/* hsk.h -- C ABI of a single-GPU sorting-based k-mer counter (HySortK,
 * arXiv 2407.07718), written for NVIDIA GB300 (sm_103a).
 *
 * What is computed (Sec. 2.1 k-mer counting; Sec. 3.1 sorting-based counting):
 * for every read and every window of k consecutive bases that are all
 * upper-case A, C, G or T, the canonical k-mer -- the numeric minimum of the
 * window's 2-bit code (A=0 C=1 G=2 T=3, first base most significant) and the
 * code of its reverse complement -- is counted.  The result is
 *   - every distinct canonical k-mer whose count c satisfies lo <= c <= hi,
 *     with c, in ascending key order (the frequency filter of Sec. 3.1 and
 *     Sec. 4; the paper uses lo=2, hi=50);
 *   - the histogram over ALL distinct k-mers before the filter: hist[c] is the
 *     number of distinct k-mers seen exactly c times, for 1 <= c < hist_len-1;
 *     hist[hist_len-1] collects every count >= hist_len-1; hist[0] = 0.
 * Any other byte (N, lower case, IUPAC codes) breaks every window containing
 * it.  Windows never cross a read boundary.  Counts are exact (Sec. 3.3).
 *
 * How (all on the GPU, no CPU fallback): 2-bit encoding (Sec. 2.2); canonical
 * k-mers with hash-scored minimizers and supermers (Sec. 3.2); supermers
 * scattered into minimizer-hashed buckets, the paper's tasks (Sec. 3.4);
 * an LSD radix sort of packed keys (Sec. 3.1); a run-length scan with the
 * filter and histogram (Sec. 3.1).
 *
 * Keys: k <= 32 -> one uint64 word per k-mer (the 2k-bit code, right
 * aligned); 33 <= k <= 64 -> two uint64 words per k-mer, little-endian
 * {lo, hi} of the 2k-bit code.
 *
 * Errors: every function returns HSK_OK (0) or a negative HSK_E* code;
 * hsk_last_error() then holds a one-line description.  A context is not
 * thread-safe: use one context per host thread.
 */
#ifndef HSK_H
#define HSK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HSK_OK 0
#define HSK_EINVAL (-1)     /* bad argument: k, m, lo/hi, pointers, offsets */
#define HSK_ENOMEM (-2)     /* the job does not fit the context's HBM budget, or host memory ran out */
#define HSK_ECUDA (-3)      /* a CUDA runtime call failed; see hsk_last_error */
#define HSK_ETIMEOUT (-4)   /* a bounded device-side wait gave up */
#define HSK_ECANCELED (-5)  /* the job was cancelled before it ran */
#define HSK_EOVERFLOW (-6)  /* a count or size exceeds the representable range */
#define HSK_ENOTFOUND (-7)  /* unknown ticket */

typedef struct hsk_ctx hsk_ctx;

/* Context configuration.  Fill with hsk_config_default() and override. */
typedef struct {
    int device;            /* CUDA device ordinal */
    uint64_t hbm_budget;   /* bytes of device memory the context may hold; 0 = 90 % of free */
    uint32_t hist_len;     /* histogram bins, >= 2 (default 65536) */
    uint32_t n_buckets;    /* minimizer buckets (tasks), a power of two <= 8192; 0 = per job */
    uint32_t radix_bits;   /* LSD digit width, 8 (default) */
    uint32_t max_chunk_kmers; /* 0 = as many as the budget allows; else cap per sort chunk */
    uint64_t seed;         /* XOR-ed into each canonical m-mer before hashing */
    int autotune;          /* 1 = hsk_count_batch applies the parameters that
                              hsk_autotune recorded for its class of job mix (if
                              any); 0 = built-in or last applied parameters */
    int local_sort;        /* 1 (default) = sort and count sub-segments that fit in
                              shared memory on chip, the rest with global radix
                              passes; 0 = global radix passes only.  The result is
                              the same either way. */
    const char* tune_cache; /* file of tuned parameters: read at hsk_create,
                               appended to by hsk_autotune; NULL = none */
    int minimizer_order;    /* 0 (default) = m-mers ordered by a hash of the
                               canonical m-mer (Sec. 3.2); 1 = lexically, by the
                               canonical m-mer's code (its top 32 bits for
                               m > 16).  Counts are the same either way; only
                               supermers, buckets and speed change. */
} hsk_config;

/* A counting result.  All arrays are owned by the context and stay valid until
 * the next counting call on the same context, hsk_release() of its ticket, or
 * hsk_destroy().  For hsk_count() they are host pointers; for
 * hsk_count_device() they are device pointers (kmers, counts, hist). */
typedef struct {
    uint64_t n_pairs;        /* entries in kmers/counts */
    const uint64_t* kmers;   /* n_pairs * key_words words, ascending */
    const uint32_t* counts;  /* n_pairs counts, each in [lo, hi] */
    const uint64_t* hist;    /* hist_len bins (see above) */
    uint32_t hist_len;
    int key_words;           /* 1 for k <= 32, 2 for 33 <= k <= 64 */
    uint64_t n_windows;      /* valid k-mer windows counted (sum of all counts) */
    uint64_t n_distinct;     /* distinct canonical k-mers */
    uint32_t max_count;      /* largest count of any k-mer */
    uint32_t n_chunks;       /* sort chunks the job was split into */
    uint64_t n_supermers;    /* supermer records formed */
    double device_ms;        /* device time of the job (CUDA events), ms */
} hsk_result;

/* One job for the batched and served forms: host pointers, borrowed until the
 * call returns (hsk_count_batch) or the job completes (hsk_submit). */
typedef struct {
    const char* reads;        /* ASCII bases of all reads, concatenated */
    const uint64_t* offsets;  /* n_reads + 1 entries, offsets[0] = 0, non-decreasing */
    uint64_t n_reads;
    int k;                    /* 1 <= k <= 64 */
    int m;                    /* 1 <= m <= min(k, 32) */
    uint32_t lo, hi;          /* inclusive count filter, lo <= hi */
} hsk_job;

/* Defaults: device 0, budget 0 (90 % of free), hist_len 65536, buckets auto,
 * 8-bit digits, seed 0x9E3779B97F4A7C15, autotune on, no tuning cache. */
int hsk_config_default(hsk_config* cfg);

/* Create a context on cfg->device (cfg = NULL: defaults).  *out receives the
 * context; on failure *out is NULL and the code says why. */
int hsk_create(hsk_ctx** out, const hsk_config* cfg);

/* Release every device and host buffer of the context.  NULL-safe. */
void hsk_destroy(hsk_ctx* ctx);

/* One-line description of the last error on this context ("" if none).  The
 * string belongs to the context. */
const char* hsk_last_error(hsk_ctx* ctx);

/* Count canonical k-mers of host-resident reads.  reads[offsets[i] ..
 * offsets[i+1]) is read i; offsets has n_reads + 1 non-decreasing entries
 * starting at 0.  Host-to-device copies, the GPU pipeline and the
 * device-to-host copies of the result all happen inside the call; the result
 * arrays are host memory owned by the context.
 * Errors: HSK_EINVAL (k outside [1,64], m outside [1, min(k,32)], lo > hi,
 * NULL pointer with n_reads > 0, offsets not monotone or not starting at 0),
 * HSK_ENOMEM, HSK_ECUDA, HSK_ETIMEOUT. */
int hsk_count(hsk_ctx* ctx, const char* reads, const uint64_t* offsets, uint64_t n_reads, int k,
              int m, uint32_t lo, uint32_t hi, hsk_result* out);

/* As hsk_count, but reads (n_bases bytes) and offsets (n_reads + 1 entries)
 * are device pointers, the work is ordered on `stream` (a cudaStream_t; NULL
 * = legacy default stream), and the result arrays are device memory owned by
 * the context.  Returns after the result is complete.  Offsets are checked on
 * the device; a violation returns HSK_EINVAL. */
int hsk_count_device(hsk_ctx* ctx, const char* d_reads, const uint64_t* d_offsets,
                     uint64_t n_reads, uint64_t n_bases, int k, int m, uint32_t lo, uint32_t hi,
                     void* stream, hsk_result* out);

/* Counting with extension information (Sec. 3.3.2: the ID of the read a
 * k-mer was extracted from and its position in that read, which seed-and-
 * extend pipelines such as long-read overlap detection need).  counts is
 * exactly what hsk_count returns.  Each kept k-mer i (in the ascending order
 * of counts.kmers) has counts.counts[i] occurrences, listed at
 * [occ_offsets[i], occ_offsets[i+1]) of occ_read (0-based read index) and
 * occ_pos (0-based start of the window in that read), in ascending (read,
 * position) order.  All arrays are host memory owned by the context, valid
 * until its next counting call.  Errors as hsk_count, and HSK_EOVERFLOW for
 * 2^32 reads or more, or a read of 2^32 bases or more. */
typedef struct {
    hsk_result counts;
    uint64_t n_occ;               /* occurrences of the kept k-mers (the sum of their counts) */
    const uint64_t* occ_offsets;  /* counts.n_pairs + 1 entries */
    const uint32_t* occ_read;     /* n_occ read indices */
    const uint32_t* occ_pos;      /* n_occ positions in the read */
} hsk_ext_result;
int hsk_count_ext(hsk_ctx* ctx, const char* reads, const uint64_t* offsets, uint64_t n_reads, int k, int m,
                  uint32_t lo, uint32_t hi, hsk_ext_result* out);

/* Copy the arrays of a result (as returned by any counting call on this
 * context) into caller memory: kmers_dst n_pairs * key_words words,
 * counts_dst n_pairs words, hist_dst hist_len words; any destination may be
 * NULL to skip it.  dst_on_device = 1 when the destinations are device
 * pointers.  Ordered on `stream` and complete on return. */
int hsk_result_copy(hsk_ctx* ctx, const hsk_result* res, uint64_t* kmers_dst, uint32_t* counts_dst,
                    uint64_t* hist_dst, int dst_on_device, void* stream);

/* Batched form: count n_jobs independent host-resident read sets.  The jobs
 * are queued, largest first, on the context's serving slots (child contexts
 * with their own streams and device arenas, running side by side).  A job of
 * at most the small-job limit of bases (default 2^28) is counted together
 * with other queued small jobs of the same k, m, lo and hi, up to a pack of
 * 2^28 bases by default (the autotuner picks both), by one pass of the
 * pipeline: their bases share one device buffer, each job owns a range of
 * minimizer buckets, and every launch serves all of them (Sec. 3.4's
 * independent tasks on shared workers).  Larger jobs run alone, on their
 * slot's highest-priority stream, so packs on the other slots fill the gaps
 * around them instead of slowing them down.  Each outs[i]
 * is bit-identical to what hsk_count() returns for jobs[i] alone, except
 * n_supermers and device_ms, which describe the pass that counted it (a
 * packed pass forms supermers with its own bucket count and times all its
 * jobs together).  Result arrays are host memory owned by the context, valid
 * until the next counting call.  With hsk_config.autotune set, the call first
 * applies the parameters hsk_autotune recorded for this class of job mix.
 * Errors as hsk_count; every job is attempted, and the first failing job's
 * code is returned with its index in hsk_last_error; on error no result is
 * valid. */
int hsk_count_batch(hsk_ctx* ctx, const hsk_job* jobs, uint32_t n_jobs, hsk_result* outs);

/* Page-lock (pin) an existing host buffer of `bytes` bytes so that copies
 * between it and the device run at link speed (the inputs of hsk_count and of
 * the batched and served forms); hsk_host_unpin(p) undoes it.  Pinning holds
 * the pages in RAM until unpinned; the buffer must stay allocated meanwhile.
 * HSK_ECUDA if the runtime refuses (already pinned, out of lockable memory). */
int hsk_host_pin(void* p, uint64_t bytes);
int hsk_host_unpin(void* p);

/* Parameters of the batched and served forms chosen by hsk_autotune. */
typedef struct {
    uint32_t group_div;          /* keys of a bucket group = 256 x on-chip sub-segment capacity / group_div */
    uint32_t plain_bucket_shift; /* large jobs run alone use (4096, or 8192 for k > 32) >> shift buckets */
    uint64_t pack_bases;         /* bases of one packed pass at most */
    uint64_t pack_small;         /* jobs of more bases run alone */
    int slots;                   /* serving slots (streams with their own arenas) */
    int trials;                  /* timed runs made */
    double first_s;              /* batch time of the sample with the parameters in force before */
    double best_s;               /* batch time of the sample with the chosen parameters */
} hsk_tune_result;

/* Autotuner: runs `jobs` (a sample of the mix to be counted) through
 * hsk_count_batch under candidate parameters -- slots, pack size, the small-job
 * limit, the bucket-group size, the bucket count of large jobs -- one
 * parameter at a time, timing each candidate after a warm-up run of it, at
 * most max_trials timed runs.  The fastest parameters are applied to the
 * context and recorded for the jobs' class (key width and binary order of
 * magnitude of the mean job size), and appended to hsk_config.tune_cache when
 * set.  *out (may be NULL) receives them.  Errors as hsk_count_batch. */
int hsk_autotune(hsk_ctx* ctx, const hsk_job* jobs, uint32_t n_jobs, int max_trials, hsk_tune_result* out);

/* The parameters in force on the context (the defaults until hsk_autotune or
 * a recorded entry changed them); trials, first_s and best_s are 0. */
int hsk_tune_current(hsk_ctx* ctx, hsk_tune_result* out);

/* Put parameters in force by hand (between calls; trials, first_s and best_s
 * are ignored).  HSK_EINVAL for values outside group_div 1..64,
 * plain_bucket_shift 0..4, pack_bases >= 2^20, slots 1..32. */
int hsk_tune_set(hsk_ctx* ctx, const hsk_tune_result* params);

/* Served form (continuous batching).  hsk_submit queues a job and returns a
 * ticket at once; a worker thread admits queued jobs while the device memory
 * they need fits the budget, runs admitted jobs concurrently on their own
 * streams (small jobs of one k, m, lo and hi packed into shared passes as in
 * hsk_count_batch; a job too large to pack on its slot's highest-priority
 * stream), and completes them in any order.  Inputs stay borrowed until the
 * job completes.  hsk_poll sets *done to 1 when the ticket's job finished;
 * hsk_wait blocks until then and fills *out (host arrays owned by the context,
 * valid until hsk_release(ticket)); hsk_cancel withdraws a job that has not
 * started (its wait then returns HSK_ECANCELED).  The submit API may be
 * called from any host thread. */
int hsk_submit(hsk_ctx* ctx, const hsk_job* job, uint64_t* ticket);
int hsk_poll(hsk_ctx* ctx, uint64_t ticket, int* done);
int hsk_wait(hsk_ctx* ctx, uint64_t ticket, hsk_result* out);
int hsk_cancel(hsk_ctx* ctx, uint64_t ticket);
int hsk_release(hsk_ctx* ctx, uint64_t ticket);

/* Latency of a completed served job: *queued_s = seconds from hsk_submit to
 * admission, *run_s = seconds from admission to completion.  HSK_EINVAL if
 * the job has not completed, HSK_ENOTFOUND for an unknown ticket. */
int hsk_ticket_times(hsk_ctx* ctx, uint64_t ticket, double* queued_s, double* run_s);

#ifdef __cplusplus
}
#endif

#endif /* HSK_H */
