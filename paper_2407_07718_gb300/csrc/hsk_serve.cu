// hsk_serve.cu -- batched and served forms of the counter.
//
// Served form (continuous batching): jobs are queued by hsk_submit and taken
// by a fixed set of slots.  Each slot is a child context with its own stream
// and its own device arena, kept resident between jobs, so admitted jobs run
// concurrently on the device.  A queued job is admitted when a slot is free
// and the device memory it needs -- estimated from its size -- fits the
// budget next to what the other slots hold; idle slots give their arenas back
// when a job would not fit otherwise.  Jobs complete in any order.
//
// Small jobs are batched at the kernel level: a slot that takes a small job
// also takes the other queued small jobs with the same k, m and filter (up to
// a pack size, and within the budget) and counts them all by one pass of the
// pipeline (hsk_pack.cu), so they share every launch and synchronization.
// Jobs that arrive while a pack runs wait for the next free slot.
//
// Batched form: hsk_count_batch queues many independent read sets on the same
// slots, largest first, and returns when all are done; the small sets are
// packed as above.
#include <algorithm>
#include <cstdlib>
#include <chrono>
#include <cstring>

#include "hsk_internal.h"
#include "hsk_pack.h"
#include "hsk_runtime.h"

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum TicketState { T_QUEUED = 0, T_RUNNING = 1, T_DONE = 2, T_CANCELED = 3 };

struct Ticket {
    hsk_job job{};
    int state = T_QUEUED;
    int rc = HSK_OK;
    std::string err;
    HostResult res;
    size_t est = 0;
    uint64_t bases = 0;
    bool packable = false;  // small enough to share a pass with other jobs
    double t_submit = 0, t_start = 0, t_done = 0;
};

}  // namespace

struct ServeState {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, std::unique_ptr<Ticket>> tickets;
    uint64_t next_ticket = 1;
    std::vector<hsk_ctx*> slots;
    std::vector<size_t> slot_est;   // estimate of the running job (0 when idle)
    std::vector<int> slot_busy;
    std::vector<std::thread> workers;
    size_t budget = 0;
    bool stop = false;
};

// Device bytes a job needs at most (inputs, encoding, records, sort buffers,
// output, fixed tables): an upper bound from its size alone.
static size_t job_estimate(const hsk_job& j) {
    uint64_t nb = j.n_reads ? j.offsets[j.n_reads] : 0;
    double kb = j.k <= 32 ? 8.0 : 16.0;
    double rec = j.k <= 32 ? 16.0 : 32.0;
    double n = (double)nb;  // windows <= bases
    double bytes = n * (1.0 + 0.25 + 0.25) + 8.0 * (double)(j.n_reads + 1) + n * rec / 2.0 +
                   n * (2 * kb + 4 + 1 + kb + 4) + (96u << 20);
    return (size_t)bytes;
}

// Pack limits (the tuned values when set): sets of more bases run alone;
// a pack holds at most pack_bases bases.
static uint64_t pack_small_limit(const hsk_ctx* c) {
    return c->tune.pack_small ? c->tune.pack_small : (256ull << 20);
}
static uint64_t pack_bases_limit(const hsk_ctx* c) {
    return c->tune.pack_bases ? c->tune.pack_bases : (256ull << 20);
}
constexpr uint32_t PACK_MAX_SETS = 1024;

// Device bytes of a pack of S sets holding `bases` bases and `reads` reads.
static size_t pack_estimate(uint64_t bases, uint64_t reads, int k, uint32_t S, uint32_t hist_len) {
    hsk_job j{};
    j.k = k;
    uint64_t off[2] = {0, bases};
    j.offsets = off;
    j.n_reads = 1;
    size_t e = job_estimate(j) + (size_t)8 * (reads + S) + (size_t)S * hist_len * 8 +
               (size_t)S * 1024 * 8;  // inputs and offsets, per-set histograms, set padding
    return e;
}

static bool same_class(const hsk_job& a, const hsk_job& b) {
    return a.k == b.k && a.m == b.m && a.lo == b.lo && a.hi == b.hi;
}

static size_t slot_held(ServeState* S, int i) {
    size_t h = S->slots[i]->allocated;
    return S->slot_busy[i] ? std::max(h, S->slot_est[i]) : h;
}

static void trim_ctx(hsk_ctx* c) {
    for (DevBuf* b : c->all_bufs()) {
        if (b->p) {
            cudaFree(b->p);
            c->allocated -= b->cap;
        }
        b->p = nullptr;
        b->cap = 0;
    }
}

static void worker_main(hsk_ctx* parent, ServeState* S, int slot) {
    hsk_ctx* c = S->slots[slot];
    cudaSetDevice(parent->cfg.device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        Ticket* T = nullptr;
        for (;;) {
            if (S->stop) return;
            if (!S->queue.empty()) {
                uint64_t cand = S->queue.front();
                Ticket* ct = S->tickets[cand].get();
                size_t others = 0;
                for (int i = 0; i < (int)S->slots.size(); ++i)
                    if (i != slot) others += slot_held(S, i);
                size_t mine = std::max(c->allocated, ct->est);
                if (others + mine > S->budget) {
                    // give back arenas of idle slots, then look again
                    for (int i = 0; i < (int)S->slots.size(); ++i)
                        if (i != slot && !S->slot_busy[i]) trim_ctx(S->slots[i]);
                    others = 0;
                    for (int i = 0; i < (int)S->slots.size(); ++i)
                        if (i != slot) others += slot_held(S, i);
                }
                bool alone = true;
                for (int i = 0; i < (int)S->slots.size(); ++i)
                    if (i != slot && S->slot_busy[i]) alone = false;
                // a job larger than the whole budget still runs when it is alone
                // (its own allocations then fail with HSK_ENOMEM if it truly does not fit)
                if (others + mine <= S->budget || alone) {
                    T = ct;
                    S->queue.pop_front();
                    break;
                }
            }
            S->cv_work.wait(lk);
        }
        // small job: other queued small jobs of its class join it in one pass
        std::vector<Ticket*> group{T};
        size_t est = T->est;
        if (T->packable) {
            uint64_t queued = T->bases;
            for (uint64_t id : S->queue) {
                Ticket* u = S->tickets[id].get();
                if (u->packable && same_class(u->job, T->job)) queued += u->bases;
            }
            // spread the queued small work over the slots, within the pack limit
            const uint64_t cap = std::min<uint64_t>(pack_bases_limit(parent),
                                                    std::max<uint64_t>(32ull << 20, queued / S->slots.size()));
            uint64_t bases = T->bases, reads = T->job.n_reads;
            const int kw = T->job.k <= 32 ? 1 : 2;
            const uint64_t gk = hsk_pack_group_keys(c, kw);
            uint32_t buckets = hsk_pack_set_buckets(T->bases, kw, gk);
            size_t others = 0;
            for (int i = 0; i < (int)S->slots.size(); ++i)
                if (i != slot) others += slot_held(S, i);
            for (auto it = S->queue.begin(); it != S->queue.end() && bases < cap && group.size() < PACK_MAX_SETS;) {
                Ticket* u = S->tickets[*it].get();
                const uint32_t ub = hsk_pack_set_buckets(u->bases, kw, gk);
                if (u->packable && same_class(u->job, T->job) && bases + u->bases <= cap &&
                    buckets + ub <= HSK_MAX_BUCKETS) {
                    const size_t e2 = pack_estimate(bases + u->bases, reads + u->job.n_reads, T->job.k,
                                                    (uint32_t)group.size() + 1, parent->cfg.hist_len);
                    if (others + std::max(c->allocated, e2) <= S->budget) {
                        group.push_back(u);
                        bases += u->bases;
                        reads += u->job.n_reads;
                        buckets += ub;
                        est = e2;
                        it = S->queue.erase(it);
                        continue;
                    }
                }
                ++it;
            }
        }
        const double t0 = now_s();
        for (Ticket* g : group) {
            g->state = T_RUNNING;
            g->t_start = t0;
        }
        S->slot_busy[slot] = 1;
        S->slot_est[slot] = est;
        lk.unlock();
        std::vector<HostResult> hrs(group.size());
        for (HostResult& h : hrs) h.set_pool(&parent->result_pool);
        std::vector<int> rcs(group.size(), HSK_OK);
        std::vector<std::string> errs(group.size());
        if (group.size() == 1) {
            const hsk_job job = group[0]->job;
            // A job too large to pack runs on the slot's highest-priority
            // stream: its blocks are dispatched before those of the packs on
            // the other slots, so it runs near its alone time (the tail of the
            // latency distribution) while the packs fill the gaps.
            cudaStream_t js = !group[0]->packable && c->hstream ? c->hstream : c->stream;
            rcs[0] = hsk_guarded(c, [&]() -> int {
                return hsk_count_host_on(c, job.reads, job.offsets, job.n_reads, job.k, job.m, job.lo, job.hi,
                                         js, c->in_reads, c->in_offsets, hrs[0]);
            });
            if (rcs[0] != HSK_OK) errs[0] = c->err_msg;
        } else {
            std::vector<PackSet> ps(group.size());
            for (size_t i = 0; i < group.size(); ++i) {
                ps[i].reads = group[i]->job.reads;
                ps[i].offsets = group[i]->job.offsets;
                ps[i].n_reads = group[i]->job.n_reads;
                ps[i].out = &hrs[i];
            }
            const hsk_job& j0 = group[0]->job;
            std::string fail;
            const int rc = hsk_guarded(c, [&]() -> int {
                return hsk_count_pack_host(c, ps.data(), (uint32_t)ps.size(), j0.k, j0.m, j0.lo, j0.hi, c->stream,
                                           &fail);
            });
            if (!fail.empty()) {
                parent->pack_fail.fetch_add(1);
                std::lock_guard<std::mutex> g2(parent->tune_mu);
                parent->pack_fail_msg = fail;
            }
            for (size_t i = 0; i < group.size(); ++i) {
                rcs[i] = rc != HSK_OK ? rc : ps[i].rc;
                errs[i] = rc != HSK_OK ? c->err_msg : ps[i].err;
                if (ps[i].alone) parent->pack_redo.fetch_add(1);
            }
            parent->pack_passes.fetch_add(1);
            parent->pack_sets.fetch_add(group.size());
        }
        lk.lock();
        const double t1 = now_s();
        for (size_t i = 0; i < group.size(); ++i) {
            Ticket* g = group[i];
            g->rc = rcs[i];
            g->err = rcs[i] == HSK_OK ? std::string() : errs[i];
            g->res = std::move(hrs[i]);
            g->res.R.kmers = g->res.kmers.data();
            g->res.R.counts = g->res.counts.data();
            g->res.R.hist = g->res.hist.data();
            g->t_done = t1;
            g->state = T_DONE;
        }
        S->slot_busy[slot] = 0;
        S->slot_est[slot] = 0;
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

static int serve_start(hsk_ctx* c) {
    if (c->serve) return HSK_OK;
    ServeState* S = new ServeState();
    S->budget = c->budget > c->allocated ? c->budget - c->allocated : 0;
    // slots (child contexts running jobs side by side); HSK_SERVE_SLOTS overrides
    int n_slots = c->tune.slots ? c->tune.slots : 4;
    if (const char* e = getenv("HSK_SERVE_SLOTS")) {
        const int v = atoi(e);
        if (v >= 1 && v <= 32) n_slots = v;
    }
    for (int i = 0; i < n_slots; ++i) {
        hsk_config cfg = c->cfg;
        cfg.hbm_budget = S->budget;
        hsk_ctx* child = nullptr;
        int rc = hsk_create(&child, &cfg);
        if (rc != HSK_OK) {
            for (hsk_ctx* s : S->slots) hsk_destroy(s);
            delete S;
            hsk_set_error(c, "could not create serving slot %d", i);
            return rc;
        }
        child->tune = c->tune;
        S->slots.push_back(child);
        S->slot_est.push_back(0);
        S->slot_busy.push_back(0);
    }
    c->serve = S;
    for (int i = 0; i < n_slots; ++i) S->workers.emplace_back(worker_main, c, S, i);
    return HSK_OK;
}

void hsk_serve_set_tune(hsk_ctx* c) {
    if (!c || !c->serve) return;
    std::lock_guard<std::mutex> g(c->serve->mu);
    for (hsk_ctx* s : c->serve->slots) s->tune = c->tune;
}

void hsk_serve_shutdown(hsk_ctx* c) {
    if (!c || !c->serve) return;
    ServeState* S = c->serve;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    for (hsk_ctx* s : S->slots) hsk_destroy(s);
    delete S;
    c->serve = nullptr;
}

static int validate_job(hsk_ctx* c, const hsk_job* j) {
    if (!j) return HSK_EINVAL;
    if (j->k < 1 || j->k > 64 || j->m < 1 || j->m > j->k || j->m > 32 || j->lo > j->hi) {
        hsk_set_error(c, "job has k=%d m=%d lo=%u hi=%u outside their ranges", j->k, j->m, j->lo, j->hi);
        return HSK_EINVAL;
    }
    if (j->n_reads && !j->offsets) {
        hsk_set_error(c, "job has NULL offsets");
        return HSK_EINVAL;
    }
    if (j->n_reads && j->offsets[j->n_reads] > 0 && !j->reads) {
        hsk_set_error(c, "job has NULL reads");
        return HSK_EINVAL;
    }
    return HSK_OK;
}

extern "C" int hsk_submit(hsk_ctx* c, const hsk_job* job, uint64_t* ticket) {
    return hsk_guarded(c, [&]() -> int {
        if (!c || !ticket) return HSK_EINVAL;
        int rc = validate_job(c, job);
        if (rc != HSK_OK) return rc;
        rc = serve_start(c);
        if (rc != HSK_OK) return rc;
        ServeState* S = c->serve;
        auto T = std::make_unique<Ticket>();
        T->job = *job;
        T->est = job_estimate(*job);
        T->bases = job->n_reads ? job->offsets[job->n_reads] : 0;
        T->packable = T->bases <= pack_small_limit(c);
        T->t_submit = now_s();
        std::lock_guard<std::mutex> g(S->mu);
        uint64_t id = S->next_ticket++;
        S->tickets[id] = std::move(T);
        S->queue.push_back(id);
        *ticket = id;
        S->cv_work.notify_all();
        return HSK_OK;
    });
}

extern "C" int hsk_poll(hsk_ctx* c, uint64_t ticket, int* done) {
    if (!c || !done) return HSK_EINVAL;
    if (!c->serve) return HSK_ENOTFOUND;
    ServeState* S = c->serve;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return HSK_ENOTFOUND;
    *done = it->second->state == T_DONE || it->second->state == T_CANCELED;
    return HSK_OK;
}

static void fill_out(const HostResult& hr, hsk_result* out) {
    memset(out, 0, sizeof(*out));
    const DevResult& R = hr.R;
    out->n_pairs = R.n_pairs;
    out->kmers = hr.kmers.data();
    out->counts = hr.counts.data();
    out->hist = hr.hist.data();
    out->hist_len = R.hist_len;
    out->key_words = R.key_words;
    out->n_windows = R.n_windows;
    out->n_distinct = R.n_distinct;
    out->max_count = R.max_count;
    out->n_chunks = R.n_chunks;
    out->n_supermers = R.n_supermers;
    out->device_ms = R.device_ms;
}

extern "C" int hsk_wait(hsk_ctx* c, uint64_t ticket, hsk_result* out) {
    return hsk_guarded(c, [&]() -> int {
        if (!c || !out) return HSK_EINVAL;
        if (!c->serve) return HSK_ENOTFOUND;
        ServeState* S = c->serve;
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->tickets.find(ticket);
        if (it == S->tickets.end()) return HSK_ENOTFOUND;
        Ticket* T = it->second.get();
        S->cv_done.wait(lk, [&] { return T->state == T_DONE || T->state == T_CANCELED; });
        if (T->state == T_CANCELED) return HSK_ECANCELED;
        if (T->rc != HSK_OK) {
            c->err_msg = T->err;
            return T->rc;
        }
        fill_out(T->res, out);
        return HSK_OK;
    });
}

extern "C" int hsk_cancel(hsk_ctx* c, uint64_t ticket) {
    if (!c) return HSK_EINVAL;
    if (!c->serve) return HSK_ENOTFOUND;
    ServeState* S = c->serve;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return HSK_ENOTFOUND;
    if (it->second->state != T_QUEUED) return HSK_EINVAL;  // already running or finished
    S->queue.erase(std::remove(S->queue.begin(), S->queue.end(), ticket), S->queue.end());
    it->second->state = T_CANCELED;
    S->cv_done.notify_all();
    return HSK_OK;
}

extern "C" int hsk_release(hsk_ctx* c, uint64_t ticket) {
    if (!c) return HSK_EINVAL;
    if (!c->serve) return HSK_ENOTFOUND;
    ServeState* S = c->serve;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return HSK_ENOTFOUND;
    if (it->second->state == T_QUEUED || it->second->state == T_RUNNING) return HSK_EINVAL;
    S->tickets.erase(it);
    return HSK_OK;
}

extern "C" int hsk_ticket_times(hsk_ctx* c, uint64_t ticket, double* queued_s, double* run_s) {
    if (!c || !c->serve) return HSK_ENOTFOUND;
    ServeState* S = c->serve;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return HSK_ENOTFOUND;
    Ticket* T = it->second.get();
    if (T->state != T_DONE) return HSK_EINVAL;
    if (queued_s) *queued_s = T->t_start - T->t_submit;
    if (run_s) *run_s = T->t_done - T->t_start;
    return HSK_OK;
}

// ---------------------------------------------------------------------------
// batched form: the jobs go through the serving slots, largest first
// ---------------------------------------------------------------------------
extern "C" int hsk_count_batch(hsk_ctx* c, const hsk_job* jobs, uint32_t n_jobs, hsk_result* outs) {
    return hsk_guarded(c, [&]() -> int {
        if (!c || (n_jobs && (!jobs || !outs))) return HSK_EINVAL;
        for (uint32_t i = 0; i < n_jobs; ++i) {
            int rc = validate_job(c, jobs + i);
            if (rc != HSK_OK) return rc;
        }
        CK(cudaSetDevice(c->cfg.device));
        c->batch_res.clear();
        c->batch_res.resize(n_jobs);
        if (n_jobs == 0) return HSK_OK;
        if (c->cfg.autotune && !c->tuning) {  // parameters recorded for this class of mix
            hsk_ctx::Tune t;
            if (hsk_tune_lookup(c, hsk_tune_class(jobs, n_jobs), &t)) hsk_tune_apply(c, t);
        }
        TRY(serve_start(c));
        ServeState* S = c->serve;
        // Largest job first (longest-processing-time order): with the slots
        // running side by side, the big jobs start early and the small ones fill
        // the gaps, which shortens the makespan.
        std::vector<uint32_t> order(n_jobs);
        for (uint32_t i = 0; i < n_jobs; ++i) order[i] = i;
        auto bases = [&](uint32_t i) { return jobs[i].n_reads ? jobs[i].offsets[jobs[i].n_reads] : 0; };
        std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return bases(a) > bases(b); });
        std::vector<uint64_t> ids(n_jobs);
        {
            std::lock_guard<std::mutex> g(S->mu);
            for (uint32_t i : order) {
                auto T = std::make_unique<Ticket>();
                T->job = jobs[i];
                T->est = job_estimate(jobs[i]);
                T->bases = bases(i);
                T->packable = T->bases <= pack_small_limit(c);
                T->t_submit = now_s();
                uint64_t id = S->next_ticket++;
                S->tickets[id] = std::move(T);
                S->queue.push_back(id);
                ids[i] = id;
            }
        }
        S->cv_work.notify_all();
        int first_rc = HSK_OK;
        std::string first_err;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (uint32_t i = 0; i < n_jobs; ++i) {
                Ticket* T = S->tickets[ids[i]].get();
                S->cv_done.wait(lk, [&] { return T->state == T_DONE; });
                if (T->rc != HSK_OK && first_rc == HSK_OK) {
                    first_rc = T->rc;
                    first_err = "job " + std::to_string(i) + ": " + T->err;
                }
                c->batch_res[i] = std::move(T->res);
                S->tickets.erase(ids[i]);
            }
        }
        if (first_rc != HSK_OK) {
            c->err_msg = first_err;
            return first_rc;
        }
        for (uint32_t i = 0; i < n_jobs; ++i) fill_out(c->batch_res[i], outs + i);
        return HSK_OK;
    });
}

extern "C" int hsk_debug_pack_stats(hsk_ctx* c, uint64_t* passes, uint64_t* sets, uint64_t* alone) {
    if (!c) return HSK_EINVAL;
    if (passes) *passes = c->pack_passes.load();
    if (sets) *sets = c->pack_sets.load();
    if (alone) *alone = c->pack_redo.load();
    return HSK_OK;
}

extern "C" const char* hsk_debug_pack_failure(hsk_ctx* c, uint64_t* failed_passes) {
    if (!c) return "";
    if (failed_passes) *failed_passes = c->pack_fail.load();
    std::lock_guard<std::mutex> g(c->tune_mu);
    return c->pack_fail_msg.c_str();
}
