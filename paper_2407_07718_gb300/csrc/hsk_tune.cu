// hsk_tune.cu -- autotuner of the batched and served forms.
//
// The forms have a handful of parameters whose best values depend on the
// job mix and the GPU: the bucket-group size of the on-chip sort (keys per
// group = 256 sub-segments x on-chip capacity / group_div), the bucket count
// of large jobs run alone, the largest pack of small jobs counted by one
// pass, the job size above which a job runs alone, and the number of serving
// slots (streams).  hsk_autotune measures them on sample jobs: it runs the
// jobs through hsk_count_batch under candidate values, one parameter at a
// time (coordinate descent, each candidate timed after one warm-up run of
// the same configuration), keeps the fastest, applies it to the context and
// records it under the jobs' class -- key width and size class -- in the
// context's table and, when the context has a cache file, in that file.
// With hsk_config.autotune set, hsk_count_batch applies the recorded entry
// of its own class before it runs.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "../../include/hsk.h"
#include "hsk_runtime.h"

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

hsk_ctx::Tune defaults() {
    hsk_ctx::Tune t;
    t.group_div = 3;
    t.plain_bucket_shift = 0;
    t.pack_bases = 256ull << 20;
    t.pack_small = 256ull << 20;
    t.slots = 4;
    return t;
}

bool same_tune(const hsk_ctx::Tune& a, const hsk_ctx::Tune& b) {
    return a.group_div == b.group_div && a.plain_bucket_shift == b.plain_bucket_shift &&
           a.pack_bases == b.pack_bases && a.pack_small == b.pack_small && a.slots == b.slots;
}

std::string line_of(const std::string& key, const hsk_ctx::Tune& t) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s group_div=%u plain_bucket_shift=%u pack_bases=%llu pack_small=%llu slots=%d",
             key.c_str(), t.group_div, t.plain_bucket_shift, (unsigned long long)t.pack_bases,
             (unsigned long long)t.pack_small, t.slots);
    return buf;
}

bool parse_line(const char* s, std::string& key, hsk_ctx::Tune& t) {
    char k[128];
    unsigned gd = 0, ps = 0;
    unsigned long long pb = 0, sm = 0;
    int sl = 0;
    if (sscanf(s, "%127s group_div=%u plain_bucket_shift=%u pack_bases=%llu pack_small=%llu slots=%d", k, &gd, &ps,
               &pb, &sm, &sl) != 6)
        return false;
    if (gd < 1 || gd > 64 || ps > 4 || pb < (1u << 20) || sl < 1 || sl > 32) return false;
    key = k;
    t.group_div = gd;
    t.plain_bucket_shift = ps;
    t.pack_bases = pb;
    t.pack_small = sm;
    t.slots = sl;
    return true;
}

}  // namespace

// Class of a job mix: key width of its jobs ("u64", "u128" or "mixed") and
// the binary order of magnitude of its mean bases per job.
std::string hsk_tune_class(const hsk_job* jobs, uint32_t n) {
    bool narrow = false, wide = false;
    double bases = 0;
    for (uint32_t i = 0; i < n; ++i) {
        (jobs[i].k <= 32 ? narrow : wide) = true;
        bases += jobs[i].n_reads ? (double)jobs[i].offsets[jobs[i].n_reads] : 0.0;
    }
    const double mean = n ? bases / n : 0.0;
    const int s = mean >= 1.0 ? (int)std::floor(std::log2(mean)) : 0;
    return std::string(narrow && wide ? "mixed" : wide ? "u128" : "u64") + ":2^" + std::to_string(s);
}

// Cached parameters from the context's file (later lines win).
void hsk_tune_load(hsk_ctx* c) {
    if (c->tune_path.empty()) return;
    FILE* f = fopen(c->tune_path.c_str(), "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        std::string key;
        hsk_ctx::Tune t;
        if (!parse_line(line, key, t)) continue;
        bool found = false;
        for (auto& e : c->tuned)
            if (e.first == key) {
                e.second = t;
                found = true;
            }
        if (!found) c->tuned.emplace_back(key, t);
    }
    fclose(f);
}

// Parameters of the class, if recorded.
bool hsk_tune_lookup(hsk_ctx* c, const std::string& key, hsk_ctx::Tune* out) {
    std::lock_guard<std::mutex> g(c->tune_mu);
    for (auto& e : c->tuned)
        if (e.first == key) {
            *out = e.second;
            return true;
        }
    return false;
}

// Make t the context's parameters.  Serving slots are children of the
// context: a new slot count restarts them (between calls, when none runs).
void hsk_tune_apply(hsk_ctx* c, const hsk_ctx::Tune& t) {
    const bool restart = c->serve && t.slots != c->tune.slots;
    if (restart) hsk_serve_shutdown(c);
    c->tune = t;
    if (c->serve) hsk_serve_set_tune(c);
}

extern "C" int hsk_autotune(hsk_ctx* c, const hsk_job* jobs, uint32_t n_jobs, int max_trials,
                            hsk_tune_result* out) {
    return hsk_guarded(c, [&]() -> int {
        if (!c || !jobs || n_jobs == 0 || max_trials < 1) return HSK_EINVAL;
        std::vector<hsk_result> outs(n_jobs);
        hsk_ctx::Tune cur = c->tune;
        const hsk_ctx::Tune def = defaults();
        if (!cur.group_div) cur.group_div = def.group_div;
        if (!cur.pack_bases) cur.pack_bases = def.pack_bases;
        if (!cur.pack_small) cur.pack_small = def.pack_small;
        if (!cur.slots) cur.slots = def.slots;
        int trials = 0;
        struct Flag {  // batches of the trials use the trial parameters, not the recorded ones
            hsk_ctx* c;
            explicit Flag(hsk_ctx* x) : c(x) { c->tuning = true; }
            ~Flag() { c->tuning = false; }
        } flag(c);
        // one warm-up run of the configuration, then the timed run
        auto trial = [&](const hsk_ctx::Tune& t, double* secs) -> int {
            hsk_tune_apply(c, t);
            int rc = hsk_count_batch(c, jobs, n_jobs, outs.data());
            if (rc != HSK_OK) return rc;
            const double t0 = now_s();
            rc = hsk_count_batch(c, jobs, n_jobs, outs.data());
            *secs = now_s() - t0;
            ++trials;
            return rc;
        };
        double best = 0;
        TRY(trial(cur, &best));
        const double first = best;
        const std::vector<uint32_t> divs = {2, 3, 4, 6};
        const std::vector<uint32_t> shifts = {0, 1};
        // packs past 512 MB gained no throughput on the batched workload and
        // lengthened served latency under load (a request waits for its pack)
        const std::vector<uint64_t> packs = {64ull << 20, 128ull << 20, 256ull << 20, 512ull << 20};
        const std::vector<uint64_t> smalls = {64ull << 20, 256ull << 20, 1ull << 30};
        const std::vector<int> slots = {2, 3, 4, 6};
        // a candidate replaces the current value only when it is clearly faster
        auto consider = [&](const hsk_ctx::Tune& t) -> int {
            if (trials >= max_trials || same_tune(t, cur)) return HSK_OK;
            double s = 0;
            TRY(trial(t, &s));
            if (s < best * 0.97) {
                best = s;
                cur = t;
            }
            return HSK_OK;
        };
        for (int v : slots) {
            hsk_ctx::Tune t = cur;
            t.slots = v;
            TRY(consider(t));
        }
        for (uint64_t v : packs) {
            hsk_ctx::Tune t = cur;
            t.pack_bases = v;
            TRY(consider(t));
        }
        for (uint64_t v : smalls) {
            hsk_ctx::Tune t = cur;
            t.pack_small = v;
            TRY(consider(t));
        }
        for (uint32_t v : divs) {
            hsk_ctx::Tune t = cur;
            t.group_div = v;
            TRY(consider(t));
        }
        for (uint32_t v : shifts) {
            hsk_ctx::Tune t = cur;
            t.plain_bucket_shift = v;
            TRY(consider(t));
        }
        hsk_tune_apply(c, cur);
        const std::string key = hsk_tune_class(jobs, n_jobs);
        {
            std::lock_guard<std::mutex> g(c->tune_mu);
            bool found = false;
            for (auto& e : c->tuned)
                if (e.first == key) {
                    e.second = cur;
                    found = true;
                }
            if (!found) c->tuned.emplace_back(key, cur);
        }
        if (!c->tune_path.empty()) {
            FILE* f = fopen(c->tune_path.c_str(), "a");
            if (!f) {
                hsk_set_error(c, "cannot append to the tuning cache %s", c->tune_path.c_str());
                return HSK_EINVAL;
            }
            fprintf(f, "%s\n", line_of(key, cur).c_str());
            fclose(f);
        }
        if (out) {
            memset(out, 0, sizeof(*out));
            out->group_div = cur.group_div;
            out->plain_bucket_shift = cur.plain_bucket_shift;
            out->pack_bases = cur.pack_bases;
            out->pack_small = cur.pack_small;
            out->slots = cur.slots;
            out->best_s = best;
            out->first_s = first;
            out->trials = trials;
        }
        return HSK_OK;
    });
}

extern "C" int hsk_tune_current(hsk_ctx* c, hsk_tune_result* out) {
    if (!c || !out) return HSK_EINVAL;
    const hsk_ctx::Tune def = defaults();
    const hsk_ctx::Tune& t = c->tune;
    memset(out, 0, sizeof(*out));
    out->group_div = t.group_div ? t.group_div : def.group_div;
    out->plain_bucket_shift = t.plain_bucket_shift;
    out->pack_bases = t.pack_bases ? t.pack_bases : def.pack_bases;
    out->pack_small = t.pack_small ? t.pack_small : def.pack_small;
    out->slots = t.slots ? t.slots : def.slots;
    return HSK_OK;
}

extern "C" int hsk_tune_set(hsk_ctx* c, const hsk_tune_result* p) {
    if (!c || !p) return HSK_EINVAL;
    if (p->group_div < 1 || p->group_div > 64 || p->plain_bucket_shift > 4 || p->pack_bases < (1u << 20) ||
        p->slots < 1 || p->slots > 32)
        return HSK_EINVAL;
    return hsk_guarded(c, [&]() -> int {
        hsk_ctx::Tune t;
        t.group_div = p->group_div;
        t.plain_bucket_shift = p->plain_bucket_shift;
        t.pack_bases = p->pack_bases;
        t.pack_small = p->pack_small;
        t.slots = p->slots;
        hsk_tune_apply(c, t);
        return HSK_OK;
    });
}
