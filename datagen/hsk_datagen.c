/* hsk_datagen.c -- seeded synthetic read sets shaped like the short-read and
 * long-read workloads k-mer counters are run on.
 *
 * Shared by the library's tests/benchmark and by the oracle checks.  It holds
 * none of the counting method's arithmetic: it only simulates genomes and
 * sequencing reads as ASCII bytes plus CSR offsets.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * splitmix64 (Steele, Lea & Flood, 2014), both written here from their
 * published definitions.  Integer thresholds decide per-base events, so the
 * base-level choices are identical on every platform; read and fragment
 * lengths go through log/exp/cos and may differ in the last unit between libm
 * builds.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint64_t s[4];
} rng_t;

static uint64_t splitmix64_next(uint64_t* x) {
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(rng_t* r) {
    uint64_t* s = r->s;
    uint64_t result = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
}

static void rng_seed(rng_t* r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&x);
}

/* Derived seed for sub-stream i of a seed (per set / per request). */
uint64_t dg_derive_seed(uint64_t seed, uint64_t i) {
    uint64_t x = seed ^ (0xd1b54a32d192ed03ULL * (i + 1));
    splitmix64_next(&x);
    return splitmix64_next(&x);
}

static double rng_unit(rng_t* r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

static uint64_t rng_below(rng_t* r, uint64_t n) { /* n > 0; negligible bias for n << 2^64 */
    return (uint64_t)(((unsigned __int128)rng_next(r) * n) >> 64);
}

static uint64_t prob_threshold(double p) {
    if (p <= 0) return 0;
    if (p >= 1) return UINT64_MAX;
    return (uint64_t)(p * 18446744073709551616.0);
}

static double rng_normal(rng_t* r) { /* Box-Muller */
    double u1 = rng_unit(r), u2 = rng_unit(r);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

static const char ACGT[4] = {'A', 'C', 'G', 'T'};

static char complement(char c) {
    switch (c) {
        case 'A': return 'T';
        case 'C': return 'G';
        case 'G': return 'C';
        case 'T': return 'A';
        default: return c;
    }
}

typedef struct {
    uint64_t seed;
    uint64_t genome_len;
    /* GC-skewed segment: [gc_start, gc_start+gc_len) drawn with P(G)=P(C)=gc/2 */
    uint64_t gc_start, gc_len;
    double gc;
    /* repeat families overwritten into the genome */
    uint32_t rep_families, rep_copies, rep_len_min, rep_len_max;
    double rep_div_max; /* per-copy substitution divergence ~ U[0, rep_div_max] */
    /* reads */
    int read_model;      /* 0 fixed length, 1 log-normal length, 2 paired fixed length */
    uint64_t n_reads;    /* model 0: exact read count (0 = from coverage) */
    double coverage;
    uint32_t read_len;   /* models 0 and 2 */
    double ln_mu, ln_sigma;
    uint32_t len_min;    /* model 1: lengths below are redrawn */
    double frag_mean, frag_sd; /* model 2 */
    double p_rc;         /* models 0 and 1: reverse-complement probability */
    double p_sub, p_ins, p_del, p_n;
} dg_params;

typedef struct {
    char* reads;
    uint64_t* offsets;
    uint64_t n_reads;
    uint64_t n_bases;
    uint64_t cap;
    uint64_t ocap;
} dg_out;

void dg_free(dg_out* o) {
    if (!o) return;
    free(o->reads);
    free(o->offsets);
    o->reads = NULL;
    o->offsets = NULL;
}

static int out_reserve(dg_out* o, uint64_t more) {
    if (o->n_bases + more > o->cap) {
        uint64_t nc = o->cap ? o->cap : (1u << 20);
        while (nc < o->n_bases + more) nc *= 2;
        char* p = (char*)realloc(o->reads, nc);
        if (!p) return -1;
        o->reads = p;
        o->cap = nc;
    }
    if (o->n_reads + 2 > o->ocap) {
        uint64_t nc = o->ocap ? o->ocap * 2 : 1024;
        uint64_t* p = (uint64_t*)realloc(o->offsets, nc * sizeof(uint64_t));
        if (!p) return -1;
        o->offsets = p;
        o->ocap = nc;
    }
    return 0;
}

static void make_genome(const dg_params* P, rng_t* r, char* g) {
    uint64_t L = P->genome_len;
    for (uint64_t i = 0; i < L; i += 32) {
        uint64_t x = rng_next(r);
        for (int j = 0; j < 32 && i + j < L; ++j) g[i + j] = ACGT[(x >> (2 * j)) & 3];
    }
    if (P->gc_len > 0) {
        /* cumulative thresholds: G below gc/2, C below gc, A below gc + (1-gc)/2, else T */
        uint64_t tg = prob_threshold(P->gc / 2), tc = prob_threshold(P->gc),
                 ta = prob_threshold(P->gc + (1.0 - P->gc) / 2);
        for (uint64_t i = P->gc_start; i < P->gc_start + P->gc_len && i < L; ++i) {
            uint64_t x = rng_next(r);
            g[i] = x < tg ? 'G' : x < tc ? 'C' : x < ta ? 'A' : 'T';
        }
    }
    for (uint32_t f = 0; f < P->rep_families; ++f) {
        double lo = log((double)P->rep_len_min), hi = log((double)P->rep_len_max);
        uint64_t rl = (uint64_t)exp(lo + rng_unit(r) * (hi - lo));
        if (rl > L) rl = L;
        char* fam = (char*)malloc(rl ? rl : 1);
        for (uint64_t i = 0; i < rl; ++i) fam[i] = ACGT[rng_next(r) & 3];
        for (uint32_t c = 0; c < P->rep_copies; ++c) {
            uint64_t at = rng_below(r, L - rl + 1);
            uint64_t td = prob_threshold(rng_unit(r) * P->rep_div_max);
            for (uint64_t i = 0; i < rl; ++i) {
                char b = fam[i];
                if (rng_next(r) < td) b = ACGT[((b == 'A' ? 0 : b == 'C' ? 1 : b == 'G' ? 2 : 3) + 1 + rng_below(r, 3)) & 3];
                g[at + i] = b;
            }
        }
        free(fam);
    }
}

/* Copy template t[0..len) (optionally reverse-complemented) into the output as
 * one read, applying insertions, deletions, substitutions and N's. */
static int emit_read(dg_out* o, const dg_params* P, rng_t* r, const char* t, uint64_t len, int rc,
                     uint64_t th_sub, uint64_t th_ins, uint64_t th_del, uint64_t th_n) {
    if (out_reserve(o, 2 * len + 8)) return -1;
    char* dst = o->reads + o->n_bases;
    uint64_t n = 0;
    for (uint64_t i = 0; i < len; ++i) {
        char b = rc ? complement(t[len - 1 - i]) : t[i];
        if (th_ins | th_del) {
            uint64_t x = rng_next(r);
            if (x < th_ins) dst[n++] = ACGT[rng_next(r) & 3];
            else if (x < th_ins + th_del) continue;
        }
        if (th_sub && rng_next(r) < th_sub) {
            int c = b == 'A' ? 0 : b == 'C' ? 1 : b == 'G' ? 2 : 3;
            b = ACGT[(c + 1 + rng_below(r, 3)) & 3];
        }
        if (th_n && rng_next(r) < th_n) b = 'N';
        dst[n++] = b;
    }
    o->offsets[o->n_reads] = o->n_bases;
    o->n_bases += n;
    o->n_reads += 1;
    o->offsets[o->n_reads] = o->n_bases;
    return 0;
}

/* Simulate one read set.  Returns 0 or -1 (allocation failure). */
int dg_generate(const dg_params* P, dg_out* o) {
    memset(o, 0, sizeof(*o));
    rng_t r;
    rng_seed(&r, P->seed);
    uint64_t L = P->genome_len;
    char* g = (char*)malloc(L ? L : 1);
    if (!g) return -1;
    make_genome(P, &r, g);
    uint64_t th_sub = prob_threshold(P->p_sub), th_ins = prob_threshold(P->p_ins),
             th_del = prob_threshold(P->p_del), th_n = prob_threshold(P->p_n);
    if (out_reserve(o, 0)) { free(g); return -1; }
    o->offsets[0] = 0;
    double target = P->coverage * (double)L;
    if (P->read_model == 0) {
        uint64_t rl = P->read_len < L ? P->read_len : L;
        uint64_t n = P->n_reads ? P->n_reads : (uint64_t)llround(target / (double)(rl ? rl : 1));
        for (uint64_t i = 0; i < n; ++i) {
            uint64_t at = rng_below(&r, L - rl + 1);
            int rc = rng_next(&r) < prob_threshold(P->p_rc);
            if (emit_read(o, P, &r, g + at, rl, rc, th_sub, th_ins, th_del, th_n)) { free(g); return -1; }
        }
    } else if (P->read_model == 1) {
        double total = 0;
        while (total < target) {
            uint64_t rl;
            do {
                rl = (uint64_t)exp(P->ln_mu + P->ln_sigma * rng_normal(&r));
            } while (rl < P->len_min);
            if (rl > L) rl = L;
            uint64_t at = rng_below(&r, L - rl + 1);
            int rc = rng_next(&r) < prob_threshold(P->p_rc);
            if (emit_read(o, P, &r, g + at, rl, rc, th_sub, th_ins, th_del, th_n)) { free(g); return -1; }
            total += (double)rl;
        }
    } else {
        uint64_t rl = P->read_len < L ? P->read_len : L;
        uint64_t pairs = (uint64_t)llround(target / (2.0 * (double)(rl ? rl : 1)));
        for (uint64_t i = 0; i < pairs; ++i) {
            double f = P->frag_mean + P->frag_sd * rng_normal(&r);
            uint64_t fl = f < (double)rl ? rl : (uint64_t)f;
            if (fl > L) fl = L;
            uint64_t at = rng_below(&r, L - fl + 1);
            if (emit_read(o, P, &r, g + at, rl, 0, th_sub, th_ins, th_del, th_n)) { free(g); return -1; }
            if (emit_read(o, P, &r, g + at + fl - rl, rl, 1, th_sub, th_ins, th_del, th_n)) { free(g); return -1; }
        }
    }
    free(g);
    return 0;
}
