// hsk_pack.cu -- many read sets counted by one pass of the pipeline (the
// packed path of the batched and served forms).
//
// The paper runs many independent tasks on shared workers (Sec. 3.4).  Here
// the read sets of a pack share every launch of the pipeline:
//   * their bases lie one after the other in one device buffer, each set
//     starting on a warp-tile boundary of the S2 walk (the gap is padding with
//     an invalid byte, so no window reaches across it);
//   * each set owns a range of minimizer buckets, so no bucket, bucket group
//     or sub-segment ever holds k-mers of two sets;
//   * S1 encode, S2 walk, S3 scatter, the S4 partition and the S4/S5 on-chip
//     sort run once over the pack; the on-chip sort keeps each set's
//     histogram, distinct count and largest count apart;
//   * S6 sorts every set's kept pairs as one segment of a segmented LSD sort;
//   * the results are copied back set by set.
// A set is counted exactly as hsk_count counts it alone: windows never cross
// a read, buckets only partition the k-mers, and the output order is the
// global key order of the set.
//
// A set whose keys do not all fit the on-chip sort (a sub-segment that no
// on-chip tier nor the heavy-hitter lists take: repeat-rich input) is counted again alone through
// the plain path, which handles that case; the pack's partial result for it
// is dropped.
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/hsk.h"
#include "hsk_internal.h"
#include "hsk_pack.h"
#include "hsk_runtime.h"

using namespace hsk;

// Buckets of one set in a pack: about one bucket group per bucket (a group
// holds a third of 256 sub-segments' on-chip capacity), a power of two.
uint32_t hsk_pack_set_buckets(uint64_t n_bases, int key_words, uint64_t group_keys) {
    const uint64_t groups = (n_bases + group_keys - 1) / group_keys;
    uint32_t b = 1;
    while (b < groups && b < HSK_PACK_MAX_SET_BUCKETS) b <<= 1;
    (void)key_words;
    return b;
}

uint64_t hsk_pack_group_keys(hsk_ctx* c, int key_words) {
    const uint64_t cap = 256ull * local_cap(key_words);
    const uint32_t div = c->tune.group_div ? c->tune.group_div : 3;
    return cap / div;
}

static int check_set(hsk_ctx* c, const PackSet& s, uint64_t* n_bases) {
    *n_bases = 0;
    if (s.n_reads == 0) return HSK_OK;
    if (!s.offsets) {
        hsk_set_error(c, "NULL offsets with n_reads=%llu", (unsigned long long)s.n_reads);
        return HSK_EINVAL;
    }
    if (s.offsets[0] != 0) {
        hsk_set_error(c, "offsets[0] must be 0");
        return HSK_EINVAL;
    }
    for (uint64_t i = 0; i < s.n_reads; ++i)
        if (s.offsets[i + 1] < s.offsets[i]) {
            hsk_set_error(c, "offsets not monotone at read %llu", (unsigned long long)i);
            return HSK_EINVAL;
        }
    *n_bases = s.offsets[s.n_reads];
    if (*n_bases && !s.reads) {
        hsk_set_error(c, "NULL reads with bases present");
        return HSK_EINVAL;
    }
    if (*n_bases >= (1ull << 40)) {
        hsk_set_error(c, "n_bases %llu exceeds 2^40", (unsigned long long)*n_bases);
        return HSK_EOVERFLOW;
    }
    return HSK_OK;
}

// Result of a set with no window at all (no reads, or no bases).
static void empty_result(hsk_ctx* c, HostResult& HR, int kw) {
    const uint32_t H = c->cfg.hist_len;
    HR.kmers.resize(0);
    HR.counts.resize(0);
    HR.hist.resize(H);
    memset(HR.hist.data(), 0, (size_t)H * 8);
    memset(&HR.R, 0, sizeof(HR.R));
    HR.R.key_words = kw;
    HR.R.hist_len = H;
    HR.R.kmers = HR.kmers.data();
    HR.R.counts = HR.counts.data();
    HR.R.hist = HR.hist.data();
}

// Device arrays the pass keeps for the sets (one allocation): see the offsets
// computed in pack_pass.
struct PackTables {
    uint64_t* base;     // S + 1: first packed base of each set (last = all bases)
    uint64_t* off0;     // S: first offsets entry of each set
    uint64_t* nreads;   // S
    uint32_t* tile0;    // S + 1
    uint32_t* bucket;   // S
    uint32_t* bmask;    // S
};

static int pack_pass(hsk_ctx* c, std::vector<PackSet*>& sets, const std::vector<uint64_t>& nb, int k, int m,
                     uint32_t lo, uint32_t hi, cudaStream_t st) {
    const uint32_t S = (uint32_t)sets.size();
    const int kw = k <= 32 ? 1 : 2;
    const size_t kb = (size_t)kw * 8;
    const uint32_t H = c->cfg.hist_len;
    const uint64_t group_keys = hsk_pack_group_keys(c, kw);
    c->zst = st;

    // ---- layout of the pack (host)
    std::vector<uint64_t> base(S + 1), off0(S), nrd(S);
    std::vector<uint32_t> tile0(S + 1), bkt(S + 1), bmask(S);
    uint64_t nr_total = 0, max_reads = 0;
    base[0] = 0;
    bkt[0] = 0;
    for (uint32_t j = 0; j < S; ++j) {
        const uint64_t padded = (nb[j] + SM_TILE_BASES - 1) / SM_TILE_BASES * SM_TILE_BASES;
        base[j + 1] = base[j] + padded;
        off0[j] = nr_total;
        nrd[j] = sets[j]->n_reads;
        nr_total += sets[j]->n_reads + 1;
        max_reads = std::max(max_reads, sets[j]->n_reads);
        tile0[j] = (uint32_t)(base[j] / SM_TILE_BASES);
        const uint32_t B = hsk_pack_set_buckets(nb[j], kw, group_keys);
        bmask[j] = B - 1;
        bkt[j + 1] = bkt[j] + B;
    }
    tile0[S] = (uint32_t)(base[S] / SM_TILE_BASES);
    const uint64_t NB = base[S];
    const uint32_t B_total = bkt[S];
    if (B_total > HSK_MAX_BUCKETS || NB >= (1ull << 40)) {
        hsk_set_error(c, "pack of %u sets needs %u buckets / %llu bases", S, B_total, (unsigned long long)NB);
        return HSK_EINVAL;
    }

    CK(cudaEventRecord(c->ev0, st));
    CK(cudaMemsetAsync(c->small, 0, 64, st));
    CK(cudaMemsetAsync(c->counters, 0, HSK_N_COUNTERS * sizeof(uint32_t), st));
    c->ctr_used = 0;

    // ---- inputs and set tables to the device
    TRY(hsk_ensure(c, c->in_reads, NB + 64, false));
    TRY(hsk_ensure(c, c->in_offsets, nr_total * 8, false));
    const size_t tab_words = (S + 1) + S + S + ((3 * (size_t)S + 1 + 1) / 2 + 1);
    std::vector<uint64_t> tab(tab_words, 0);
    memcpy(tab.data(), base.data(), (S + 1) * 8);
    memcpy(tab.data() + S + 1, off0.data(), S * 8);
    memcpy(tab.data() + 2 * S + 1, nrd.data(), S * 8);
    uint32_t* t32 = reinterpret_cast<uint32_t*>(tab.data() + 3 * S + 1);
    memcpy(t32, tile0.data(), (S + 1) * 4);
    memcpy(t32 + S + 1, bkt.data(), S * 4);
    memcpy(t32 + 2 * S + 1, bmask.data(), S * 4);
    TRY(hsk_ensure(c, c->pack_tab, tab_words * 8, false));
    PackTables T;
    T.base = (uint64_t*)c->pack_tab.p;
    T.off0 = T.base + S + 1;
    T.nreads = T.off0 + S;
    T.tile0 = reinterpret_cast<uint32_t*>(T.nreads + S);
    T.bucket = T.tile0 + S + 1;
    T.bmask = T.bucket + S;
    char* d_reads = (char*)c->in_reads.p;
    uint64_t* d_offs = (uint64_t*)c->in_offsets.p;
    CK(cudaMemcpyAsync(c->pack_tab.p, tab.data(), tab_words * 8, cudaMemcpyHostToDevice, st));
    for (uint32_t j = 0; j < S; ++j) {
        if (nb[j]) CK(cudaMemcpyAsync(d_reads + base[j], sets[j]->reads, nb[j], cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_offs + off0[j], sets[j]->offsets, (sets[j]->n_reads + 1) * 8, cudaMemcpyHostToDevice,
                           st));
    }

    // ---- S1: read starts of every set (padding zeroed), then the encoding
    Encoded E;
    E.n_bases = NB;
    E.n_pw = (NB + 31) / 32;
    E.n_mw = (NB + 63) / 64;
    TRY(hsk_ensure(c, c->pk, (E.n_pw + 8) * 8, false));
    TRY(hsk_ensure(c, c->iv, (E.n_mw + 8) * 8, false));
    TRY(hsk_ensure(c, c->rs, (E.n_mw + 8) * 8, false));
    CK(cudaMemsetAsync((uint64_t*)c->pk.p + E.n_pw, 0, 8 * 8, st));
    CK(cudaMemsetAsync((uint64_t*)c->iv.p + E.n_mw, 0, 8 * 8, st));
    CK(cudaMemsetAsync(c->rs.p, 0, (E.n_mw + 8) * 8, st));
    launch_mark_starts_sets(d_offs, T.off0, T.nreads, T.base, S, max_reads, d_reads, (uint64_t*)c->rs.p, c->d_err,
                            st);
    launch_encode(d_reads, NB, (uint64_t*)c->pk.p, (uint64_t*)c->iv.p, E.n_pw, E.n_mw, st);
    CK(cudaGetLastError());
    E.packed = (const uint64_t*)c->pk.p;
    E.invalid = (const uint64_t*)c->iv.p;
    E.start = (const uint64_t*)c->rs.p;

    // ---- S2/S3: supermers into the sets' bucket ranges
    SetMap map;
    map.tile0 = T.tile0;
    map.bucket = T.bucket;
    map.bmask = T.bmask;
    map.n = S;
    Supermers SMR;
    TRY(hsk_supermers(c, E, k, m, B_total, SMR, st, nullptr, &map));

    // ---- bucket groups, set by set (a group never spans two sets)
    std::vector<uint64_t> set_kmers(S, 0), set_recs(S, 0);
    std::vector<uint32_t> cut, grp_set, grp0(S + 1);
    for (uint32_t j = 0; j < S; ++j) {
        for (uint32_t b = bkt[j]; b < bkt[j + 1]; ++b) set_kmers[j] += SMR.h_bucket_kmers[b];
        set_recs[j] = SMR.h_bucket_rec[bkt[j + 1]] - SMR.h_bucket_rec[bkt[j]];
        grp0[j] = (uint32_t)grp_set.size();
        if (set_kmers[j] == 0) continue;
        const uint32_t Bj = bkt[j + 1] - bkt[j];
        const uint32_t want = (uint32_t)std::min<uint64_t>(Bj, std::max<uint64_t>(1, set_kmers[j] / group_keys));
        std::vector<uint32_t> g = hsk_group_buckets(SMR, bkt[j], bkt[j + 1], want);
        for (size_t i = 0; i + 1 < g.size(); ++i) {
            cut.push_back(g[i]);
            grp_set.push_back(j);
        }
    }
    grp0[S] = (uint32_t)grp_set.size();
    cut.push_back(B_total);
    const uint32_t C = (uint32_t)grp_set.size();
    const uint64_t nk = SMR.n_kmers;
    std::vector<uint64_t> pair_off(S + 1, 0), distinct(S, 0);
    std::vector<uint32_t> maxc(S, 0);
    std::vector<char> redo(S, 0);

    // per-set statistics: histograms (S x H), distinct counts, largest counts
    TRY(hsk_ensure(c, c->hist, (size_t)S * H * 8, false));
    TRY(hsk_ensure(c, c->pack_stat, (size_t)S * 12 + 64, false));
    uint64_t* d_distinct = (uint64_t*)c->pack_stat.p;
    uint32_t* d_max = (uint32_t*)(d_distinct + S);
    CK(cudaMemsetAsync(c->hist.p, 0, (size_t)S * H * 8, st));
    CK(cudaMemsetAsync(c->pack_stat.p, 0, (size_t)S * 12, st));

    if (C > 0) {
        // the pack must fit the budget as one sort chunk
        std::vector<std::pair<uint32_t, uint32_t>> chunks;
        TRY(hsk_plan_chunks(c, SMR, kw, chunks));
        if (chunks.size() > 1) {
            hsk_set_error(c, "a pack of %llu k-mers does not fit one sort chunk", (unsigned long long)nk);
            return HSK_ENOMEM;
        }
        const uint64_t NS = (uint64_t)C * 256;
        const int key_bits = 2 * k;
        const int shift0 = key_bits > 8 ? key_bits - 8 : 0;
        std::vector<uint64_t> rbase(C + 1), tbase(C + 1);
        uint64_t nt = 0;
        for (uint32_t i = 0; i <= C; ++i) rbase[i] = SMR.h_bucket_rec[cut[i]];
        for (uint32_t i = 0; i < C; ++i) {
            tbase[i] = nt;
            nt += expand_tiles(rbase[i + 1] - rbase[i]);
        }
        tbase[C] = nt;
        if (nt >= 0xFFFFFFFFull) {
            hsk_set_error(c, "%llu record tiles in one pack", (unsigned long long)nt);
            return HSK_EOVERFLOW;
        }
        std::vector<uint32_t> tseg(nt + C);
        for (uint32_t i = 0; i < C; ++i)
            for (uint64_t t = tbase[i]; t < tbase[i + 1]; ++t) tseg[t] = i;
        memcpy(tseg.data() + nt, grp_set.data(), (size_t)C * 4);  // group -> set after the tile map
        TRY(hsk_ensure(c, c->keys, nk * kb, false));
        TRY(hsk_ensure(c, c->alt, nk * 4, false));
        const size_t t32b = (6 * NS * 4 + 7) & ~(size_t)7;
        TRY(hsk_ensure(c, c->loc_tab, t32b + (3 * NS + 2) * 8, false));
        uint32_t* sub_cnt = (uint32_t*)c->loc_tab.p;
        uint32_t* kcv = sub_cnt + NS;
        uint32_t* ov_list = kcv + NS;
        uint32_t* ov_list2 = ov_list + NS;
        uint32_t* ov_list3 = ov_list2 + NS;
        uint32_t* ov_list_m = ov_list3 + NS;
        uint64_t* sub_off = (uint64_t*)((char*)c->loc_tab.p + t32b);
        uint64_t* cursor = sub_off + NS + 1;
        uint64_t* kc_off = cursor + NS;
        TRY(hsk_ensure(c, c->batch_d, (nt + C) * 4 + 4, false));
        TRY(hsk_upload_segments(c, rbase, &tbase, st));
        CK(cudaMemcpyAsync(c->batch_d.p, tseg.data(), (nt + C) * 4, cudaMemcpyHostToDevice, st));
        const uint64_t* d_rbase = (const uint64_t*)c->seg.p;
        const uint64_t* d_tbase = d_rbase + (C + 1);
        const uint32_t* d_tseg = (const uint32_t*)c->batch_d.p;
        const uint32_t* d_grp_set = d_tseg + nt;
        // S4: keys counted and scattered into (group, top digit) sub-segments
        CK(cudaMemsetAsync(sub_cnt, 0, NS * 4, st));
        uint32_t *ctr, ep;
        TRY(hsk_next_counter(c, st, &ctr));
        launch_part(0, SMR.records, d_rbase, d_tbase, d_tseg, (uint32_t)nt, k, shift0, ctr, sub_cnt, nullptr, nullptr,
                    nullptr, c->d_err, expand_grid(c->num_sms), st);
        TRY(hsk_ensure_status(c, scan_status_words(NS), st));
        TRY(hsk_next_epoch(c, st, &ep));
        TRY(hsk_next_counter(c, st, &ctr));
        launch_scan_u32(sub_cnt, NS, sub_off, (uint64_t*)c->lb_status.p, ctr, ep, c->d_err, st);
        CK(cudaMemcpyAsync(cursor, sub_off, NS * 8, cudaMemcpyDeviceToDevice, st));
        TRY(hsk_next_counter(c, st, &ctr));
        launch_part(1, SMR.records, d_rbase, d_tbase, d_tseg, (uint32_t)nt, k, shift0, ctr, nullptr, cursor,
                    sub_off + 1, c->keys.p, c->d_err, expand_grid(c->num_sms), st);
        CK(cudaGetLastError());
        // S4/S5 on chip, statistics per set; the larger sub-segments take the
        // larger on-chip tiers and the heavy-hitter k-mer lists (as in the plain path)
        CK(cudaMemsetAsync(c->d_nlocal, 0, 72, st));
        TRY(hsk_next_counter(c, st, &ctr));
        launch_local_sort(sub_off, nullptr, (uint32_t)NS, 0, shift0, kw, c->keys.p, (uint32_t*)c->alt.p, kcv,
                          ov_list, c->d_ovstats, lo, hi, (uint64_t*)c->hist.p, H, d_max, d_distinct, d_grp_set, ctr,
                          c->d_err, c->num_sms, st);
        CK(cudaGetLastError());
        uint64_t st3[3] = {0, 0, 0};
        CK(cudaMemcpyAsync(st3, c->d_nlocal, sizeof(st3), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        uint32_t* left = nullptr;
        uint32_t n_ov = 0;
        uint64_t ov_keys = 0;
        TRY(hsk_local_overflow(c, sub_off, (uint32_t)(st3[1] & 0xFFFFFFFFull), ov_list, ov_list_m, ov_list2, ov_list3, kw,
                               shift0, c->keys.p, (uint32_t*)c->alt.p, kcv, lo, hi, (uint64_t*)c->hist.p, H, d_max,
                               d_distinct, d_grp_set, st, &left, &n_ov, &ov_keys));
        TRY(hsk_next_epoch(c, st, &ep));
        TRY(hsk_next_counter(c, st, &ctr));
        launch_scan_u32(kcv, NS, kc_off, (uint64_t*)c->lb_status.p, ctr, ep, c->d_err, st);
        // kept pairs per set: the scan at each set's first sub-segment
        std::vector<uint64_t> at(S + 1);
        for (uint32_t j = 0; j <= S; ++j) at[j] = (uint64_t)grp0[j] * 256;
        TRY(hsk_ensure(c, c->batch_c, (2 * (size_t)S + 2) * 8, false));
        uint64_t* d_at = (uint64_t*)c->batch_c.p;
        uint64_t* d_poff = d_at + S + 1;
        CK(cudaMemcpyAsync(d_at, at.data(), (S + 1) * 8, cudaMemcpyHostToDevice, st));
        launch_gather_u64(kc_off, d_at, S + 1, d_poff, st);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(pair_off.data(), d_poff, (S + 1) * 8, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (n_ov) {  // sets with a sub-segment the on-chip steps could not take: counted again alone
            std::vector<uint32_t> ovs(n_ov);
            CK(cudaMemcpyAsync(ovs.data(), left, (size_t)n_ov * 4, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            for (uint32_t s : ovs) redo[grp_set[s >> 8]] = 1;
        }
        // kept pairs of all sets, set after set, into the output buffers
        const uint64_t kept = pair_off[S];
        Output O;
        TRY(hsk_grow_output(c, O, std::max<uint64_t>(kept, 1), kw, st));
        launch_compact(sub_off, kcv, kc_off, (uint32_t)NS, 0, kw, c->keys.p, (const uint32_t*)c->alt.p, c->out_keys.p,
                       (uint32_t*)c->out_counts.p, kept, c->d_err, c->num_sms * 8, st);
        CK(cudaGetLastError());
    }

    // ---- S6: each set's pairs in key order (one segment per set)
    const uint64_t kept = pair_off[S];
    void* fin_keys = c->out_keys.p;
    uint32_t* fin_counts = (uint32_t*)c->out_counts.p;
    if (kept > 1) {
        const int key_bits = 2 * k;
        const int P = (key_bits + 7) / 8;
        const int cshift = 8 * P;
        const int spare = 64 * kw - cshift;
        const bool packed = spare > 0 && spare < 64 && (uint64_t)hi < (1ull << spare);
        const uint64_t TILE = onesweep_tile_keys(kw);
        std::vector<uint64_t> seg(S + 1 + (S + 2) / 2, 0);
        memcpy(seg.data(), pair_off.data(), (S + 1) * 8);
        uint32_t* ts = reinterpret_cast<uint32_t*>(seg.data() + S + 1);
        uint64_t tiles = 0;
        for (uint32_t j = 0; j < S; ++j) {
            ts[j] = (uint32_t)tiles;
            tiles += (pair_off[j + 1] - pair_off[j] + TILE - 1) / TILE;
        }
        ts[S] = (uint32_t)tiles;
        if (tiles >= 0xFFFFFFFFull) {
            hsk_set_error(c, "%llu sort tiles in one pack", (unsigned long long)tiles);
            return HSK_EOVERFLOW;
        }
        TRY(hsk_ensure(c, c->seg, seg.size() * 8, false));
        CK(cudaMemcpyAsync(c->seg.p, seg.data(), seg.size() * 8, cudaMemcpyHostToDevice, st));
        const uint64_t* d_kbase = (const uint64_t*)c->seg.p;
        const uint32_t* d_ts = reinterpret_cast<const uint32_t*>(d_kbase + S + 1);
        TRY(hsk_ensure(c, c->pass_hist, (size_t)S * P * 256 * 8, false));
        TRY(hsk_ensure(c, c->digit_off, (size_t)S * P * 256 * 8, false));
        TRY(hsk_ensure(c, c->pair_alt_keys, kept * kb, false));
        if (!packed) TRY(hsk_ensure(c, c->pair_alt_counts, kept * 4, false));
        TRY(hsk_ensure_status(c, tiles * 256 + 1, st));
        if (packed)
            launch_pack_pairs(c->out_keys.p, (uint32_t*)c->out_counts.p, kept, kw, cshift, false, c->num_sms * 8, st);
        CK(cudaMemsetAsync(c->pass_hist.p, 0, (size_t)S * P * 256 * 8, st));
        launch_digit_hist_seg(c->out_keys.p, kw, d_kbase, S, kept, (uint64_t*)c->pass_hist.p, P, st);
        launch_digit_offsets_seg((const uint64_t*)c->pass_hist.p, d_kbase, (uint64_t*)c->digit_off.p, P, S, st);
        void *src = c->out_keys.p, *dst = c->pair_alt_keys.p;
        uint32_t* vs = packed ? nullptr : (uint32_t*)c->out_counts.p;
        uint32_t* vd = packed ? nullptr : (uint32_t*)c->pair_alt_counts.p;
        for (int p = 0; p < P; ++p) {
            uint32_t ep, *ctr;
            TRY(hsk_next_epoch(c, st, &ep));
            TRY(hsk_next_counter(c, st, &ctr));
            launch_onesweep_seg(src, dst, vs, vd, d_kbase, S, (uint32_t)tiles, d_ts, kw, 8 * p,
                                (const uint64_t*)c->digit_off.p + (size_t)p * S * 256, (uint64_t*)c->lb_status.p,
                                ctr, ep, c->d_err, st);
            std::swap(src, dst);
            std::swap(vs, vd);
        }
        CK(cudaGetLastError());
        fin_keys = src;
        if (packed) launch_pack_pairs(fin_keys, (uint32_t*)c->out_counts.p, kept, kw, cshift, true, c->num_sms * 8, st);
        else fin_counts = vs;
    }
    CK(cudaEventRecord(c->ev1, st));
    // device statistics of the sets
    if (C > 0) {
        CK(cudaMemcpyAsync(distinct.data(), d_distinct, (size_t)S * 8, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(maxc.data(), d_max, (size_t)S * 4, cudaMemcpyDeviceToHost, st));
    }
    TRY(hsk_read_device_error(c, st));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));

    // ---- results, set by set
    for (uint32_t j = 0; j < S; ++j) {
        if (redo[j]) continue;
        HostResult& HR = *sets[j]->out;
        const uint64_t n = pair_off[j + 1] - pair_off[j];
        HR.kmers.resize(n * kw);
        HR.counts.resize(n);
        HR.hist.resize(H);
        if (n) {
            CK(cudaMemcpyAsync(HR.kmers.data(), (const char*)fin_keys + pair_off[j] * kb, n * kb,
                               cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(HR.counts.data(), fin_counts + pair_off[j], n * 4, cudaMemcpyDeviceToHost, st));
        }
        CK(cudaMemcpyAsync(HR.hist.data(), (const uint64_t*)c->hist.p + (size_t)j * H, (size_t)H * 8,
                           cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    for (uint32_t j = 0; j < S; ++j) {
        if (redo[j]) continue;
        HostResult& HR = *sets[j]->out;
        DevResult& R = HR.R;
        memset(&R, 0, sizeof(R));
        R.n_pairs = pair_off[j + 1] - pair_off[j];
        R.key_words = kw;
        R.hist_len = H;
        R.n_windows = set_kmers[j];
        R.n_distinct = distinct[j];
        R.max_count = maxc[j];
        R.n_chunks = 1;
        R.n_supermers = set_recs[j];
        R.device_ms = ms;
        R.kmers = HR.kmers.data();
        R.counts = HR.counts.data();
        R.hist = HR.hist.data();
        sets[j]->rc = HSK_OK;
    }
    for (uint32_t j = 0; j < S; ++j)
        if (redo[j]) sets[j]->rc = HSK_PACK_REDO;
    return HSK_OK;
}

int hsk_count_pack_host(hsk_ctx* c, PackSet* sets, uint32_t n_sets, int k, int m, uint32_t lo, uint32_t hi,
                        cudaStream_t st, std::string* fail_msg) {
    const int kw = k <= 32 ? 1 : 2;
    std::vector<PackSet*> run;
    std::vector<uint64_t> nb;
    for (uint32_t i = 0; i < n_sets; ++i) {
        uint64_t b = 0;
        sets[i].rc = check_set(c, sets[i], &b);
        if (sets[i].rc != HSK_OK) {
            sets[i].err = c->err_msg;
            continue;
        }
        if (b == 0) {
            empty_result(c, *sets[i].out, kw);
            continue;
        }
        run.push_back(&sets[i]);
        nb.push_back(b);
    }
    if (run.empty()) return HSK_OK;
    int rc = pack_pass(c, run, nb, k, m, lo, hi, st);
    if (rc != HSK_OK) {
        // the pass failed as a whole: every set that took part is counted alone
        // (that also tells which set, if any, holds the fault)
        if (fail_msg) *fail_msg = c->err_msg;
        for (PackSet* s : run) s->rc = HSK_PACK_REDO;
        cudaStreamSynchronize(st);
    }
    for (PackSet* s : run) {
        if (s->rc != HSK_PACK_REDO) continue;
        s->rc = hsk_count_host_on(c, s->reads, s->offsets, s->n_reads, k, m, lo, hi, st, c->in_reads, c->in_offsets,
                                  *s->out);
        if (s->rc != HSK_OK) s->err = c->err_msg;
        else s->alone = 1;
    }
    return HSK_OK;
}
