// hsk_ext.cu -- C ABI of the extension information (Sec. 3.3.2): counting
// with each kept k-mer's occurrence list, and the paper's compact encoding of
// extension information (device kernels in k_ext.cu).
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/hsk.h"
#include "../../include/hsk_stages.h"
#include "hsk_internal.h"
#include "hsk_runtime.h"

using namespace hsk;

extern "C" int hsk_count_ext(hsk_ctx* c, const char* reads, const uint64_t* offsets, uint64_t n_reads, int k,
                             int m, uint32_t lo, uint32_t hi, hsk_ext_result* out) {
    return hsk_guarded(c, [&]() -> int {
        if (!c || !out) return HSK_EINVAL;
        if (n_reads >= 0xFFFFFFFFull) {
            hsk_set_error(c, "%llu reads: read indices are 32-bit", (unsigned long long)n_reads);
            return HSK_EOVERFLOW;
        }
        for (uint64_t i = 0; offsets && i < n_reads; ++i)
            if (offsets[i + 1] >= offsets[i] && offsets[i + 1] - offsets[i] > 0xFFFFFFFFull) {
                hsk_set_error(c, "read %llu is longer than 2^32 bases", (unsigned long long)i);
                return HSK_EOVERFLOW;
            }
        hsk_result plain;
        TRY(hsk_count(c, reads, offsets, n_reads, k, m, lo, hi, &plain));
        cudaStream_t st = c->stream;
        c->zst = st;
        const int kw = k <= 32 ? 1 : 2;
        const uint64_t np = plain.n_pairs;
        const uint64_t n_bases = n_reads ? offsets[n_reads] : 0;
        c->ext_off.pinned = c->ext_read.pinned = c->ext_pos.pinned = true;
        c->ext_off.resize(np + 1);
        uint64_t n_occ = 0;
        if (np == 0) {
            c->ext_off.data()[0] = 0;
            c->ext_read.resize(0);
            c->ext_pos.resize(0);
        } else {
            // the kept keys (sorted, on the device since the count) into a table of indices
            uint32_t slots = 1024;
            while (slots < 2 * np) slots <<= 1;
            // composites: (index << 40) | start, 64-bit while the index fits 24 bits
            int ib = 0;
            while ((1ull << ib) < np) ++ib;
            const bool wide = ib > 24;
            const int comp_bits = 40 + std::max(ib, 1);
            const size_t cb = wide ? 16 : 8;
            // occurrence offsets = exclusive scan of the kept counts
            TRY(hsk_ensure(c, c->ext_tab, (size_t)slots * 4 + (np + 1) * 8 + 64, false));
            uint32_t* table = (uint32_t*)c->ext_tab.p;
            uint64_t* occ_off = (uint64_t*)((char*)c->ext_tab.p + (size_t)slots * 4);
            CK(cudaMemsetAsync(table, 0, (size_t)slots * 4, st));
            CK(cudaMemsetAsync(c->small, 0, 64, st));
            launch_ext_insert(c->out_keys.p, kw, np, table, slots - 1, c->d_err, st);
            TRY(hsk_ensure_status(c, scan_status_words(np), st));
            uint32_t ep, *ctr;
            TRY(hsk_next_epoch(c, st, &ep));
            TRY(hsk_next_counter(c, st, &ctr));
            launch_scan_u32((const uint32_t*)c->out_counts.p, np, occ_off, (uint64_t*)c->lb_status.p, ctr, ep,
                            c->d_err, st);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(&n_occ, occ_off + np, 8, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            // every window looked up; kept occurrences as composites, then sorted
            TRY(hsk_ensure(c, c->batch_a, std::max<uint64_t>(n_occ, 1) * cb, false));
            TRY(hsk_ensure(c, c->ext_occ, std::max<uint64_t>(n_occ, 1) * 8, false));
            launch_ext_scan((const uint64_t*)c->pk.p, (const uint64_t*)c->iv.p, (const uint64_t*)c->rs.p, n_bases, k,
                            c->out_keys.p, table, slots - 1, wide, c->batch_a.p, n_occ, c->d_nout, c->d_err,
                            c->num_sms * 8, st);
            CK(cudaGetLastError());
            uint64_t emitted = 0;
            CK(cudaMemcpyAsync(&emitted, c->d_nout, 8, cudaMemcpyDeviceToHost, st));
            TRY(hsk_read_device_error(c, st));
            if (emitted != n_occ) {
                hsk_set_error(c, "extension scan found %llu occurrences of kept k-mers, counts say %llu",
                              (unsigned long long)emitted, (unsigned long long)n_occ);
                return HSK_ECUDA;
            }
            TRY(hsk_plain_sort(c, c->batch_a.p, nullptr, n_occ, wide ? 2 : 1, comp_bits, c->batch_b, nullptr, st));
            uint32_t* occ_read = (uint32_t*)c->ext_occ.p;
            uint32_t* occ_pos = occ_read + n_occ;
            launch_ext_decode_pos(c->batch_a.p, wide, n_occ, (const uint64_t*)c->in_offsets.p, n_reads, occ_read,
                                  occ_pos, c->num_sms * 8, st);
            CK(cudaGetLastError());
            c->ext_read.resize(n_occ);
            c->ext_pos.resize(n_occ);
            CK(cudaMemcpyAsync(c->ext_off.data(), occ_off, (np + 1) * 8, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(c->ext_read.data(), occ_read, n_occ * 4, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(c->ext_pos.data(), occ_pos, n_occ * 4, cudaMemcpyDeviceToHost, st));
            TRY(hsk_read_device_error(c, st));
        }
        memset(out, 0, sizeof(*out));
        out->counts = plain;
        out->n_occ = n_occ;
        out->occ_offsets = c->ext_off.data();
        out->occ_read = c->ext_read.data();
        out->occ_pos = c->ext_pos.data();
        return HSK_OK;
    });
}

extern "C" int hsk_stage_ext_encode(hsk_ctx* c, const uint32_t* d_read, const uint32_t* d_pos, uint64_t n,
                                    uint8_t* d_out, uint64_t out_cap, uint64_t* d_chunk_off, uint64_t* n_bytes,
                                    void* stream) {
    return hsk_guarded(c, [&]() -> int {
        if (!c || !n_bytes || (n && (!d_read || !d_pos || !d_out || !d_chunk_off))) return HSK_EINVAL;
        if (out_cap < 9 * n) {
            hsk_set_error(c, "the encoded stream may need 9 bytes per item");
            return HSK_EINVAL;
        }
        CK(cudaSetDevice(c->cfg.device));
        cudaStream_t st = (cudaStream_t)stream;
        c->zst = st;
        *n_bytes = 0;
        if (n == 0) return HSK_OK;
        CK(cudaMemsetAsync(c->small, 0, 64, st));
        TRY(hsk_ensure(c, c->batch_c, n * 4 + 16, false));
        TRY(hsk_ensure(c, c->batch_d, (n + 1) * 8 + 16, false));
        uint32_t* size = (uint32_t*)c->batch_c.p;
        uint64_t* off = (uint64_t*)c->batch_d.p;
        launch_ext_sizes(d_read, d_pos, n, size, c->num_sms * 8, st);
        TRY(hsk_ensure_status(c, scan_status_words(n), st));
        uint32_t ep, *ctr;
        TRY(hsk_next_epoch(c, st, &ep));
        TRY(hsk_next_counter(c, st, &ctr));
        launch_scan_u32(size, n, off, (uint64_t*)c->lb_status.p, ctr, ep, c->d_err, st);
        launch_ext_encode(d_read, d_pos, n, off, d_out, c->num_sms * 8, st);
        launch_ext_chunk_off(off, n, d_chunk_off, c->num_sms * 8, st);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(n_bytes, off + n, 8, cudaMemcpyDeviceToHost, st));
        return hsk_read_device_error(c, st);
    });
}

extern "C" int hsk_stage_ext_decode(hsk_ctx* c, const uint8_t* d_in, uint64_t n_bytes, const uint64_t* d_chunk_off,
                                    uint64_t n, uint32_t* d_read, uint32_t* d_pos, void* stream) {
    return hsk_guarded(c, [&]() -> int {
        if (!c || (n && (!d_in || !d_chunk_off || !d_read || !d_pos))) return HSK_EINVAL;
        CK(cudaSetDevice(c->cfg.device));
        cudaStream_t st = (cudaStream_t)stream;
        c->zst = st;
        CK(cudaMemsetAsync(c->small, 0, 64, st));
        launch_ext_decode(d_in, n_bytes, n, d_chunk_off, d_read, d_pos, c->d_err, c->num_sms * 8, st);
        CK(cudaGetLastError());
        const int rc = hsk_read_device_error(c, st);
        if (rc == HSK_ECUDA) hsk_set_error(c, "the encoded stream is malformed");
        return rc == HSK_ECUDA ? HSK_EINVAL : rc;
    });
}
