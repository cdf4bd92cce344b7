// hsk_pack.h -- the packed path of the batched and served forms (host side,
// not part of the public ABI): many read sets with the same k, m and filter
// counted by one pass of the pipeline (hsk_pack.cu).
#pragma once

#include <cstdint>
#include <string>

#include "hsk_runtime.h"

// A set's code after a pass that could not finish it (it is then counted alone).
#define HSK_PACK_REDO 1
// Buckets one set may take in a pack (sets are small; the pack's total stays
// within HSK_MAX_BUCKETS, the S2 walk's per-CTA bucket table).
#define HSK_PACK_MAX_SET_BUCKETS 4096

struct PackSet {
    const char* reads = nullptr;       // host bases (borrowed)
    const uint64_t* offsets = nullptr; // host offsets, n_reads + 1 entries
    uint64_t n_reads = 0;
    HostResult* out = nullptr;         // where the result goes
    int rc = 0;                        // HSK_OK or the set's error
    int alone = 0;                     // 1 when it was counted alone after the pass
    std::string err;                   // error text when rc != HSK_OK
};

// Buckets of a set of n_bases bases in a pack, and keys per bucket group.
uint32_t hsk_pack_set_buckets(uint64_t n_bases, int key_words, uint64_t group_keys);
uint64_t hsk_pack_group_keys(hsk_ctx* c, int key_words);

// Count the sets (all with k, m, lo, hi) by one pass on stream st; each set's
// rc and out are filled.  Sets the pass could not finish are counted alone.
// Returns HSK_OK unless the context itself failed.
// *fail_msg (may be NULL) receives the reason when the pass as a whole failed.
int hsk_count_pack_host(hsk_ctx* c, PackSet* sets, uint32_t n_sets, int k, int m, uint32_t lo, uint32_t hi,
                        cudaStream_t st, std::string* fail_msg = nullptr);
