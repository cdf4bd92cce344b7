"""Pins for the CPU oracle, independent of the oracle's own code.

Each test fixes the oracle to something other than itself: a brute force over
strings (canonical = lexicographic min of a k-mer and its reverse complement,
A<C<G<T), the hand-worked fixtures in tests/golden/, closed forms for the
window count, invariants of the counted result, and a brute-force window
minimum for the paper's deque (Sec. 3.2).
"""
import json
import os
from collections import Counter, defaultdict

import numpy as np
import pytest

import datagen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
COMP = {ord("A"): "T", ord("C"): "G", ord("G"): "C", ord("T"): "A"}


def revcomp(s: str) -> str:
    return s.translate(COMP)[::-1]


def canonical_str(s: str) -> str:
    r = revcomp(s)
    return s if s <= r else r


def to_int(s: str) -> int:
    """Base-4 number with A,C,G,T = digits 0..3 (lexicographic order = numeric order)."""
    return int(s.translate(str.maketrans("ACGT", "0123")), 4) if s else 0


def brute_force(read_strs, k):
    c = Counter()
    for s in read_strs:
        for i in range(len(s) - k + 1):
            w = s[i:i + k]
            if all(ch in "ACGT" for ch in w):
                c[canonical_str(w)] += 1
    return c


def pack(read_strs):
    offs = np.zeros(len(read_strs) + 1, np.uint64)
    offs[1:] = np.cumsum([len(s) for s in read_strs])
    reads = np.frombuffer("".join(read_strs).encode(), np.uint8) if read_strs else np.zeros(0, np.uint8)
    return reads.copy(), offs


def strs_of(reads, offsets):
    b = reads.tobytes()
    return [b[offsets[i]:offsets[i + 1]].decode() for i in range(offsets.size - 1)]


def key_int(res, i):
    if res.key_words == 1:
        return int(res.kmers[i])
    return int(res.kmers[i, 0]) | (int(res.kmers[i, 1]) << 64)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 8, 15, 16, 17, 31, 32, 33, 40, 63, 64])
@pytest.mark.parametrize("seed", [0, 1])
def test_oracle_matches_string_brute_force(k, seed):
    reads, offs = datagen.random_reads(seed * 100 + k, 150, 0, 90, p_invalid=0.02,
                                       alphabet=b"ACGT", invalid=b"NnRx")
    # a few low-complexity reads so counts above 1 occur at every k
    strs = strs_of(reads, offs) + ["A" * 80, "T" * 70, "AC" * 40, "GT" * 35]
    reads, offs = pack(strs)
    bf = brute_force(strs, k)
    res = oracle.count(reads, offs, k, 1, 1 << 31, hist_len=4096)
    got = {key_int(res, i): int(res.counts[i]) for i in range(len(res.counts))}
    want = {to_int(s): c for s, c in bf.items()}
    assert got == want
    assert res.n_windows == sum(bf.values())
    assert res.n_distinct == len(bf)
    assert res.max_count == (max(bf.values()) if bf else 0)
    keys = [key_int(res, i) for i in range(len(res.counts))]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)


def test_oracle_golden_hand_examples():
    cases = json.load(open(os.path.join(GOLDEN, "hand_example.json")))["cases"]
    for c in cases:
        reads, offs = pack(c["reads"])
        res = oracle.count(reads, offs, c["k"], c["lo"], c["hi"], hist_len=64)
        assert res.n_windows == c["n_windows"], c["name"]
        assert res.n_distinct == c["n_distinct"], c["name"]
        assert res.max_count == c["max_count"], c["name"]
        pairs = [[key_int(res, i), int(res.counts[i])] for i in range(len(res.counts))]
        assert pairs == c["pairs"], c["name"]
        nz = [[int(i), int(res.hist[i])] for i in np.nonzero(res.hist)[0]]
        assert nz == c["hist_nonzero"], c["name"]
        allc = oracle.count(reads, offs, c["k"], 1, 1 << 31, hist_len=64)
        assert [[key_int(allc, i), int(allc.counts[i])] for i in range(len(allc.counts))] == c["all_counts"]


def valid_segment_lengths(strs):
    for s in strs:
        run = 0
        for ch in s + "$":
            if ch in "ACGT":
                run += 1
            else:
                if run:
                    yield run
                run = 0


@pytest.mark.parametrize("k", [1, 7, 31, 55])
def test_window_count_closed_form(k):
    reads, offs = datagen.random_reads(7, 300, 0, 400, p_invalid=0.01)
    strs = strs_of(reads, offs)
    closed = sum(max(0, L - k + 1) for L in valid_segment_lengths(strs))
    res = oracle.count(reads, offs, k, 1, 1 << 31)
    assert res.n_windows == closed
    # sum over the histogram of count * (number of k-mers with that count) = N
    assert int((np.arange(res.hist.size, dtype=np.uint64) * res.hist).sum()) == closed


@pytest.fixture(scope="module")
def small_set():
    # 1/10 of the tiny workload's reads keeps these invariants fast
    rs = datagen.tiny()
    n = 2000
    return rs.reads[: int(rs.offsets[n])].copy(), rs.offsets[: n + 1].copy()


def _same(a, b):
    assert a.n_windows == b.n_windows
    assert a.n_distinct == b.n_distinct
    assert np.array_equal(a.kmers, b.kmers)
    assert np.array_equal(a.counts, b.counts)
    assert np.array_equal(a.hist, b.hist)


@pytest.mark.parametrize("k", [31, 55])
def test_invariant_reverse_complement_all_reads(small_set, k):
    reads, offs = small_set
    strs = strs_of(reads, offs)
    rc_reads, rc_offs = pack([revcomp(s) for s in strs])
    _same(oracle.count(reads, offs, k, 2, 1000), oracle.count(rc_reads, rc_offs, k, 2, 1000))


def test_invariant_read_permutation(small_set):
    reads, offs = small_set
    strs = strs_of(reads, offs)
    perm = np.random.default_rng(5).permutation(len(strs))
    p_reads, p_offs = pack([strs[i] for i in perm])
    _same(oracle.count(reads, offs, 31, 2, 1000), oracle.count(p_reads, p_offs, 31, 2, 1000))


def test_invariant_split_read_at_invalid_base():
    reads, offs = datagen.random_reads(11, 200, 50, 300, p_invalid=0.01)
    strs = strs_of(reads, offs)
    split = []
    for s in strs:
        split.extend(s.split("N"))
    s_reads, s_offs = pack(split)
    _same(oracle.count(reads, offs, 21, 1, 100), oracle.count(s_reads, s_offs, 21, 1, 100))


def test_histogram_last_bin_collects_large_counts():
    reads, offs = pack(["A" * 100])
    res = oracle.count(reads, offs, 5, 1, 1000, hist_len=8)
    assert res.max_count == 96
    assert int(res.hist[7]) == 1 and int(res.hist.sum()) == 1


def test_filter_bounds_are_inclusive(small_set):
    reads, offs = small_set
    full = oracle.count(reads, offs, 31, 1, 1 << 31)
    for lo, hi in [(2, 2), (2, 8), (3, 5), (1, 1)]:
        r = oracle.count(reads, offs, 31, lo, hi)
        sel = (full.counts >= lo) & (full.counts <= hi)
        assert np.array_equal(r.kmers, full.kmers[sel])
        assert np.array_equal(r.counts, full.counts[sel])
        assert len(r.counts) == int(full.hist[lo:hi + 1].sum())


def test_count_keys_agrees_with_count(small_set):
    reads, offs = small_set
    full = oracle.count(reads, offs, 31, 1, 1 << 31)
    idx = np.random.default_rng(3).choice(len(full.counts), 500, replace=False)
    idx.sort()
    got, nw = oracle.count_keys(reads, offs, 31, full.kmers[idx], n_threads=3)
    assert nw == full.n_windows
    assert np.array_equal(got, full.counts[idx].astype(np.uint64))


def test_sort_stage_is_library_sort():
    x = np.random.default_rng(0).integers(0, 2**63, 100_000, dtype=np.uint64)
    assert np.array_equal(oracle.sort_u64(x), np.sort(x))


# --- minimizer stage (Sec. 3.2) ------------------------------------------------

def test_score_function_is_the_murmur3_finalizer():
    """fmix64 is a bijection whose inverse uses the modular inverses of its two
    published multipliers; a wrong constant or shift breaks the round trip."""
    M = (1 << 64) - 1
    c1, c2 = 0xFF51AFD7ED558CCD, 0xC4CEB9FE1A85EC53
    i1, i2 = pow(c1, -1, 1 << 64), pow(c2, -1, 1 << 64)

    def unshift(h):  # inverse of h ^= h >> 33
        return h ^ (h >> 33)

    def inverse(h):
        h = unshift(h)
        h = (h * i2) & M
        h = unshift(h)
        h = (h * i1) & M
        return unshift(h)

    assert oracle.fmix64(0) == 0
    rng = np.random.default_rng(1)
    for x in [1, 2, 3, 12345, M] + [int(v) for v in rng.integers(0, 2**63, 200, dtype=np.uint64)]:
        assert inverse(oracle.fmix64(x)) == x


def test_score_finalizer_fmix32_is_the_murmur3_one():
    """fmix32 is a bijection whose inverse uses the modular inverses of its two
    published multipliers; a wrong constant or shift breaks the round trip."""
    M = (1 << 32) - 1
    i1, i2 = pow(0x85EBCA6B, -1, 1 << 32), pow(0xC2B2AE35, -1, 1 << 32)

    def inverse(h):
        h ^= h >> 16                      # undo h ^= h >> 16
        h = (h * i2) & M
        h ^= (h >> 13) ^ (h >> 26)        # undo h ^= h >> 13
        h = (h * i1) & M
        return h ^ (h >> 16)

    assert oracle.fmix32(0) == 0
    rng = np.random.default_rng(2)
    for x in [1, 2, 3, 0xDEADBEEF, M] + [int(v) for v in rng.integers(0, 2**32, 200, dtype=np.uint64)]:
        assert inverse(oracle.fmix32(x)) == x


def score(mmer: str, seed: int) -> int:
    """m-mer score written from its definition: fmix32 of the canonical code
    folded to 32 bits, XOR the seed's low 32 bits."""
    c = to_int(canonical_str(mmer))
    return oracle.fmix32(((c & 0xFFFFFFFF) ^ (c >> 32) ^ seed) & 0xFFFFFFFF)


@pytest.mark.parametrize("k,m", [(5, 2), (9, 4), (21, 11), (31, 17), (31, 31), (40, 1), (55, 21), (64, 32)])
def test_deque_minimizer_matches_window_minimum(k, m):
    reads, offs = datagen.random_reads(k * 7 + m, 60, 0, 150, p_invalid=0.01)
    strs = strs_of(reads, offs)
    seed = oracle.DEFAULT_SEED
    pos, key, mh, mp = oracle.windows(reads, offs, k, m, seed)
    want = []
    for r, s in enumerate(strs):
        for i in range(len(s) - k + 1):
            w = s[i:i + k]
            if not all(ch in "ACGT" for ch in w):
                continue
            scores = [score(w[j:j + m], seed) for j in range(k - m + 1)]
            best = min(scores)
            last = max(j for j in range(len(scores)) if scores[j] == best)  # right-most tie
            want.append((int(offs[r]) + i, to_int(canonical_str(w)), best, int(offs[r]) + i + last))
    got = [(int(pos[i]), int(key[i, 0]) | (int(key[i, 1]) << 64), int(mh[i]), int(mp[i]))
           for i in range(len(pos))]
    assert got == want


def test_minimizer_is_a_function_of_the_canonical_kmer():
    """Canonical m-mers make a k-mer and its reverse complement share their
    minimizer score, so every occurrence lands in the same task (Sec. 3.4)."""
    rs = datagen.tiny()
    n = 800
    reads, offs = rs.reads[: int(rs.offsets[n])], rs.offsets[: n + 1]
    strs = strs_of(reads, offs)
    rc_reads, rc_offs = pack([revcomp(s) for s in strs])
    both = np.concatenate([reads, rc_reads])
    boffs = np.concatenate([offs, rc_offs[1:] + offs[-1]])
    _, key, mh, _ = oracle.windows(both, boffs, 31, 17)
    seen = {}
    for i in range(len(mh)):
        kk = int(key[i, 0])
        assert seen.setdefault(kk, int(mh[i])) == int(mh[i])


@pytest.mark.parametrize("n_buckets", [1, 3, 64, 4096])
def test_supermers_against_brute_force_runs(n_buckets):
    reads, offs = datagen.random_reads(17, 80, 0, 200, p_invalid=0.01)
    k, m = 21, 11
    pos, key, mh, _ = oracle.windows(reads, offs, k, m)
    bucket = [int(h) % n_buckets for h in mh]
    read_of = np.searchsorted(offs, pos, side="right") - 1
    want = []
    i = 0
    while i < len(pos):
        j = i + 1
        while j < len(pos) and pos[j] == pos[j - 1] + 1 and read_of[j] == read_of[i] and bucket[j] == bucket[i]:
            j += 1
        want.append((int(pos[i]), j - i, bucket[i]))
        i = j
    sp, sn, sb, bk = oracle.supermers(reads, offs, k, m, n_buckets)
    assert list(zip(sp.tolist(), sn.tolist(), sb.tolist())) == want
    per = defaultdict(int)
    for b in bucket:
        per[b] += 1
    assert bk.tolist() == [per[b] for b in range(n_buckets)]
    assert int(sn.sum()) == len(pos)


# --- encoding stage (Sec. 2.2) and the window count ----------------------------

def test_encode_matches_the_byte_table():
    """Every one of the 256 byte values against the hand-written table in
    tests/golden/encode_table.json: a swapped code or a wrong invalid flag on
    any byte (lower case, N, IUPAC, high bytes) fails here."""
    rows = json.load(open(os.path.join(GOLDEN, "encode_table.json")))["rows"]
    assert [r[0] for r in rows] == list(range(256))
    all_bytes = np.arange(256, dtype=np.uint8)
    code, inv = oracle.encode(all_bytes)
    assert code.tolist() == [r[1] for r in rows]
    assert inv.tolist() == [r[2] for r in rows]
    # the same bytes in another order and repeated: the code is per byte, position-free
    perm = np.random.default_rng(4).permutation(np.tile(all_bytes, 3))
    code2, inv2 = oracle.encode(perm)
    assert code2.tolist() == [rows[b][1] for b in perm.tolist()]
    assert inv2.tolist() == [rows[b][2] for b in perm.tolist()]
    # exactly four valid bytes, with four distinct codes
    assert sorted(r[1] for r in rows if r[2] == 0) == [0, 1, 2, 3]


@pytest.mark.parametrize("k", [1, 2, 7, 31, 32, 33, 55, 64])
def test_n_windows_matches_closed_form(k):
    """oracle.n_windows (the full-size window-count checker) against the closed
    form: the sum over maximal stretches of upper-case ACGT bytes, within each
    read, of max(0, L - k + 1)."""
    reads, offs = datagen.random_reads(31 + k, 400, 0, 300, p_invalid=0.01, invalid=b"NnRx\x00\xff")
    extra = [b"", b"A" * (k - 1), b"A" * k, b"C" * (k + 5) + b"N" + b"G" * k]
    blobs = [reads[int(offs[i]):int(offs[i + 1])].tobytes() for i in range(offs.size - 1)] + extra

    def closed_form(bs):
        total = 0
        for b in bs:
            run = 0
            for ch in b + b"$":
                if ch in b"ACGT":
                    run += 1
                else:
                    total += max(0, run - k + 1)
                    run = 0
        return total

    r = np.frombuffer(b"".join(blobs), np.uint8).copy()
    o = np.zeros(len(blobs) + 1, np.uint64)
    o[1:] = np.cumsum([len(b) for b in blobs])
    assert oracle.n_windows(r, o, k) == closed_form(blobs)
    # windows never cross a read boundary: one read holding all bytes has more
    one = np.array([0, r.size], np.uint64)
    assert oracle.n_windows(r, one, k) == closed_form([b"".join(blobs)])


# --- extension information (Sec. 3.3.2) -----------------------------------------

def test_count_ext_golden_hand_examples():
    cases = json.load(open(os.path.join(GOLDEN, "ext_example.json")))["cases"]
    for c in cases:
        reads, offs = pack(c["reads"])
        r = oracle.count_ext(reads, offs, c["k"], c["lo"], c["hi"])
        assert r.kmers.tolist() == c["kmers"], c["name"]
        assert r.counts.tolist() == c["counts"], c["name"]
        occ = [[[int(r.occ_read[j]), int(r.occ_pos[j])] for j in range(int(r.occ_offsets[i]), int(r.occ_offsets[i + 1]))]
               for i in range(len(r.counts))]
        assert occ == c["occurrences"], c["name"]


@pytest.mark.parametrize("k", [3, 8, 21, 31, 33, 64])
def test_count_ext_matches_string_brute_force(k):
    reads, offs = datagen.random_reads(500 + k, 120, 0, 90, p_invalid=0.02, invalid=b"Nn")
    strs = strs_of(reads, offs) + ["AC" * 40, "A" * 70, "AC" * 40]
    reads, offs = pack(strs)
    where = defaultdict(list)
    for ri, s in enumerate(strs):
        for i in range(len(s) - k + 1):
            w = s[i:i + k]
            if all(ch in "ACGT" for ch in w):
                where[to_int(canonical_str(w))].append((ri, i))
    lo, hi = 2, 50
    want = sorted((key, occ) for key, occ in where.items() if lo <= len(occ) <= hi)
    r = oracle.count_ext(reads, offs, k, lo, hi)
    got = []
    for i in range(len(r.counts)):
        key = key_int(r, i)
        occ = [(int(r.occ_read[j]), int(r.occ_pos[j])) for j in range(int(r.occ_offsets[i]), int(r.occ_offsets[i + 1]))]
        assert len(occ) == int(r.counts[i])
        got.append((key, occ))
    assert got == want
    # the same kept k-mers and counts as the plain count
    plain = oracle.count(reads, offs, k, lo, hi)
    assert np.array_equal(plain.kmers, r.kmers) and np.array_equal(plain.counts, r.counts)
