"""End-to-end parity of hsk_count / hsk_count_device with the CPU oracle:
bit-exact (k-mer, count) pairs, histogram, window / distinct / max counts."""
import numpy as np
import pytest

import datagen
import oracle
from gpu_util import assert_same_result, dev, dev_u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    return datagen.tiny()


def test_tiny_workload_bit_exact(hsk, tiny):
    """1 Mbp genome, 20,000 x 150 bp reads, k=31, m=17, filter [2, 1000]."""
    want = oracle.count(tiny.reads, tiny.offsets, tiny.k, tiny.lo, tiny.hi)
    with hsk.Context() as ctx:
        got = ctx.count(tiny.reads, tiny.offsets, tiny.k, tiny.m, tiny.lo, tiny.hi)
        assert_same_result(got, want, "tiny")
        assert got.n_windows == 20_000 * 120
        # device-pointer entry point gives the same bytes
        r = ctx.count_device(dev(tiny.reads), dev_u64(tiny.offsets), tiny.k, tiny.m, tiny.lo, tiny.hi)
        assert_same_result(ctx.result_to_host(r), want, "tiny-device")


@pytest.mark.parametrize("k,m", [(1, 1), (2, 1), (11, 6), (16, 8), (21, 11), (31, 17), (32, 16), (33, 17),
                                 (47, 23), (55, 21), (63, 31), (64, 32), (64, 1)])
def test_k_range_with_invalid_bases(hsk, k, m):
    reads, offs = datagen.random_reads(k * 31 + m, 400, 0, 600, p_invalid=0.005, invalid=b"NnRY.")
    # low-complexity reads so many k-mers repeat at every k
    extra = ["ACGT" * 50, "AAAAAAAAAA" * 20, "GATTACA" * 30, "T" * 65, "CG" * 40]
    strs = [reads[offs[i]:offs[i + 1]].tobytes().decode() for i in range(len(offs) - 1)] + extra
    o = np.zeros(len(strs) + 1, np.uint64)
    o[1:] = np.cumsum([len(s) for s in strs])
    r = np.frombuffer("".join(strs).encode(), np.uint8).copy()
    want = oracle.count(r, o, k, 1, 1 << 31, hist_len=256)
    with hsk.Context(hist_len=256) as ctx:
        got = ctx.count(r, o, k, m, 1, 1 << 31)
    assert_same_result(got, want, f"k={k} m={m}")


@pytest.mark.parametrize("n_buckets", [1, 2, 256, 8192])
def test_result_independent_of_bucket_count(hsk, tiny, n_buckets):
    n = 5000
    reads, offs = tiny.reads[: int(tiny.offsets[n])], tiny.offsets[: n + 1]
    want = oracle.count(reads, offs, 31, 2, 1000)
    with hsk.Context(n_buckets=n_buckets) as ctx:
        assert_same_result(ctx.count(reads, offs, 31, 17, 2, 1000), want, f"B={n_buckets}")


@pytest.mark.parametrize("m", [1, 9, 16, 31])
def test_result_independent_of_m(hsk, tiny, m):
    n = 3000
    reads, offs = tiny.reads[: int(tiny.offsets[n])], tiny.offsets[: n + 1]
    want = oracle.count(reads, offs, 31, 1, 10)
    with hsk.Context() as ctx:
        assert_same_result(ctx.count(reads, offs, 31, m, 1, 10), want, f"m={m}")


@pytest.mark.parametrize("k", [31, 55])
def test_chunked_sort_and_output_order(hsk, tiny, k):
    """Force many sort chunks (S6 then orders the pairs of all chunks)."""
    n = 6000
    reads, offs = tiny.reads[: int(tiny.offsets[n])], tiny.offsets[: n + 1]
    want = oracle.count(reads, offs, k, 1, 5)
    with hsk.Context(n_buckets=512, max_chunk_kmers=40_000) as ctx:
        got = ctx.count(reads, offs, k, 17, 1, 5)
    assert got.n_chunks > 5
    assert_same_result(got, want, "chunked")


def test_edge_cases(hsk):
    with hsk.Context(hist_len=16) as ctx:
        # empty input
        r = ctx.count(np.zeros(0, np.uint8), np.zeros(1, np.uint64), 31, 17, 2, 10)
        assert r.n_windows == 0 and r.kmers.size == 0 and not r.hist.any()
        # only empty reads
        r = ctx.count(np.zeros(0, np.uint8), np.zeros(5, np.uint64), 31, 17, 2, 10)
        assert r.n_windows == 0
        # reads shorter than k, all invalid, and one exact-length read
        strs = ["ACGT", "NNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNN", "A" * 31, "acgtacgtacgtacgtacgtacgtacgtacgt"]
        o = np.zeros(len(strs) + 1, np.uint64)
        o[1:] = np.cumsum([len(s) for s in strs])
        b = np.frombuffer("".join(strs).encode(), np.uint8).copy()
        r = ctx.count(b, o, 31, 17, 1, 10)
        assert r.n_windows == 1 and r.kmers.tolist() == [0] and r.counts.tolist() == [1]
        # histogram last bin collects counts >= hist_len - 1
        s = "A" * 200
        r = ctx.count(np.frombuffer(s.encode(), np.uint8).copy(), np.array([0, 200], np.uint64), 5, 3, 1, 1000)
        assert r.max_count == 196 and int(r.hist[15]) == 1 and int(r.hist.sum()) == 1


def test_argument_errors(hsk, tiny):
    with pytest.raises(hsk.HskError):
        hsk.Context(n_buckets=3)  # buckets must be a power of two
    n = 10
    reads, offs = tiny.reads[: int(tiny.offsets[n])], tiny.offsets[: n + 1]
    with hsk.Context() as ctx:
        for k, m, lo, hi in [(0, 1, 1, 2), (65, 17, 1, 2), (31, 0, 1, 2), (31, 32, 1, 2), (20, 21, 1, 2),
                             (31, 17, 5, 4)]:
            with pytest.raises(hsk.HskError) as e:
                ctx.count(reads, offs, k, m, lo, hi)
            assert e.value.code == hsk.HSK_EINVAL
        bad = offs.copy()
        bad[3], bad[4] = bad[4], bad[3]
        with pytest.raises(hsk.HskError) as e:
            ctx.count(reads, bad, 31, 17, 2, 8)
        assert e.value.code == hsk.HSK_EINVAL
        # device-side offset check: last offset must equal n_bases
        with pytest.raises(hsk.HskError) as e:
            ctx.count_device(dev(reads), dev_u64(offs), 31, 17, 2, 8, n_bases=int(offs[-1]) + 5)
        assert e.value.code == hsk.HSK_EINVAL
        # the context still works afterwards
        assert_same_result(ctx.count(reads, offs, 31, 17, 1, 9), oracle.count(reads, offs, 31, 1, 9))


def test_budget_and_injected_allocation_failure(hsk, tiny):
    n = 2000
    reads, offs = tiny.reads[: int(tiny.offsets[n])], tiny.offsets[: n + 1]
    want = oracle.count(reads, offs, 31, 2, 100)
    with hsk.Context(hbm_budget=8 << 20) as ctx:
        with pytest.raises(hsk.HskError) as e:
            ctx.count(reads, offs, 31, 17, 2, 100)
        assert e.value.code == hsk.HSK_ENOMEM
    for i in range(8):  # the i-th device allocation of a fresh context fails
        with hsk.Context() as ctx:
            ctx.fail_alloc_after(i)
            with pytest.raises(hsk.HskError) as e:
                ctx.count(reads, offs, 31, 17, 2, 100)
            assert e.value.code == hsk.HSK_ENOMEM
            ctx.fail_alloc_after(-1)
            assert_same_result(ctx.count(reads, offs, 31, 17, 2, 100), want, f"after failure {i}")


def test_repeated_calls_reuse_the_arena(hsk, tiny):
    """The same context gives identical bytes call after call (look-back epochs,
    tile counters and buffers are reused)."""
    n = 4000
    reads, offs = tiny.reads[: int(tiny.offsets[n])], tiny.offsets[: n + 1]
    want = oracle.count(reads, offs, 31, 2, 50)
    with hsk.Context() as ctx:
        for i in range(25):
            assert_same_result(ctx.count(reads, offs, 31, 17, 2, 50), want, f"call {i}")


@pytest.mark.parametrize("case", ["tiny", "one_bucket", "k55", "repeats", "small_hist"])
def test_on_chip_and_global_paths_agree(hsk, tiny, case):
    """The on-chip sub-segment sort and the global radix passes give the same
    bytes; one bucket forces sub-segments over the on-chip sort's capacity,
    which the heavy-hitter path then counts on chip as k-mer lists."""
    kw = dict(hist_len=65536)
    k, m, lo, hi = 31, 17, 2, 1000
    if case == "tiny":
        reads, offs = tiny.reads, tiny.offsets
    elif case == "one_bucket":
        # 2.4 M keys in one bucket: 256 sub-segments of ~9 K keys, past the
        # first pass's capacity: heavy-hitter tasks
        reads, offs = tiny.reads, tiny.offsets
        kw["n_buckets"] = 1
    elif case == "k55":
        rs = datagen.batched_set(datagen.derive_seed(5, 1), 300_000, 20.0)
        reads, offs, k, m, lo, hi = rs.reads, rs.offsets, 55, 21, 2, 500
    elif case == "repeats":
        # a few sequences repeated thousands of times next to random reads
        r, o = datagen.random_reads(31, 2000, 50, 300)
        rep = np.frombuffer(b"ACGTTGCAAGGCTTAACCGGATCGATTACGGCATCAGGACTTGACA" * 3, np.uint8)
        parts = [r] + [rep] * 3000
        reads = np.concatenate(parts)
        lens = np.concatenate([np.diff(o.astype(np.int64)), np.full(3000, rep.size)])
        offs = np.zeros(lens.size + 1, np.uint64)
        offs[1:] = np.cumsum(lens)
        lo, hi = 1, 100000
    else:
        n = 4000
        reads, offs = tiny.reads[: int(tiny.offsets[n])], tiny.offsets[: n + 1]
        kw["hist_len"] = 7
        lo, hi = 1, 3
    want = oracle.count(reads, offs, k, lo, hi, hist_len=kw["hist_len"])
    with hsk.Context(local_sort=True, **kw) as a, hsk.Context(local_sort=False, **kw) as b:
        ga = a.count(reads, offs, k, m, lo, hi)
        gb = b.count(reads, offs, k, m, lo, hi)
        if case == "one_bucket":
            assert a.last_overflow() == 0  # every heavy task was counted on chip
    assert_same_result(ga, want, f"{case} on-chip")
    assert_same_result(gb, want, f"{case} global")


def test_host_input_in_chunks_matches_device_input(hsk):
    """Inputs of 64 MB or more reach the device in chunks while S1/S2 run on
    the chunks already there; the result is the same as from device input."""
    import torch
    rs = datagen.long_read(scale=0.1)  # 150 Mbp
    assert rs.n_bases >= (64 << 20)
    with hsk.Context() as ctx:
        got = ctx.count(rs.reads, rs.offsets, rs.k, rs.m, rs.lo, rs.hi)
        r = ctx.count_device(dev(rs.reads), dev_u64(rs.offsets), rs.k, rs.m, rs.lo, rs.hi)
        want = ctx.result_to_host(r)
        again = ctx.count(rs.reads, rs.offsets, rs.k, rs.m, rs.lo, rs.hi)
    assert_same_result(got, want, "chunked host input")
    assert_same_result(again, want, "chunked host input, second call")
    assert got.n_windows == oracle.n_windows(rs.reads, rs.offsets, rs.k)


@pytest.mark.parametrize("limit", [1, 1000, 50_000])
def test_bounded_wait_gives_up_and_context_stays_usable(hsk, tiny, limit):
    """A look-back wait on a status word nothing publishes gives up after its
    spin limit: the kernel returns, the host reads HSK_ETIMEOUT, and the same
    context then counts correctly (no GPU fault, no hang)."""
    n = 2000
    reads, offs = tiny.reads[: int(tiny.offsets[n])], tiny.offsets[: n + 1]
    want = oracle.count(reads, offs, 31, 2, 1000)
    with hsk.Context() as ctx:
        assert ctx.wait_timeout(limit) == -4  # HSK_ETIMEOUT
        assert_same_result(ctx.count(reads, offs, 31, 17, 2, 1000), want, "after a timed-out wait")
        assert ctx.wait_timeout(limit) == -4


def test_heavy_hitter_task_is_counted_on_chip(hsk):
    """Sec. 3.5: a task far above the mean size (here: one k-mer with ~20,000
    copies) is turned into a k-mer list on chip; nothing goes to the global
    radix path, and the result is the oracle's."""
    strs = ["A" * 20_000, "ACGTTGCA" * 40, "C" * 5_000]
    offs = np.zeros(len(strs) + 1, np.uint64)
    offs[1:] = np.cumsum([len(x) for x in strs])
    reads = np.frombuffer("".join(strs).encode(), np.uint8).copy()
    want = oracle.count(reads, offs, 31, 2, 100000)
    with hsk.Context() as ctx:
        got = ctx.count(reads, offs, 31, 17, 2, 100000)
        assert ctx.last_overflow() == 0
    assert_same_result(got, want, "poly-A")


def test_task_with_too_many_distinct_keys_takes_the_global_path(hsk):
    """A heavy task whose distinct keys overfill the on-chip k-mer list (20,000
    distinct 31-mers sharing their top digit, each twice) goes to the global
    radix passes; the result is the oracle's."""
    rng = np.random.default_rng(3)
    body = rng.choice(np.array(list("ACGT")), size=(20_000, 27))
    strs = ["AAAA" + "".join(r) for r in body]
    strs = strs + strs
    offs = np.zeros(len(strs) + 1, np.uint64)
    offs[1:] = np.cumsum([len(x) for x in strs])
    reads = np.frombuffer("".join(strs).encode(), np.uint8).copy()
    want = oracle.count(reads, offs, 31, 2, 1000)
    with hsk.Context() as ctx:
        got = ctx.count(reads, offs, 31, 17, 2, 1000)
        assert ctx.last_overflow() == 40_000
    assert_same_result(got, want, "distinct-heavy")


@pytest.mark.parametrize("k,m,B", [(31, 17, 0), (55, 21, 0), (21, 11, 64), (31, 11, 1)])
def test_lexical_minimizer_order_gives_the_same_counts(hsk, tiny, k, m, B):
    """E14: ordering m-mers lexically instead of by hash changes supermers and
    buckets (poly-A-like m-mers attract many k-mers) but not one count."""
    n = 6000
    reads, offs = tiny.reads[: int(tiny.offsets[n])], tiny.offsets[: n + 1]
    reads = np.concatenate([reads, np.frombuffer(b"A" * 3000 + b"C" * 500, np.uint8)])
    offs = np.concatenate([offs, [offs[-1] + 3000, offs[-1] + 3500]]).astype(np.uint64)
    want = oracle.count(reads, offs, k, 2, 1000)
    with hsk.Context(lexical_minimizers=True, n_buckets=B) as lex, hsk.Context(n_buckets=B) as hsh:
        a = lex.count(reads, offs, k, m, 2, 1000)
        b = hsh.count(reads, offs, k, m, 2, 1000)
    assert_same_result(a, want, f"lexical k={k}")
    assert_same_result(b, want, f"hash k={k}")
    assert a.n_supermers != b.n_supermers or B == 1
