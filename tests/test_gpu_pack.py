"""Packed passes of the batched and served forms (hsk_pack.cu): many small
read sets with the same k, m and filter counted by one pass of the pipeline.
Every set's result must be bit-exact with the CPU oracle run on that set
alone, whatever sets share its pass -- including empty sets, sets whose reads
are all shorter than k or all invalid, sets whose size is or is not a whole
number of warp tiles, and a set too repetitive for the on-chip sort (which
the pass hands back to be counted alone)."""
import numpy as np
import pytest

import datagen
import oracle
from gpu_util import assert_same_result

pytestmark = pytest.mark.gpu


def _pack(strs):
    offs = np.zeros(len(strs) + 1, np.uint64)
    offs[1:] = np.cumsum([len(s) for s in strs])
    reads = np.frombuffer("".join(strs).encode(), np.uint8).copy() if strs else np.zeros(0, np.uint8)
    return reads, offs


def _edge_sets(k):
    """Degenerate sets that a pass must carry without disturbing the others."""
    rng = np.random.default_rng(k)
    acgt = np.array(list("ACGT"))
    out = []
    out.append(_pack([]))                                            # no reads
    out.append(_pack(["ACG"[: min(3, k - 1)], "A" * (k - 1)]))        # every read shorter than k
    out.append(_pack(["N" * 500, "n" * 300]))                        # no valid base
    out.append(_pack(["".join(rng.choice(acgt, 1024))]))             # exactly one warp tile
    out.append(_pack(["".join(rng.choice(acgt, 1025))]))             # one base over
    s = "".join(rng.choice(acgt, 3000))
    out.append(_pack([s, s, s[::-1], "N" * 7 + s[:400]]))            # repeats, invalid bases
    return out


def _small_jobs(k, m, lo, hi, n_sets, seed):
    jobs = []
    rng = np.random.default_rng(seed)
    for i in range(n_sets):
        g = int(np.exp(rng.uniform(np.log(2_000), np.log(60_000))))
        cov = float(rng.uniform(5, 20))
        if k == 31:
            rs = datagen.batched_set(datagen.derive_seed(seed, i), g, cov)
        else:
            rs = datagen.served_request(datagen.derive_seed(seed, i), g, cov, bool(i % 3 == 0), k, m)
        jobs.append((rs.reads, rs.offsets, k, m, lo, hi))
    for r, o in _edge_sets(k):
        jobs.insert(int(rng.integers(0, len(jobs) + 1)), (r, o, k, m, lo, hi))
    return jobs


def _oracle(jobs):
    return [oracle.count(r, o, k, lo, hi) for (r, o, k, m, lo, hi) in jobs]


@pytest.mark.parametrize("k,m,lo,hi", [(31, 17, 2, 1000), (55, 21, 2, 1000), (21, 11, 2, 1000), (64, 32, 1, 5),
                                       (33, 17, 2, 8)])
def test_count_batch_packs_small_sets_bit_exact(hsk, k, m, lo, hi):
    jobs = _small_jobs(k, m, lo, hi, 24, 100 + k)
    wants = _oracle(jobs)
    with hsk.Context() as ctx:
        got = ctx.count_batch(jobs)
        stats = ctx.pack_stats()
        for i, (g, w) in enumerate(zip(got, wants)):
            assert_same_result(g, w, f"k={k} set {i}")
        assert stats["passes"] >= 1 and stats["sets"] >= 8, stats
        # the same batch again on the warm slots, in another order
        order = np.random.default_rng(1).permutation(len(jobs))
        again = ctx.count_batch([jobs[i] for i in order])
        for g, i in zip(again, order):
            assert_same_result(g, wants[i], f"k={k} set {i} (permuted)")


def _distinct_heavy_set(n=20_000, seed=3):
    """n distinct 31-mers that all start with AAAA, each read twice: their
    canonical keys share the top digit, so one sub-segment holds all of them --
    more distinct keys than the heavy-hitter table holds."""
    rng = np.random.default_rng(seed)
    acgt = np.array(list("ACGT"))
    body = rng.choice(acgt, size=(n, 27))
    reads = ["AAAA" + "".join(r) for r in body]
    return _pack(reads + reads)


def test_pack_handles_heavy_hitters_and_hands_back_what_it_cannot(hsk):
    """A poly-A read makes one k-mer with ~20,000 copies: its sub-segment is a
    heavy-hitter task (over the on-chip capacity), folded into a k-mer list on
    chip inside the pass.  A set whose one sub-segment holds more distinct
    keys than that table is handed back and counted alone.  Every set stays
    bit-exact."""
    jobs = _small_jobs(31, 17, 2, 100000, 12, 7)
    r, o = _pack(["A" * 20_000, "ACGT" * 50])
    jobs.insert(5, (r, o, 31, 17, 2, 100000))
    r2, o2 = _distinct_heavy_set()
    jobs.insert(9, (r2, o2, 31, 17, 2, 100000))
    wants = _oracle(jobs)
    with hsk.Context() as ctx:
        got = ctx.count_batch(jobs)
        stats = ctx.pack_stats()
    for i, (g, w) in enumerate(zip(got, wants)):
        assert_same_result(g, w, f"set {i}")
    assert got[5].max_count == 20_000 - 31 + 1
    assert stats["alone"] == 1, stats  # the distinct-heavy set only


def test_packed_results_equal_plain_calls(hsk):
    jobs = _small_jobs(31, 17, 2, 1000, 16, 11)
    with hsk.Context() as ctx:
        plain = [ctx.count(*j) for j in jobs]
        batch = ctx.count_batch(jobs)
        assert ctx.pack_stats()["sets"] >= 8
    for i, (p, b) in enumerate(zip(plain, batch)):
        assert_same_result(b, p, f"set {i}")


def test_served_small_requests_share_passes(hsk):
    """Requests queued while the slots are busy are packed together; each
    result is the oracle's for that request alone."""
    jobs = _small_jobs(31, 17, 2, 1000, 30, 21) + _small_jobs(55, 21, 2, 1000, 10, 22)
    wants = _oracle(jobs)
    with hsk.Context() as ctx:
        tickets = [ctx.submit(*j) for j in jobs]
        for i in np.random.default_rng(3).permutation(len(jobs)):
            assert_same_result(ctx.wait(tickets[i]), wants[i], f"request {i}")
        for t in tickets:
            ctx.release(t)
        stats = ctx.pack_stats()
    assert stats["passes"] >= 1, stats


def test_pack_with_a_failing_set_reports_it_and_keeps_the_others(hsk):
    jobs = _small_jobs(31, 17, 2, 1000, 10, 31)
    wants = _oracle(jobs)
    i_bad = next(i for i, j in enumerate(jobs) if j[1].size > 10)
    r, o = jobs[i_bad][0], jobs[i_bad][1].copy()
    o[2], o[3] = o[3], o[2]  # not monotone: this set fails with HSK_EINVAL
    bad = list(jobs)
    bad[i_bad] = (r, o, 31, 17, 2, 1000)
    with hsk.Context() as ctx:
        with pytest.raises(hsk.HskError) as e:
            ctx.count_batch(bad)
        assert e.value.code == -1 and f"job {i_bad}" in str(e.value)
        got = ctx.count_batch(jobs)
    for i, (g, w) in enumerate(zip(got, wants)):
        assert_same_result(g, w, f"set {i} after a failed batch")
