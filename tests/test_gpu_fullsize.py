"""Full-size workloads in the launch configuration the benchmark times
(hsk_count_device on device-resident reads, default context).

The oracle cannot sort 1.5 G windows in seconds, so the full output is
checked by properties that hold at any size, and sampled k-mers are checked
one by one against the oracle's exact occurrence count over the whole read
set:
  * n_windows equals the closed form (valid windows per read, no sort);
  * output keys strictly ascending, counts inside [lo, hi];
  * histogram: hist[0] = 0, sum c*hist[c] = n_windows, sum hist = n_distinct,
    sum over [lo, hi] of hist = n_pairs;
  * sampled output pairs: their counts equal the oracle's;
  * sampled k-mers of the input, present or not in the output: present exactly
    when the oracle's count lies in [lo, hi], and then with that count;
  * and the whole result, bit for bit: the SHA-256 of the (k-mer, count) pairs
    and of the histogram, and every scalar, against the oracle's full-size run
    recorded in tests/golden/fullsize_digests.json (written by the oracle alone;
    the SHA-256 of the simulated reads is checked first, so a simulator that
    drifted between machines fails as such, not as counting).
"""
import numpy as np
import pytest

import datagen
import oracle
import digests
from gpu_util import dev, dev_u64

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

_PAIR = np.dtype([("hi", "<u8"), ("lo", "<u8")])


def _as_pairs(keys, kw):
    """Keys in an array whose order is the numeric order of the 2k-bit value."""
    if kw == 1:
        return np.ascontiguousarray(keys, dtype=np.uint64)
    p = np.empty(keys.shape[0], _PAIR)
    p["hi"], p["lo"] = keys[:, 1], keys[:, 0]
    return p


@pytest.fixture(scope="module", params=["long_read", "short_read"])
def case(request, hsk):
    rs = datagen.long_read() if request.param == "long_read" else datagen.short_read()
    with hsk.Context() as ctx:
        r = ctx.count_device(dev(rs.reads), dev_u64(rs.offsets), rs.k, rs.m, rs.lo, rs.hi)
        got = ctx.result_to_host(r)
    import torch
    torch.cuda.empty_cache()
    return request.param, rs, got


def test_invariants(case):
    name, rs, got = case
    kw = 1 if rs.k <= 32 else 2
    assert got.key_words == kw
    assert got.n_windows == oracle.n_windows(rs.reads, rs.offsets, rs.k)
    n = got.counts.size
    assert n > 0 and got.kmers.shape[0] == n
    if kw == 1:
        assert np.all(got.kmers[1:] > got.kmers[:-1]), name
        assert int(got.kmers.max()) < (1 << (2 * rs.k))
    else:
        hi, lo = got.kmers[:, 1], got.kmers[:, 0]
        asc = (hi[1:] > hi[:-1]) | ((hi[1:] == hi[:-1]) & (lo[1:] > lo[:-1]))
        assert np.all(asc), name
        assert int(hi.max()) < (1 << (2 * rs.k - 64))
    assert got.counts.min() >= rs.lo and got.counts.max() <= rs.hi
    h = got.hist.astype(np.uint64)
    H = h.size
    assert got.max_count < H - 1, "histogram must hold every count for the sum check"
    c = np.arange(H, dtype=np.uint64)
    assert h[0] == 0
    assert int((c * h).sum()) == got.n_windows
    assert int(h.sum()) == got.n_distinct
    assert int(h[rs.lo: rs.hi + 1].sum()) == n


def test_sampled_output_pairs(case):
    name, rs, got = case
    rng = np.random.default_rng(17)
    idx = np.unique(rng.integers(0, got.counts.size, size=3000))
    q = got.kmers[idx]
    want, nw = oracle.count_keys(rs.reads, rs.offsets, rs.k, q)
    assert nw == got.n_windows
    assert np.array_equal(want, got.counts[idx].astype(np.uint64)), name


def test_sampled_input_kmers_present_iff_in_range(case):
    name, rs, got = case
    kw = got.key_words
    # candidate k-mers: windows of a few reads spread over the set
    rng = np.random.default_rng(23)
    picks = np.sort(rng.choice(rs.n_reads, size=40, replace=False))
    cand = []
    for i in picks:
        a, b = int(rs.offsets[i]), int(rs.offsets[i + 1])
        _, key, _, _ = oracle.windows(rs.reads[a:b], np.array([0, b - a], np.uint64), rs.k, rs.m)
        if key.shape[0]:
            cand.append(key[rng.integers(0, key.shape[0], size=min(100, key.shape[0]))])
    key = np.concatenate(cand)
    key = np.unique(key, axis=0)
    q = key[:, 0].copy() if kw == 1 else key
    want, _ = oracle.count_keys(rs.reads, rs.offsets, rs.k, q)
    out = _as_pairs(got.kmers, kw)
    qs = _as_pairs(q, kw)
    pos = np.searchsorted(out, qs)
    found = (pos < out.size) & (out[np.minimum(pos, out.size - 1)] == qs)
    in_range = (want >= rs.lo) & (want <= rs.hi)
    assert np.array_equal(found, in_range), name
    assert np.array_equal(got.counts[pos[found]].astype(np.uint64), want[found]), name
    # both outcomes were sampled
    assert found.any() and (~found).any(), (name, int(found.sum()), found.size)


def test_bit_exact_against_the_oracles_full_size_run(case):
    name, rs, got = case
    want = digests.golden()[name]
    assert digests.reads_sha(rs.reads, rs.offsets) == want["reads_sha256"], \
        f"{name}: the simulator produced other reads than when the digests were written"
    assert (rs.k, rs.m, rs.lo, rs.hi) == (want["k"], want["m"], want["lo"], want["hi"])
    digests.check(got, want, name)
