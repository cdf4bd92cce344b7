"""Stage-by-stage parity of the CUDA path against the CPU oracle (S1-S6),
called through the C ABI's stage entry points."""
from collections import Counter

import numpy as np
import pytest

import datagen
import oracle
from gpu_util import dev, dev_u64, empty_dev, host_u64

pytestmark = pytest.mark.gpu


def _inputs(seed, n_reads=300, lo=0, hi=400, p_inv=0.01, extra=()):
    reads, offs = datagen.random_reads(seed, n_reads, lo, hi, p_invalid=p_inv, invalid=b"NnX")
    strs = [reads[offs[i]:offs[i + 1]].tobytes().decode() for i in range(len(offs) - 1)] + list(extra)
    offs = np.zeros(len(strs) + 1, np.uint64)
    offs[1:] = np.cumsum([len(s) for s in strs])
    reads = np.frombuffer("".join(strs).encode(), np.uint8).copy()
    return reads, offs


@pytest.mark.parametrize("seed", [0, 1])
def test_s1_encode(hsk, seed):
    import torch
    reads, offs = _inputs(seed, extra=["", "A", "ACGTN" * 30, ""])
    n = reads.size
    code, inv = oracle.encode(reads)
    with hsk.Context() as ctx:
        pk = empty_dev((n + 31) // 32 + 4, torch.int64)
        iv = empty_dev((n + 63) // 64 + 4, torch.int64)
        st = empty_dev((n + 63) // 64 + 4, torch.int64)
        ctx.stage_encode(dev(reads), dev_u64(offs), pk, iv, st)
        pk, iv, st = host_u64(pk), host_u64(iv), host_u64(st)
    g = np.arange(n)
    got_code = (pk[g // 32] >> (62 - 2 * (g % 32)).astype(np.uint64)) & np.uint64(3)
    got_inv = (iv[g // 64] >> (63 - g % 64).astype(np.uint64)) & np.uint64(1)
    got_st = (st[g // 64] >> (63 - g % 64).astype(np.uint64)) & np.uint64(1)
    assert np.array_equal(got_code.astype(np.uint8), code)
    assert np.array_equal(got_inv.astype(np.uint8), inv)
    starts = np.zeros(n, np.uint8)
    for i in range(len(offs) - 1):
        if offs[i + 1] > offs[i]:
            starts[offs[i]] = 1
    assert np.array_equal(got_st.astype(np.uint8), starts)
    assert not pk[(n + 31) // 32:].any() and not st[(n + 63) // 64:].any()


@pytest.mark.parametrize("k,m", [(1, 1), (5, 3), (21, 11), (31, 17), (32, 32), (33, 12), (55, 21),
                                 (64, 1), (64, 32), (40, 8)])
def test_s2_windows(hsk, k, m):
    import torch
    reads, offs = _inputs(k * 100 + m, n_reads=120, lo=0, hi=3000, extra=["ACGT" * 40, "G" * 200])
    n = reads.size
    pos, key, mh, _ = oracle.windows(reads, offs, k, m)
    with hsk.Context() as ctx:
        valid = empty_dev(n, torch.uint8)
        keys = empty_dev(2 * n, torch.int64)
        mins = empty_dev(n, torch.int64)
        ctx.stage_windows(dev(reads), dev_u64(offs), k, m, valid, keys, mins)
        valid = valid.cpu().numpy()[:n]
        keys = host_u64(keys)[: 2 * n].reshape(n, 2)
        mins = host_u64(mins)[:n]
    gv = np.nonzero(valid)[0]
    assert np.array_equal(gv.astype(np.uint64), pos)
    assert np.array_equal(keys[gv], key)
    assert np.array_equal(mins[gv], mh)


def _record_kmers(words, rw, k):
    """(n, canonical keys) of one record, decoded from its words in Python."""
    n = int(words[rw - 1]) & 0xFF
    bits = 0
    for w in words:
        bits = (bits << 64) | int(w)
    total = 64 * rw
    out = []
    mask = (1 << (2 * k)) - 1
    for j in range(n):
        f = (bits >> (total - 2 * (j + k))) & mask
        r = 0
        x = f
        for _ in range(k):
            r = (r << 2) | (3 - (x & 3))
            x >>= 2
        out.append(min(f, r))
    return n, out


@pytest.mark.parametrize("k,m,B", [(31, 17, 64), (31, 17, 1), (21, 11, 4), (55, 21, 128), (16, 8, 4096),
                                   (64, 31, 8), (33, 5, 8192)])
def test_s3_supermers(hsk, k, m, B):
    import torch
    reads, offs = _inputs(k + B, n_reads=150, lo=0, hi=2500)
    pos, key, mh, _ = oracle.windows(reads, offs, k, m)
    _, _, _, want_bk = oracle.supermers(reads, offs, k, m, B)
    want = Counter()
    for i in range(len(pos)):
        want[(int(mh[i]) % B, int(key[i, 0]) | (int(key[i, 1]) << 64))] += 1
    with hsk.Context() as ctx:
        bk = empty_dev(B, torch.int64)
        br = empty_dev(B + 1, torch.int64)
        recp, nrec, rw, nmax = ctx.stage_supermers(dev(reads), dev_u64(offs), k, m, B, bk, br)
        bk, br = host_u64(bk)[:B], host_u64(br)[: B + 1]
        recs = ctx.copy_device_words(recp, nrec * rw).reshape(max(nrec, 0), rw) if nrec else np.zeros((0, rw), np.uint64)
    assert np.array_equal(bk, want_bk)
    assert int(br[B]) == nrec and np.all(np.diff(br.astype(np.int64)) >= 0)
    got = Counter()
    for b in range(B):
        for r in range(int(br[b]), int(br[b + 1])):
            n, ks = _record_kmers(recs[r], rw, k)
            assert 1 <= n <= nmax
            for kk in ks:
                got[(b, kk)] += 1
    assert got == want
    # a supermer holds several k-mers on average (density of minimizers)
    if B > 1 and len(pos) > 1000:
        assert nrec < len(pos) / 2


@pytest.mark.parametrize("bits", [1, 8, 9, 31, 62, 64])
@pytest.mark.parametrize("n", [1, 4095, 4096, 70_001, 1_000_003])
def test_s4_sort_u64(hsk, bits, n):
    rng = np.random.default_rng(bits * 7 + n)
    hi = (1 << bits) if bits < 64 else None
    x = rng.integers(0, hi if hi else 2**63, size=n, dtype=np.uint64)
    if bits == 64:
        x ^= rng.integers(0, 2, size=n, dtype=np.uint64) << np.uint64(63)
    t = dev_u64(x)
    with hsk.Context() as ctx:
        ctx.stage_sort(t, n, 1, bits)
    assert np.array_equal(host_u64(t), np.sort(x))


def test_s4_sort_u64_special_patterns(hsk):
    n = 300_000
    pats = {
        "all_equal": np.full(n, 12345, np.uint64),
        "two_values": np.where(np.arange(n) % 3 == 0, 5, 2**61).astype(np.uint64),
        "descending": np.arange(n, 0, -1).astype(np.uint64) * np.uint64(1 << 20),
        "constant_low_digits": (np.random.default_rng(0).integers(0, 1000, n).astype(np.uint64) << np.uint64(40)),
    }
    with hsk.Context() as ctx:
        for name, x in pats.items():
            t = dev_u64(x)
            ctx.stage_sort(t, n, 1, 62)
            assert np.array_equal(host_u64(t), np.sort(x)), name


@pytest.mark.parametrize("bits", [66, 110, 128])
@pytest.mark.parametrize("n", [5, 2048, 333_333])
def test_s4_sort_u128(hsk, bits, n):
    rng = np.random.default_rng(bits + n)
    lo = rng.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=n, dtype=np.uint64)
    hb = bits - 64
    hi = rng.integers(0, 1 << min(hb, 63), size=n, dtype=np.uint64)
    if hb == 64:
        hi ^= rng.integers(0, 2, size=n, dtype=np.uint64) << np.uint64(63)
    # duplicate a fifth of the keys so equal high words force ordering on the low word
    dup = rng.integers(0, n, size=n // 5)
    hi[dup] = hi[0]
    x = np.stack([lo, hi], axis=1)
    t = dev_u64(x.reshape(-1))
    with hsk.Context() as ctx:
        ctx.stage_sort(t, n, 2, bits)
    got = host_u64(t).reshape(n, 2)
    order = np.lexsort((x[:, 0], x[:, 1]))
    assert np.array_equal(got, x[order])


def _rle_oracle(keys, lo, hi, H):
    u, c = np.unique(keys, return_counts=True, axis=0) if keys.ndim == 2 else np.unique(keys, return_counts=True)
    hist = np.zeros(H, np.uint64)
    np.add.at(hist, np.minimum(c, H - 1), 1)
    sel = (c >= lo) & (c <= hi)
    return u[sel], c[sel].astype(np.uint32), hist, len(u), int(c.max()) if len(c) else 0


@pytest.mark.parametrize("case", ["random", "one_run", "long_runs", "singletons", "tile_edges"])
def test_s5_rle(hsk, case):
    rng = np.random.default_rng(0)
    n = 200_000
    if case == "random":
        x = np.sort(rng.integers(0, 30_000, n).astype(np.uint64))
    elif case == "one_run":
        x = np.full(n, 7, np.uint64)
    elif case == "long_runs":
        x = np.sort(rng.integers(0, 40, n).astype(np.uint64))
    elif case == "singletons":
        x = np.arange(n, dtype=np.uint64) * np.uint64(3)
    else:  # runs of exactly the tile size and tile size +- 1
        lens = [4095, 4096, 4097, 1, 8192, 3, 4096 * 3 + 5]
        x = np.concatenate([np.full(L, i, np.uint64) for i, L in enumerate(lens)])
        n = x.size
    with hsk.Context(hist_len=4096) as ctx:
        for lo, hi in [(1, 2**32 - 1), (2, 8), (3, 100_000)]:
            r = ctx.stage_rle(dev_u64(x), n, 1, lo, hi)
            u, c, hist, d, mx = _rle_oracle(x, lo, hi, 4096)
            assert np.array_equal(r.kmers, u) and np.array_equal(r.counts, c)
            assert np.array_equal(r.hist, hist) and r.n_distinct == d and r.max_count == mx


def test_s5_rle_u128(hsk):
    rng = np.random.default_rng(1)
    n = 100_000
    base = rng.integers(0, 2**62, size=(5000, 2), dtype=np.uint64)
    x = base[rng.integers(0, 5000, n)]
    x = x[np.lexsort((x[:, 0], x[:, 1]))]
    with hsk.Context(hist_len=1024) as ctx:
        r = ctx.stage_rle(dev_u64(x.reshape(-1)), n, 2, 2, 30)
    u, c = np.unique(x, axis=0, return_counts=True)
    order = np.lexsort((u[:, 0], u[:, 1]))
    u, c = u[order], c[order]
    sel = (c >= 2) & (c <= 30)
    assert np.array_equal(r.kmers, u[sel]) and np.array_equal(r.counts, c[sel].astype(np.uint32))
    assert r.n_distinct == len(u)


@pytest.mark.parametrize("kw,bits", [(1, 62), (2, 110)])
def test_s6_order_pairs(hsk, kw, bits):
    import torch
    rng = np.random.default_rng(kw)
    n = 250_000
    if kw == 1:
        keys = rng.choice(2**61, size=n, replace=False).astype(np.uint64)
        order = np.argsort(keys, kind="stable")
    else:
        keys = np.stack([rng.integers(0, 2**63, n, dtype=np.uint64),
                         rng.integers(0, 1 << (bits - 64), n, dtype=np.uint64)], axis=1)
        order = np.lexsort((keys[:, 0], keys[:, 1]))
    counts = rng.integers(1, 1000, n).astype(np.uint32)
    tk, tc = dev_u64(keys.reshape(-1)), dev(counts.view(np.int32), torch.int32)
    with hsk.Context() as ctx:
        ctx.stage_order(tk, tc, n, kw, bits)
    gk = host_u64(tk).reshape(keys.shape)
    gc = tc.cpu().numpy().view(np.uint32)
    assert np.array_equal(gk, keys[order]) and np.array_equal(gc, counts[order])


def _lexical_minimum(strs_offs, k, m, pos):
    """Per valid window start: the smallest lexical score (the canonical m-mer's
    code, its top 32 bits when m > 16) over the window's k - m + 1 m-mers."""
    reads, offs = strs_offs
    b = reads.tobytes().decode()
    code = {"A": 0, "C": 1, "G": 2, "T": 3}

    def canon(s):
        f = 0
        for ch in s:
            f = (f << 2) | code[ch]
        r = 0
        for ch in reversed(s):
            r = (r << 2) | (3 - code[ch])
        c = min(f, r)
        return c >> (2 * m - 32) if m > 16 else c

    return np.array([min(canon(b[p + j:p + j + m]) for j in range(k - m + 1)) for p in pos.tolist()], np.uint64)


@pytest.mark.parametrize("k,m", [(21, 11), (31, 17), (55, 21), (16, 16)])
def test_s2_windows_lexical_order(hsk, k, m):
    """E14's alternative minimizer order (Sec. 3.2): with lexical order the
    window minimum is the smallest canonical m-mer code, checked against a
    brute force over the window's m-mers."""
    import torch
    reads, offs = _inputs(k * 10 + m, n_reads=40, lo=0, hi=400, extra=["ACGT" * 20, "G" * 90])
    n = reads.size
    pos, key, _, _ = oracle.windows(reads, offs, k, m)
    with hsk.Context(lexical_minimizers=True) as ctx:
        valid = empty_dev(n, torch.uint8)
        keys = empty_dev(2 * n, torch.int64)
        mins = empty_dev(n, torch.int64)
        ctx.stage_windows(dev(reads), dev_u64(offs), k, m, valid, keys, mins)
        valid = valid.cpu().numpy()[:n]
        keys = host_u64(keys)[: 2 * n].reshape(n, 2)
        mins = host_u64(mins)[:n]
    gv = np.nonzero(valid)[0]
    assert np.array_equal(gv.astype(np.uint64), pos)
    assert np.array_equal(keys[gv], key)
    assert np.array_equal(mins[gv], _lexical_minimum((reads, offs), k, m, pos))
