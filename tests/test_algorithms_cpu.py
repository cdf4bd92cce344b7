"""CPU checks of two facts the GPU kernels are built on (no GPU, no oracle).

1. The partition's count pass needs only the top 8-bit digit of each
   canonical k-mer, and takes it as the smaller of the forward k-mer's first
   four bases and the reverse complement's first four (the last four bases,
   complemented, read backwards): the top digit of min(x, y) is the smaller
   of the top digits of x and y.

2. The S2 walk takes each window minimum over w = k - m + 1 m-mer scores
   from 32-lane blocks of scores: for w <= 33 as two overlapping runs of
   D = 2^L <= w scores, whose minima are computed within a block and
   completed by a prefix minimum of the next block; for w > 33 as a suffix
   minimum of the first block, then a prefix minimum of the next (and the
   whole block between when the window reaches a third).  The tests restate
   those decompositions lane by lane in numpy and compare them with the
   brute-force sliding minimum for every w the kernel accepts.
"""
import numpy as np
import pytest


def _code(bases):
    v = 0
    for b in bases:
        v = (v << 2) | int(b)
    return v


@pytest.mark.parametrize("k", [4, 5, 8, 17, 31, 32, 33, 55, 64])
def test_canonical_top_digit_is_the_smaller_end_digit(k):
    rng = np.random.default_rng(k)
    for trial in range(3000):
        if trial % 7 == 0:  # low-complexity k-mers (ties between the end digits)
            bases = rng.integers(0, 2, k)
        else:
            bases = rng.integers(0, 4, k)
        fwd = _code(bases)
        rc = _code(3 - bases[::-1])
        canon = min(fwd, rc)
        top = canon >> (2 * k - 8)
        first4 = _code(bases[:4])
        rc_first4 = _code(3 - bases[::-1][:4])  # complemented last four, read backwards
        assert top == min(first4, rc_first4), (k, bases)


def _brute_minima(x, w, n):
    return np.array([x[i:i + w].min() for i in range(n)], dtype=np.int64)


def _range_min_trunc(v, L):
    """min(v[l .. l + 2^L - 1]) within a 32-lane block, lanes past 31 ignored."""
    v = v.copy()
    lanes = np.arange(32)
    for j in range(L):
        d = 1 << j
        o = np.roll(v, -d)  # shfl_down by d
        v = np.where(lanes + d < 32, np.minimum(v, o), v)
    return v


def _prefix_min_upto(v, n):
    v = v.copy()
    lanes = np.arange(32)
    d = 1
    while d < n:
        o = np.roll(v, d)  # shfl_up by d
        v = np.where(lanes >= d, np.minimum(v, o), v)
        d <<= 1
    return v


def _suffix_min(v):
    return np.minimum.accumulate(v[::-1])[::-1]


def _narrow_minima(x, w, steps):
    """w <= 33: the carried-run form, step by step (lane l of step s = window 32 s + l)."""
    L = 0
    while (2 << L) <= w:
        L += 1
    D = 1 << L
    lanes = np.arange(32)
    blocks = [x[32 * s:32 * s + 32] for s in range(steps + 1)]
    t_cur = _range_min_trunc(blocks[0], L)
    out = []
    for s in range(steps):
        x1 = blocks[s + 1]
        t_new = _range_min_trunc(x1, L)
        pm1 = _prefix_min_upto(x1, D - 1)
        i1 = lanes + D - 33
        pv = pm1[i1 & 31]
        tc = np.where(i1 >= 0, np.minimum(t_cur, pv), t_cur)
        q = lanes + w - D
        a = tc[q & 31]
        b = t_new[(q - 32) & 31]
        out.append(np.minimum(tc, np.where(q < 32, a, b)))
        t_cur = t_new
    return np.concatenate(out)


def _wide_minima(x, w, steps):
    """33 < w <= 65: suffix minima of block 0, prefix minima of blocks 1 and 2."""
    lanes = np.arange(32)
    blocks = [x[32 * s:32 * s + 32] for s in range(steps + 2)]
    pm_next = np.minimum.accumulate(blocks[1])
    out = []
    for s in range(steps):
        pm2 = np.minimum.accumulate(blocks[s + 2])
        sm0 = _suffix_min(blocks[s])
        e = lanes + w - 1
        a = pm_next[(e - 32) & 31]
        b = pm2[(e - 64) & 31]
        full1 = pm_next[31]
        out.append(np.minimum(sm0, np.where(e < 64, a, np.minimum(full1, b))))
        pm_next = pm2
    return np.concatenate(out)


@pytest.mark.parametrize("w", list(range(1, 66)))
def test_block_window_minima_equal_the_sliding_minimum(w):
    rng = np.random.default_rng(1000 + w)
    steps = 6
    x = rng.integers(0, 1 << 12, 32 * (steps + 3)).astype(np.int64)  # small range: many ties
    want = _brute_minima(x, w, 32 * steps)
    got = _narrow_minima(x, w, steps) if w <= 33 else _wide_minima(x, w, steps)
    assert np.array_equal(got, want), w
