"""Helpers shared by the GPU tests (device tensors from numpy, key decoding)."""
import numpy as np


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def dev_u64(a):
    import torch
    return dev(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64), torch.int64)


def host_u64(t):
    return t.cpu().numpy().view(np.uint64)


def empty_dev(n, dtype):
    import torch
    return torch.zeros(max(int(n), 1), dtype=dtype, device="cuda")


def as_int_keys(kmers, key_words):
    """Python ints of a key array ((n,) or (n, 2) {lo, hi})."""
    if key_words == 1:
        return [int(x) for x in kmers]
    return [int(r[0]) | (int(r[1]) << 64) for r in kmers]


def assert_same_result(got, want, label=""):
    assert got.n_windows == want.n_windows, (label, got.n_windows, want.n_windows)
    assert got.n_distinct == want.n_distinct, (label, got.n_distinct, want.n_distinct)
    assert got.max_count == want.max_count, (label, got.max_count, want.max_count)
    assert got.key_words == want.key_words
    assert got.kmers.shape == want.kmers.shape, (label, got.kmers.shape, want.kmers.shape)
    assert np.array_equal(got.kmers, want.kmers), label
    assert np.array_equal(got.counts, want.counts), label
    assert np.array_equal(got.hist, want.hist), label
