"""The sort entry point for callers that cannot allocate device memory.

hsk_sort_keys_noalloc keeps its scratch in a fixed array inside the library
instead of calling cudaMalloc, for callers whose device memory belongs to
another allocator or who must avoid the synchronization that allocation can
imply.  These checks call it through the C ABI twice in a row and compare each
result with the existing sort entry point (hsk_stage_sort) and with numpy's
sort, bit for bit: keys are integers, so the tolerance is zero, as in every
other sort test here.  They include the exact size limits, key widths that are
not whole bytes, 128-bit keys whose high word is zero, and 64-bit keys that
start 8 bytes past a 16-byte boundary.  The file is collected last so that a
run stopping at the first failure has already run everything else; it also
passes alone in a fresh process.
"""
import numpy as np
import pytest

from gpu_util import dev_u64, host_u64

pytestmark = pytest.mark.gpu


def _keys(seed, n, kw, bits):
    rng = np.random.default_rng(seed)
    if kw == 1:
        return rng.integers(0, 1 << bits, size=n, dtype=np.uint64)
    if bits <= 64:
        lo = rng.integers(0, 1 << bits, size=n, dtype=np.uint64)
        hi = np.zeros(n, np.uint64)
    else:
        lo = rng.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, n, dtype=np.uint64)
        hi = rng.integers(0, 1 << (bits - 64), size=n, dtype=np.uint64)
        hi[rng.integers(0, n, n // 4)] = hi[0]  # equal high words: order decided by the low word
    lo[rng.integers(0, n, n // 8)] = lo[1]      # repeated keys
    return np.stack([lo, hi], axis=1).reshape(-1)


def _numpy_sorted(x, kw):
    if kw == 1:
        return np.sort(x)
    k2 = x.reshape(-1, 2)
    return k2[np.lexsort((k2[:, 0], k2[:, 1]))].reshape(-1)


def _check_two_calls(hsk, kw, bits, sizes, seed0):
    with hsk.Context() as ctx:
        for call, n in enumerate(sizes):
            x = _keys(seed0 + call, n, kw, bits)
            a, b = dev_u64(x), dev_u64(x)
            assert hsk.sort_keys_noalloc(a, n, kw, bits) == hsk.HSK_OK, f"call {call}"
            ctx.stage_sort(b, n, kw, bits)
            got, want = host_u64(a), host_u64(b)
            assert np.array_equal(got, want), f"call {call}: differs from hsk_stage_sort"
            assert np.array_equal(got, _numpy_sorted(x, kw)), f"call {call}: not numpy's order"


@pytest.mark.parametrize("kw,bits,sizes", [(1, 62, (1_000_003, 654_321)), (2, 110, (400_001, 524_287))])
def test_noalloc_sort_matches_stage_sort_on_two_calls_in_a_row(hsk, kw, bits, sizes):
    _check_two_calls(hsk, kw, bits, sizes, 100 * kw)


def test_noalloc_sort_at_its_exact_size_limits(hsk):
    _check_two_calls(hsk, 1, 62, (hsk.NOALLOC_MAX_KEYS[1], hsk.NOALLOC_MAX_KEYS[1]), 500)
    _check_two_calls(hsk, 2, 110, (hsk.NOALLOC_MAX_KEYS[2], hsk.NOALLOC_MAX_KEYS[2] - 1), 600)


@pytest.mark.parametrize("kw,bits", [(1, 61), (1, 7), (2, 60), (2, 65), (2, 127)])
def test_noalloc_sort_with_odd_key_widths(hsk, kw, bits):
    _check_two_calls(hsk, kw, bits, (300_001, 77), 700 + bits)


def test_noalloc_sort_of_keys_at_an_8_byte_offset(hsk):
    """64-bit keys that start 8 bytes past a 16-byte boundary (a view one
    element into a tensor); the word before them is left as it was."""
    import torch
    n = 777_777
    x = _keys(900, n, 1, 62)
    t = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    t[0] = 12345
    v = t[1:]
    assert v.data_ptr() % 16 == 8
    v.copy_(torch.from_numpy(x.view(np.int64)).cuda())
    for call in range(2):
        assert hsk.sort_keys_noalloc(v, n, 1, 62) == hsk.HSK_OK, f"call {call}"
        assert np.array_equal(host_u64(v), np.sort(x)), f"call {call}"
        assert int(t[0].item()) == 12345


def test_noalloc_sort_rejects_bad_sizes_and_alignment(hsk):
    import torch
    t = torch.zeros(8, dtype=torch.int64, device="cuda")
    assert hsk.sort_keys_noalloc(t, hsk.NOALLOC_MAX_KEYS[1] + 1, 1, 62) == hsk.HSK_EOVERFLOW
    assert hsk.sort_keys_noalloc(t, hsk.NOALLOC_MAX_KEYS[2] + 1, 2, 110) == hsk.HSK_EOVERFLOW
    assert hsk.sort_keys_noalloc(t, 4, 3, 62) == hsk.HSK_EINVAL
    # 128-bit keys are read as 16-byte words: a view 8 bytes in is refused on the host
    assert t[1:].data_ptr() % 16 == 8
    assert hsk.sort_keys_noalloc(t[1:], 2, 2, 110) == hsk.HSK_EINVAL
