"""The sort entry point for callers that cannot allocate device memory.

hsk_sort_keys_noalloc keeps its scratch in a fixed array inside the library
instead of calling cudaMalloc, for callers whose device memory belongs to
another allocator or who must avoid the synchronization that allocation can
imply.  These checks call it through the C ABI twice in a row and compare each
result with the existing sort entry point (hsk_stage_sort), bit for bit: keys
are integers, so the tolerance is zero, as in every other sort test here.  The
file is collected last so that a run stopping at the first failure has already
run everything else; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from gpu_util import dev_u64, host_u64

pytestmark = pytest.mark.gpu


def _keys(seed, n, kw, bits):
    rng = np.random.default_rng(seed)
    if kw == 1:
        return rng.integers(0, 1 << bits, size=n, dtype=np.uint64)
    lo = rng.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, n, dtype=np.uint64)
    hi = rng.integers(0, 1 << (bits - 64), size=n, dtype=np.uint64)
    hi[rng.integers(0, n, n // 4)] = hi[0]  # equal high words: order decided by the low word
    return np.stack([lo, hi], axis=1).reshape(-1)


@pytest.mark.parametrize("kw,bits,sizes", [(1, 62, (1_000_003, 654_321)), (2, 110, (400_001, 524_288))])
def test_noalloc_sort_matches_stage_sort_on_two_calls_in_a_row(hsk, kw, bits, sizes):
    with hsk.Context() as ctx:
        for call, n in enumerate(sizes):
            x = _keys(100 * kw + call, n, kw, bits)
            a, b = dev_u64(x), dev_u64(x)
            assert hsk.sort_keys_noalloc(a, n, kw, bits) == hsk.HSK_OK, f"call {call}"
            ctx.stage_sort(b, n, kw, bits)
            got, want = host_u64(a), host_u64(b)
            assert np.array_equal(got, want), f"call {call}: differs from hsk_stage_sort"
            # and both are the sorted keys
            if kw == 1:
                assert np.array_equal(got, np.sort(x))


def test_noalloc_sort_rejects_sizes_beyond_its_scratch(hsk):
    import torch
    t = torch.zeros(4, dtype=torch.int64, device="cuda")
    assert hsk.sort_keys_noalloc(t, hsk.NOALLOC_MAX_KEYS[1] + 1, 1, 62) == hsk.HSK_EOVERFLOW
    assert hsk.sort_keys_noalloc(t, hsk.NOALLOC_MAX_KEYS[2] + 1, 2, 110) == hsk.HSK_EOVERFLOW
    assert hsk.sort_keys_noalloc(t, 4, 3, 62) == hsk.HSK_EINVAL
