"""Extension information (Sec. 3.3.2) on the GPU: every kept k-mer's
occurrences as (read, position), bit-exact against the oracle's definition
(oracle.count_ext), and the paper's compact encoding of extension
information round-tripped through the device encoder and decoder."""
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


def _check(hsk, reads, offs, k, m, lo, hi, label):
    want = oracle.count_ext(reads, offs, k, lo, hi)
    with hsk.Context() as ctx:
        res, off, rd, ps = ctx.count_ext(reads, offs, k, m, lo, hi)
        plain = ctx.count(reads, offs, k, m, lo, hi)
    assert_same_result(res, plain, label)
    assert np.array_equal(res.kmers, want.kmers), label
    assert np.array_equal(res.counts, want.counts), label
    assert np.array_equal(off, want.occ_offsets), label
    assert np.array_equal(rd, want.occ_read), label
    assert np.array_equal(ps, want.occ_pos), label
    return res, off, rd, ps


@pytest.mark.parametrize("k,m,lo,hi", [(31, 17, 2, 1000), (55, 21, 2, 500), (21, 11, 1, 3), (64, 32, 2, 9),
                                       (13, 7, 2, 100000)])
def test_occurrences_match_the_oracle(hsk, k, m, lo, hi):
    rs = datagen.tiny()
    n = 3000
    reads, offs = rs.reads[: int(rs.offsets[n])].copy(), rs.offsets[: n + 1].copy()
    _check(hsk, reads, offs, k, m, lo, hi, f"tiny k={k}")


def test_occurrences_with_invalid_bases_empty_reads_and_repeats(hsk):
    r, o = datagen.random_reads(41, 400, 0, 300, p_invalid=0.01, invalid=b"Nn")
    strs = [r[int(o[i]):int(o[i + 1])].tobytes().decode() for i in range(o.size - 1)]
    strs = strs + ["", "ACGTACGTAC" * 20, "", "A" * 200] + strs[:50]
    reads, offs = _pack(strs)
    _check(hsk, reads, offs, 31, 17, 2, 1000, "mixed")
    _check(hsk, reads, offs, 15, 9, 1, 2, "mixed k=15")


def test_no_kept_kmer_and_no_reads(hsk):
    reads, offs = _pack(["ACGTTGCA" * 10])
    res, off, rd, ps = _check(hsk, reads, offs, 31, 17, 100, 200, "none kept")
    assert res.counts.size == 0 and off.tolist() == [0] and rd.size == 0
    reads, offs = _pack([])
    _check(hsk, reads, offs, 31, 17, 2, 1000, "no reads")


def test_more_than_2_24_kept_kmers_use_wide_composites(hsk):
    """Over 2^24 kept k-mers: the (index, position) composites take 128 bits."""
    rs = datagen.batched_set(datagen.derive_seed(77, 0), 30_000_000, 1.0)
    res, off, rd, ps = _check(hsk, rs.reads, rs.offsets, 31, 17, 1, 1000, "wide composites")
    assert res.counts.size > (1 << 24)


def _expected_bytes(rd, ps, chunk):
    n = rd.size
    total = 0
    for i in range(n):
        dr, dp = int(rd[i]) - int(rd[i - 1]), int(ps[i]) - int(ps[i - 1])
        small = (i % chunk) != 0 and -128 <= dr <= 127 and -128 <= dp <= 127
        total += 3 if small else 9
    return total


def test_extension_codec_round_trip(hsk):
    """Encode a stream with the paper's flag byte + int8 differences (full
    values when a difference does not fit), decode it, get it back; the
    length is 3 bytes per small-difference item and 9 per full item."""
    import torch
    rng = np.random.default_rng(8)
    n = 5000
    rd = np.cumsum(rng.integers(0, 2, n) * rng.choice([1, 1, 1, 300], n)).astype(np.uint32)
    ps = np.where(rng.random(n) < 0.9, np.cumsum(rng.integers(-5, 6, n)) % 100000,
                  rng.integers(0, 2**32 - 1, n)).astype(np.uint32)
    d_rd = torch.from_numpy(rd.view(np.int32)).cuda()
    d_ps = torch.from_numpy(ps.view(np.int32)).cuda()
    out = torch.zeros(9 * n, dtype=torch.uint8, device="cuda")
    chunks = (n + hsk.EXT_CHUNK - 1) // hsk.EXT_CHUNK
    coff = torch.zeros(chunks, dtype=torch.int64, device="cuda")
    with hsk.Context() as ctx:
        nb = ctx.stage_ext_encode(d_rd, d_ps, out, coff)
        assert nb == _expected_bytes(rd, ps, hsk.EXT_CHUNK)
        assert nb < 9 * n
        back_rd = torch.zeros(n, dtype=torch.int32, device="cuda")
        back_ps = torch.zeros(n, dtype=torch.int32, device="cuda")
        ctx.stage_ext_decode(out, nb, coff, n, back_rd, back_ps)
        assert np.array_equal(back_rd.cpu().numpy().view(np.uint32), rd)
        assert np.array_equal(back_ps.cpu().numpy().view(np.uint32), ps)
        # a stream cut short is refused, not read past its end
        with pytest.raises(hsk.HskError) as e:
            ctx.stage_ext_decode(out, nb - 5, coff, n, back_rd, back_ps)
        assert e.value.code == -1
