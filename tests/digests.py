"""Digests of counting results in the format of tests/golden/fullsize_digests.json
(written by tests/golden/make_fullsize_digests.py from the oracle alone)."""
import hashlib
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize_digests.json")


def golden():
    return json.load(open(GOLDEN))["jobs"]


def reads_sha(reads, offsets) -> str:
    h = hashlib.sha256()
    h.update(memoryview(np.ascontiguousarray(reads, dtype=np.uint8)))
    h.update(memoryview(np.ascontiguousarray(offsets, dtype="<u8")))
    return h.hexdigest()


def pairs_sha(kmers, counts) -> str:
    h = hashlib.sha256()
    h.update(memoryview(np.ascontiguousarray(kmers, dtype="<u8").reshape(-1)))
    h.update(memoryview(np.ascontiguousarray(counts, dtype="<u4")))
    return h.hexdigest()


def hist_sha(hist) -> str:
    return hashlib.sha256(memoryview(np.ascontiguousarray(hist, dtype="<u8"))).hexdigest()


def check(res, want: dict, label: str):
    """A result against its golden entry: scalars, then the pair and histogram digests."""
    got = {"n_windows": res.n_windows, "n_distinct": res.n_distinct, "max_count": res.max_count,
           "n_pairs": int(res.counts.size)}
    exp = {k: want[k] for k in got}
    assert got == exp, (label, got, exp)
    assert [int(x) for x in res.hist[:64]] == want["hist_head"], label
    assert hist_sha(res.hist) == want["hist_sha256"], label
    assert pairs_sha(res.kmers, res.counts) == want["pairs_sha256"], label
