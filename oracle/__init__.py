"""CPU oracle for sorting-based k-mer counting (HySortK, arXiv 2407.07718).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this package.  The library
(``paper_2407_07718_gb300``) never imports it and shares no code with it.

The counting itself is plain single-threaded C++ in ``hsk_oracle.cpp`` (one
window at a time, ``std::sort``, one linear scan); this module only compiles it
with g++ and marshals numpy arrays through ctypes.

Functions and the passage each follows:
  count          -- Sec. 2.1 (k-mer counting) and Sec. 3.1 (sort, linear scan,
                    frequency filter, histogram).
  count_keys     -- the same definition, restricted to chosen k-mers (sampled
                    parity at full size).
  encode         -- Sec. 2.2 (2-bit encoding of reads).
  windows        -- Sec. 3.2 (hash-scored minimizer via the monotone deque).
  supermers      -- Sec. 2.4 and Sec. 3.2 (supermers), Sec. 3.4 (tasks).
  sort_u64       -- Sec. 3.1 (the sort alone is std::sort).
  count_ext      -- Sec. 3.3.2 (extension information: each kept k-mer's
                    occurrences as (read, position)).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hsk_oracle.cpp")
_LIB = os.path.join(_HERE, "libhsk_oracle.so")
_lock = threading.Lock()
_lib = None

# Seed XOR-ed into each folded canonical m-mer before the finalizer (its low
# 32 bits are used; fmix32(0) = 0 would otherwise always make poly-A the
# minimizer).  Passed explicitly to both the oracle and the library; counts
# never depend on it.
DEFAULT_SEED = 0x9E3779B97F4A7C15


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain -O2, no -march flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC,
                               "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class _Result(C.Structure):
    _fields_ = [
        ("n_windows", C.c_uint64),
        ("n_distinct", C.c_uint64),
        ("n_pairs", C.c_uint64),
        ("max_count", C.c_uint32),
        ("key_words", C.c_int),
        ("kmers", C.POINTER(C.c_uint64)),
        ("counts", C.POINTER(C.c_uint32)),
        ("hist", C.POINTER(C.c_uint64)),
        ("hist_len", C.c_uint32),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            u64, u32, i32 = C.c_uint64, C.c_uint32, C.c_int
            lib.oracle_count.argtypes = [P, P, u64, i32, u32, u32, u32, C.POINTER(_Result)]
            lib.oracle_count.restype = i32
            lib.oracle_free.argtypes = [C.POINTER(_Result)]
            lib.oracle_count_keys.argtypes = [P, P, u64, i32, P, u64, i32, P, P]
            lib.oracle_count_keys.restype = i32
            lib.oracle_encode.argtypes = [P, u64, P, P]
            lib.oracle_n_windows.argtypes = [P, P, u64, i32]
            lib.oracle_n_windows.restype = u64
            lib.oracle_windows.argtypes = [P, P, u64, i32, i32, u64, P, P, P, P]
            lib.oracle_windows.restype = u64
            lib.oracle_supermers.argtypes = [P, P, u64, i32, i32, u64, u32, P, P, P, P]
            lib.oracle_supermers.restype = u64
            lib.oracle_sort_u64.argtypes = [P, u64]
            lib.oracle_count_ext.argtypes = [P, P, u64, i32, u32, u32, P, P, P, P, P]
            lib.oracle_count_ext.restype = C.c_int64
            lib.oracle_fmix64.argtypes = [u64]
            lib.oracle_fmix64.restype = u64
            lib.oracle_fmix32.argtypes = [u32]
            lib.oracle_fmix32.restype = u32
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _as_inputs(reads, offsets):
    reads = np.ascontiguousarray(np.frombuffer(reads, dtype=np.uint8)
                                 if isinstance(reads, (bytes, bytearray)) else reads,
                                 dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    if reads.size == 0:
        reads = np.zeros(1, dtype=np.uint8)  # valid pointer for empty input
    return reads, offsets


@dataclass
class CountResult:
    kmers: np.ndarray       # (n_pairs,) uint64, or (n_pairs, 2) uint64 {lo, hi}
    counts: np.ndarray      # (n_pairs,) uint32
    hist: np.ndarray        # (hist_len,) uint64
    n_windows: int
    n_distinct: int
    max_count: int
    key_words: int


def count(reads, offsets, k: int, lo: int, hi: int, hist_len: int = 65536) -> CountResult:
    """Exact canonical k-mer counts of the reads (see module docstring)."""
    lib = _load()
    reads, offsets = _as_inputs(reads, offsets)
    n_reads = offsets.size - 1
    r = _Result()
    rc = lib.oracle_count(_ptr(reads), _ptr(offsets), n_reads, k, lo, hi, hist_len, C.byref(r))
    if rc != 0:
        lib.oracle_free(C.byref(r))
        raise ValueError(f"oracle_count rejected its arguments (k={k}, lo={lo}, hi={hi})")
    try:
        n, kw = r.n_pairs, r.key_words
        kmers = np.ctypeslib.as_array(r.kmers, shape=(max(n * kw, 1),))[: n * kw].copy()
        if kw == 2:
            kmers = kmers.reshape(n, 2)
        counts = np.ctypeslib.as_array(r.counts, shape=(max(n, 1),))[:n].copy()
        hist = np.ctypeslib.as_array(r.hist, shape=(r.hist_len,)).copy()
        return CountResult(kmers, counts, hist, int(r.n_windows), int(r.n_distinct),
                           int(r.max_count), kw)
    finally:
        lib.oracle_free(C.byref(r))


def count_keys(reads, offsets, k: int, query: np.ndarray, n_threads: int = 0):
    """Occurrence count of each given canonical k-mer, by a full scan of the reads.

    ``query`` is (n,) uint64 for k <= 32 or (n, 2) uint64 {lo, hi} for k > 32.
    Returns (counts uint64[n], n_windows).
    """
    lib = _load()
    reads, offsets = _as_inputs(reads, offsets)
    q = np.ascontiguousarray(query, dtype=np.uint64)
    nq = q.shape[0] if q.size else 0
    out = np.zeros(max(nq, 1), dtype=np.uint64)
    nw = np.zeros(1, dtype=np.uint64)
    nt = n_threads or max(1, min(os.cpu_count() or 1, 64))
    rc = lib.oracle_count_keys(_ptr(reads), _ptr(offsets), offsets.size - 1, k,
                               _ptr(q if q.size else np.zeros(2, np.uint64)), nq, nt,
                               _ptr(out), _ptr(nw))
    if rc != 0:
        raise ValueError("oracle_count_keys rejected its arguments")
    return out[:nq], int(nw[0])


def encode(reads):
    """Per-base 2-bit code (invalid bases read as 0) and invalid flag."""
    lib = _load()
    reads = np.ascontiguousarray(np.frombuffer(reads, np.uint8) if isinstance(reads, (bytes, bytearray)) else reads, dtype=np.uint8)
    code = np.zeros(reads.size, np.uint8)
    inv = np.zeros(reads.size, np.uint8)
    if reads.size:
        lib.oracle_encode(_ptr(reads), reads.size, _ptr(code), _ptr(inv))
    return code, inv


def n_windows(reads, offsets, k: int) -> int:
    lib = _load()
    reads, offsets = _as_inputs(reads, offsets)
    return int(lib.oracle_n_windows(_ptr(reads), _ptr(offsets), offsets.size - 1, k))


def windows(reads, offsets, k: int, m: int, seed: int = DEFAULT_SEED):
    """Per valid window: (pos, key (n,2) {lo,hi}, minhash, minimizer position)."""
    lib = _load()
    reads, offsets = _as_inputs(reads, offsets)
    n = n_windows(reads, offsets, k)
    pos = np.zeros(n + 1, np.uint64)
    key = np.zeros((n + 1, 2), np.uint64)
    mh = np.zeros(n + 1, np.uint64)
    mp = np.zeros(n + 1, np.uint64)
    got = lib.oracle_windows(_ptr(reads), _ptr(offsets), offsets.size - 1, k, m, seed,
                             _ptr(pos), _ptr(key), _ptr(mh), _ptr(mp))
    assert got == n
    return pos[:n], key[:n], mh[:n], mp[:n]


def supermers(reads, offsets, k: int, m: int, n_buckets: int, seed: int = DEFAULT_SEED):
    """Maximal same-bucket runs: (start pos, n_kmers, bucket) and k-mers per bucket."""
    lib = _load()
    reads, offsets = _as_inputs(reads, offsets)
    n = n_windows(reads, offsets, k)
    sp = np.zeros(n + 1, np.uint64)
    sn = np.zeros(n + 1, np.uint32)
    sb = np.zeros(n + 1, np.uint32)
    bk = np.zeros(n_buckets, np.uint64)
    ns = lib.oracle_supermers(_ptr(reads), _ptr(offsets), offsets.size - 1, k, m, seed,
                              n_buckets, _ptr(sp), _ptr(sn), _ptr(sb), _ptr(bk))
    return sp[:ns], sn[:ns], sb[:ns], bk


@dataclass
class ExtResult:
    kmers: np.ndarray       # (n,) uint64 or (n, 2) uint64 {lo, hi}, ascending
    counts: np.ndarray      # (n,) uint32
    occ_offsets: np.ndarray  # (n + 1,) uint64: k-mer i's occurrences are [occ_offsets[i], occ_offsets[i+1])
    occ_read: np.ndarray    # uint32 read index of each occurrence
    occ_pos: np.ndarray     # uint32 position in the read (window start)
    key_words: int = 1


def count_ext(reads, offsets, k: int, lo: int, hi: int) -> ExtResult:
    """Kept k-mers with their occurrences (read, position), Sec. 3.3.2."""
    lib = _load()
    reads, offsets = _as_inputs(reads, offsets)
    n = offsets.size - 1
    npairs = np.zeros(1, np.uint64)
    no = lib.oracle_count_ext(_ptr(reads), _ptr(offsets), n, k, lo, hi, _ptr(npairs), None, None, None, None)
    if no < 0:
        raise ValueError("oracle_count_ext rejected its arguments")
    kw = 1 if k <= 32 else 2
    np_ = int(npairs[0])
    kmers = np.zeros(max(np_ * kw, 1), np.uint64)
    counts = np.zeros(max(np_, 1), np.uint32)
    occ_read = np.zeros(max(no, 1), np.uint32)
    occ_pos = np.zeros(max(no, 1), np.uint32)
    lib.oracle_count_ext(_ptr(reads), _ptr(offsets), n, k, lo, hi, _ptr(npairs), _ptr(kmers), _ptr(counts),
                         _ptr(occ_read), _ptr(occ_pos))
    kmers, counts = kmers[: np_ * kw], counts[:np_]
    if kw == 2:
        kmers = kmers.reshape(np_, 2)
    offs = np.zeros(np_ + 1, np.uint64)
    offs[1:] = np.cumsum(counts, dtype=np.uint64)
    return ExtResult(kmers, counts, offs, occ_read[:no], occ_pos[:no], kw)


def sort_u64(keys: np.ndarray) -> np.ndarray:
    lib = _load()
    a = np.ascontiguousarray(keys, dtype=np.uint64).copy()
    if a.size:
        lib.oracle_sort_u64(_ptr(a), a.size)
    return a


def fmix64(x: int) -> int:
    return int(_load().oracle_fmix64(x))


def fmix32(x: int) -> int:
    return int(_load().oracle_fmix32(x))
