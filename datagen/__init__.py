"""Seeded synthetic read sets for the k-mer counter's tests and benchmark.

This module holds none of the counting method's arithmetic; both the CUDA path
and the CPU oracle are fed from it.  Genomes and reads are simulated in
``hsk_datagen.c`` (xoshiro256** seeded by splitmix64) and returned as ASCII
bytes plus CSR offsets (``offsets[i] .. offsets[i+1]`` is read i).

The paper's own datasets (C. elegans, H. sapiens, Citrus, A. baumannii;
Table 1) are not available here; these workloads stand in for them:

  tiny            1 Mbp uniform genome; 20,000 x 150 bp reads, 50 % reverse
                  complemented, 1 % substitutions, no N (k=31, m=17).
  long_read       50 Mbp genome with 20 repeat families x 100 copies
                  (1-20 kb, 0-2 % divergence); 30x coverage of log-normal
                  reads (mean 10 kb, sd 4 kb, min 1 kb), 0.5 % substitutions,
                  0.05 % insertions + 0.05 % deletions, random strand
                  (k=31, m=17).
  short_read      100 Mbp genome with a 20 Mbp 60 %-GC segment; 20x coverage of
                  150 bp read pairs from Normal(400, 50) fragments (mate 2
                  reverse complemented), 1 % substitutions, N with p = 1e-4
                  (k=55, m=21).
  batched_sets    256 sets, genome log-uniform on [0.1, 20] Mbp, coverage
                  uniform on [10, 40]x, 150 bp reads with 1 % substitutions.
  served_requests Poisson request stream; genome log-normal (median 2 Mbp,
                  sigma_ln 1.0, clipped to [0.05, 50] Mbp), coverage
                  uniform on [10, 30]x, short or long reads, k in {21, 31, 55}.

``scale`` shrinks genome length (and so the read count) for tests.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hsk_datagen.c")
_LIB = os.path.join(_HERE, "libhsk_datagen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [
        ("seed", C.c_uint64), ("genome_len", C.c_uint64),
        ("gc_start", C.c_uint64), ("gc_len", C.c_uint64), ("gc", C.c_double),
        ("rep_families", C.c_uint32), ("rep_copies", C.c_uint32),
        ("rep_len_min", C.c_uint32), ("rep_len_max", C.c_uint32), ("rep_div_max", C.c_double),
        ("read_model", C.c_int), ("n_reads", C.c_uint64), ("coverage", C.c_double),
        ("read_len", C.c_uint32), ("ln_mu", C.c_double), ("ln_sigma", C.c_double),
        ("len_min", C.c_uint32), ("frag_mean", C.c_double), ("frag_sd", C.c_double),
        ("p_rc", C.c_double), ("p_sub", C.c_double), ("p_ins", C.c_double),
        ("p_del", C.c_double), ("p_n", C.c_double),
    ]


class _Out(C.Structure):
    _fields_ = [("reads", C.POINTER(C.c_uint8)), ("offsets", C.POINTER(C.c_uint64)),
                ("n_reads", C.c_uint64), ("n_bases", C.c_uint64),
                ("cap", C.c_uint64), ("ocap", C.c_uint64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.dg_generate.argtypes = [C.POINTER(_Params), C.POINTER(_Out)]
            lib.dg_generate.restype = C.c_int
            lib.dg_free.argtypes = [C.POINTER(_Out)]
            lib.dg_derive_seed.argtypes = [C.c_uint64, C.c_uint64]
            lib.dg_derive_seed.restype = C.c_uint64
            _lib = lib
    return _lib


@dataclass
class ReadSet:
    reads: np.ndarray     # uint8 ASCII, all reads concatenated
    offsets: np.ndarray   # uint64 [n_reads + 1]
    k: int
    m: int
    lo: int
    hi: int
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_reads(self) -> int:
        return int(self.offsets.size - 1)

    @property
    def n_bases(self) -> int:
        return int(self.reads.size)

    def window_upper_bound(self) -> int:
        """Sum over reads of max(0, len - k + 1): N when no base is invalid."""
        lens = np.diff(self.offsets.astype(np.int64))
        return int(np.maximum(lens - self.k + 1, 0).sum())


def derive_seed(seed: int, i: int) -> int:
    return int(_load().dg_derive_seed(seed, i))


def simulate(**kw) -> tuple[np.ndarray, np.ndarray]:
    """Run the C simulator with the given parameter fields; returns (reads, offsets)."""
    lib = _load()
    p = _Params()
    defaults = dict(p_rc=0.5, ln_mu=0.0, ln_sigma=0.0, frag_mean=400.0, frag_sd=50.0)
    defaults.update(kw)
    for k, v in defaults.items():
        setattr(p, k, v)
    o = _Out()
    if lib.dg_generate(C.byref(p), C.byref(o)) != 0:
        lib.dg_free(C.byref(o))
        raise MemoryError("read simulation ran out of host memory")
    try:
        n, nb = int(o.n_reads), int(o.n_bases)
        reads = np.ctypeslib.as_array(o.reads, shape=(max(nb, 1),))[:nb].copy()
        offsets = np.ctypeslib.as_array(o.offsets, shape=(n + 1,)).copy()
    finally:
        lib.dg_free(C.byref(o))
    return reads, offsets


# ---------------------------------------------------------------------------
# the named workloads
# ---------------------------------------------------------------------------

def tiny(seed: int = 0) -> ReadSet:
    r, o = simulate(seed=seed, genome_len=1_000_000, read_model=0, n_reads=20_000,
                    read_len=150, p_rc=0.5, p_sub=0.01)
    return ReadSet(r, o, k=31, m=17, lo=2, hi=1000, name="tiny-1Mbp-20k-150bp-k31")


def long_read(seed: int = 1, scale: float = 1.0) -> ReadSet:
    g = max(int(50_000_000 * scale), 100_000)
    # log-normal with mean 10 kb and sd 4 kb: sigma^2 = ln(1 + (4/10)^2)
    sigma = math.sqrt(math.log(1 + 0.16))
    mu = math.log(10_000) - sigma * sigma / 2
    fam = 20 if scale >= 0.1 else 4
    r, o = simulate(seed=seed, genome_len=g, rep_families=fam, rep_copies=100,
                    rep_len_min=1000, rep_len_max=min(20_000, g // 4), rep_div_max=0.02,
                    read_model=1, coverage=30.0, ln_mu=mu, ln_sigma=sigma, len_min=1000,
                    p_rc=0.5, p_sub=0.005, p_ins=0.0005, p_del=0.0005)
    return ReadSet(r, o, k=31, m=17, lo=2, hi=8,
                   name=f"long-read-{g / 1e6:g}Mbp-30x-10kb-k31", meta=dict(genome=g))


def short_read(seed: int = 2, scale: float = 1.0) -> ReadSet:
    g = max(int(100_000_000 * scale), 100_000)
    r, o = simulate(seed=seed, genome_len=g, gc_start=g // 5, gc_len=g // 5, gc=0.6,
                    read_model=2, coverage=20.0, read_len=150, frag_mean=400.0, frag_sd=50.0,
                    p_sub=0.01, p_n=1e-4)
    return ReadSet(r, o, k=55, m=21, lo=2, hi=500,
                   name=f"short-read-{g / 1e6:g}Mbp-20x-2x150bp-k55", meta=dict(genome=g))


def batched_set_params(seed: int = 3, n_sets: int = 256, scale: float = 1.0):
    """Per-set (seed, genome length, coverage) of the batched workload."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_sets):
        g = math.exp(rng.uniform(math.log(0.1e6), math.log(20e6))) * scale
        cov = rng.uniform(10, 40)
        out.append((derive_seed(seed, i), max(int(g), 2000), float(cov)))
    return out


def batched_set(seed: int, genome: int, coverage: float) -> ReadSet:
    r, o = simulate(seed=seed, genome_len=genome, read_model=0, coverage=coverage,
                    read_len=150, p_rc=0.5, p_sub=0.01)
    return ReadSet(r, o, k=31, m=17, lo=2, hi=1000, name=f"set-{genome}")


def served_request_params(seed: int = 4, n: int = 2000, scale: float = 1.0):
    """Per-request (seed, genome, coverage, long?, k, m)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        g = min(max(math.exp(math.log(2e6) + rng.normal()), 0.05e6), 50e6) * scale
        cov = rng.uniform(10, 30)
        long_reads = bool(rng.integers(0, 2))
        k = int(rng.choice([21, 31, 55]))
        m = {21: 11, 31: 17, 55: 21}[k]
        out.append((derive_seed(seed, i), max(int(g), 20_000), float(cov), long_reads, k, m))
    return out


def served_request(seed: int, genome: int, coverage: float, long_reads: bool, k: int,
                   m: int) -> ReadSet:
    if long_reads:
        sigma = math.sqrt(math.log(1 + 0.16))
        mu = math.log(10_000) - sigma * sigma / 2
        r, o = simulate(seed=seed, genome_len=genome, read_model=1, coverage=coverage,
                        ln_mu=mu, ln_sigma=sigma, len_min=1000, p_rc=0.5, p_sub=0.005,
                        p_ins=0.0005, p_del=0.0005)
    else:
        r, o = simulate(seed=seed, genome_len=genome, read_model=0, coverage=coverage,
                        read_len=150, p_rc=0.5, p_sub=0.01)
    return ReadSet(r, o, k=k, m=m, lo=2, hi=1000, name=f"req-{genome}-k{k}")


def random_reads(seed: int, n_reads: int, min_len: int, max_len: int, p_invalid: float = 0.0,
                 alphabet: bytes = b"ACGT", invalid: bytes = b"N") -> tuple[np.ndarray, np.ndarray]:
    """Small i.i.d. reads for edge cases (numpy PCG64; not genome-shaped)."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(min_len, max_len + 1, size=n_reads)
    offsets = np.zeros(n_reads + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(lens)
    total = int(offsets[-1])
    a = np.frombuffer(alphabet, dtype=np.uint8)
    reads = a[rng.integers(0, a.size, size=total)]
    if p_invalid > 0 and total:
        bad = rng.random(total) < p_invalid
        iv = np.frombuffer(invalid, dtype=np.uint8)
        reads = reads.copy()
        reads[bad] = iv[rng.integers(0, iv.size, size=int(bad.sum()))]
    return reads.astype(np.uint8), offsets
