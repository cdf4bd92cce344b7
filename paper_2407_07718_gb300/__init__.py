"""Python binding of ``libhsk.so``, a GB300 (sm_103a) sorting-based k-mer
counter (HySortK, arXiv 2407.07718).

Argument marshalling only: every step of the counting pipeline runs in the
library's CUDA kernels.  There is no CPU fallback; if the library cannot be
loaded (or built in-tree with nvcc) every entry point raises.  PyTorch is used
only to hold device memory and streams (``torch.Tensor`` inputs of the
device-side entry points).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass, field

import numpy as np

from . import _build

__all__ = ["load", "Context", "CountResult", "HskError", "build"]

HSK_OK, HSK_EINVAL, HSK_ENOMEM, HSK_ECUDA, HSK_ETIMEOUT, HSK_ECANCELED, HSK_EOVERFLOW, HSK_ENOTFOUND = \
    0, -1, -2, -3, -4, -5, -6, -7
_NAMES = {HSK_EINVAL: "HSK_EINVAL", HSK_ENOMEM: "HSK_ENOMEM", HSK_ECUDA: "HSK_ECUDA",
          HSK_ETIMEOUT: "HSK_ETIMEOUT", HSK_ECANCELED: "HSK_ECANCELED",
          HSK_EOVERFLOW: "HSK_EOVERFLOW", HSK_ENOTFOUND: "HSK_ENOTFOUND"}
DEFAULT_SEED = 0x9E3779B97F4A7C15

_lock = threading.Lock()
_lib = None


class HskError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class _Config(C.Structure):
    _fields_ = [("device", C.c_int), ("hbm_budget", C.c_uint64), ("hist_len", C.c_uint32),
                ("n_buckets", C.c_uint32), ("radix_bits", C.c_uint32),
                ("max_chunk_kmers", C.c_uint32), ("seed", C.c_uint64), ("autotune", C.c_int),
                ("local_sort", C.c_int), ("tune_cache", C.c_char_p), ("minimizer_order", C.c_int)]


class _TuneResult(C.Structure):
    _fields_ = [("group_div", C.c_uint32), ("plain_bucket_shift", C.c_uint32), ("pack_bases", C.c_uint64),
                ("pack_small", C.c_uint64), ("slots", C.c_int), ("trials", C.c_int), ("first_s", C.c_double),
                ("best_s", C.c_double)]


class _Result(C.Structure):
    _fields_ = [("n_pairs", C.c_uint64), ("kmers", C.c_void_p), ("counts", C.c_void_p),
                ("hist", C.c_void_p), ("hist_len", C.c_uint32), ("key_words", C.c_int),
                ("n_windows", C.c_uint64), ("n_distinct", C.c_uint64), ("max_count", C.c_uint32),
                ("n_chunks", C.c_uint32), ("n_supermers", C.c_uint64), ("device_ms", C.c_double)]


class _ExtResult(C.Structure):
    _fields_ = [("counts", _Result), ("n_occ", C.c_uint64), ("occ_offsets", C.c_void_p), ("occ_read", C.c_void_p),
                ("occ_pos", C.c_void_p)]


class _Job(C.Structure):
    _fields_ = [("reads", C.c_void_p), ("offsets", C.c_void_p), ("n_reads", C.c_uint64),
                ("k", C.c_int), ("m", C.c_int), ("lo", C.c_uint32), ("hi", C.c_uint32)]


def build(force: bool = False) -> str:
    return _build.build(force=force)


def load():
    """Load libhsk.so (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        lib = C.CDLL(path)
        P, u64, u32, i32, d = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int, C.c_double
        sigs = {
            "hsk_config_default": ([C.POINTER(_Config)], i32),
            "hsk_create": ([C.POINTER(P), C.POINTER(_Config)], i32),
            "hsk_destroy": ([P], None),
            "hsk_last_error": ([P], C.c_char_p),
            "hsk_count": ([P, P, P, u64, i32, i32, u32, u32, C.POINTER(_Result)], i32),
            "hsk_count_device": ([P, P, P, u64, u64, i32, i32, u32, u32, P, C.POINTER(_Result)], i32),
            "hsk_result_copy": ([P, C.POINTER(_Result), P, P, P, i32, P], i32),
            "hsk_count_batch": ([P, C.POINTER(_Job), u32, C.POINTER(_Result)], i32),
            "hsk_autotune": ([P, C.POINTER(_Job), u32, i32, C.POINTER(_TuneResult)], i32),
            "hsk_tune_current": ([P, C.POINTER(_TuneResult)], i32),
            "hsk_host_pin": ([P, u64], i32),
            "hsk_count_ext": ([P, P, P, u64, i32, i32, u32, u32, C.POINTER(_ExtResult)], i32),
            "hsk_stage_ext_encode": ([P, P, P, u64, P, u64, P, C.POINTER(u64), P], i32),
            "hsk_stage_ext_decode": ([P, P, u64, P, u64, P, P, P], i32),
            "hsk_host_unpin": ([P], i32),
            "hsk_tune_set": ([P, C.POINTER(_TuneResult)], i32),
            "hsk_submit": ([P, C.POINTER(_Job), C.POINTER(u64)], i32),
            "hsk_poll": ([P, u64, C.POINTER(i32)], i32),
            "hsk_wait": ([P, u64, C.POINTER(_Result)], i32),
            "hsk_cancel": ([P, u64], i32),
            "hsk_release": ([P, u64], i32),
            "hsk_ticket_times": ([P, u64, C.POINTER(d), C.POINTER(d)], i32),
            "hsk_stage_encode": ([P, P, u64, P, u64, P, P, P, P], i32),
            "hsk_stage_windows": ([P, P, P, u64, u64, i32, i32, P, P, P, P], i32),
            "hsk_stage_supermers": ([P, P, P, u64, u64, i32, i32, u32, P, P, C.POINTER(P),
                                     C.POINTER(u64), C.POINTER(i32), C.POINTER(i32), P], i32),
            "hsk_stage_sort": ([P, P, u64, i32, i32, P], i32),
            "hsk_stage_rle": ([P, P, u64, i32, u32, u32, P, C.POINTER(_Result)], i32),
            "hsk_stage_order": ([P, P, P, u64, i32, i32, P], i32),
            "hsk_debug_fail_alloc_after": ([P, i32], i32),
            "hsk_debug_allocated": ([P], u64),
            "hsk_debug_last_overflow": ([P], u64),
            "hsk_debug_wait_timeout": ([P, u32], C.c_int),
            "hsk_debug_host_pool_check": ([], C.c_int),
            "hsk_profile_enable": ([P, i32], i32),
            "hsk_profile_read": ([P, C.POINTER(d), C.POINTER(u64), i32], i32),
            "hsk_launch_count": ([], u64),
            "hsk_sort_keys_noalloc": ([P, u64, i32, i32, P], i32),
            "hsk_debug_pack_stats": ([P, C.POINTER(u64), C.POINTER(u64), C.POINTER(u64)], i32),
            "hsk_debug_pack_failure": ([P, C.POINTER(u64)], C.c_char_p),
        }
        for name, (args, res) in sigs.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray)):
        a = np.frombuffer(a, dtype=np.uint8)
    return np.ascontiguousarray(a, dtype=np.uint8)


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint64)


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data) if a.size else C.c_void_p(0)


def _tptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() else C.c_void_p(0)


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


NOALLOC_MAX_KEYS = {1: 1 << 20, 2: 1 << 19}
EXT_CHUNK = 1024  # items per independently decodable chunk of the extension codec (HSK_EXT_CHUNK)


def pinned_empty(nbytes: int) -> np.ndarray:
    """A page-aligned host byte buffer of whole pages, pinned with
    hsk_host_pin (exact size, no rounding).  Call host_unpin(buf) before the
    buffer is dropped."""
    import mmap
    size = max(mmap.PAGESIZE, (int(nbytes) + mmap.PAGESIZE - 1) // mmap.PAGESIZE * mmap.PAGESIZE)
    buf = np.frombuffer(mmap.mmap(-1, size), dtype=np.uint8)
    rc = load().hsk_host_pin(C.c_void_p(buf.ctypes.data), size)
    if rc != HSK_OK:
        raise HskError(rc, f"hsk_host_pin of {size} bytes failed")
    return buf


def host_unpin(buf: np.ndarray):
    rc = load().hsk_host_unpin(C.c_void_p(buf.ctypes.data))
    if rc != HSK_OK:
        raise HskError(rc, "hsk_host_unpin failed")


def sort_keys_noalloc(keys_t, n: int, key_words: int, key_bits: int, stream=None) -> int:
    """Sort n keys of a device tensor in place without any device allocation
    (for callers that cannot allocate; see hsk_sort_keys_noalloc in
    include/hsk_stages.h).  Returns the library's status code."""
    return int(load().hsk_sort_keys_noalloc(_tptr(keys_t), n, key_words, key_bits, _stream_ptr(stream)))


@dataclass
class CountResult:
    kmers: np.ndarray        # (n,) uint64 for k <= 32; (n, 2) uint64 {lo, hi} otherwise
    counts: np.ndarray       # (n,) uint32
    hist: np.ndarray         # (hist_len,) uint64
    n_windows: int
    n_distinct: int
    max_count: int
    key_words: int
    n_chunks: int = 1
    n_supermers: int = 0
    device_ms: float = 0.0
    extra: dict = field(default_factory=dict)


def _summary(r: _Result) -> CountResult:
    """Scalars of a result only (its arrays stay in library memory, unread)."""
    return CountResult(None, None, None, int(r.n_windows), int(r.n_distinct), int(r.max_count),
                       int(r.key_words), int(r.n_chunks), int(r.n_supermers), float(r.device_ms),
                       extra={"n_pairs": int(r.n_pairs)})


def _host_result(r: _Result, copy=True) -> CountResult:
    """copy=True: numpy copies of the arrays; False: scalars only; "view":
    numpy views of the library's host arrays, valid only while the result is
    (until the next call on the context, or the ticket's release)."""
    if copy is False:
        return _summary(r)
    take = (lambda a: a) if copy == "view" else (lambda a: a.copy())
    n, kw = int(r.n_pairs), int(r.key_words)
    if n:
        kmers = take(np.ctypeslib.as_array(C.cast(r.kmers, C.POINTER(C.c_uint64)), shape=(n * kw,)))
        counts = take(np.ctypeslib.as_array(C.cast(r.counts, C.POINTER(C.c_uint32)), shape=(n,)))
    else:
        kmers = np.zeros(0, np.uint64)
        counts = np.zeros(0, np.uint32)
    if kw == 2:
        kmers = kmers.reshape(n, 2)
    hist = take(np.ctypeslib.as_array(C.cast(r.hist, C.POINTER(C.c_uint64)), shape=(int(r.hist_len),)))
    return CountResult(kmers, counts, hist, int(r.n_windows), int(r.n_distinct), int(r.max_count), kw,
                       int(r.n_chunks), int(r.n_supermers), float(r.device_ms))


class Context:
    """One library context (device arena, stream, serving slots) on one GPU."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, hist_len: int = 65536, n_buckets: int = 0,
                 max_chunk_kmers: int = 0, seed: int = DEFAULT_SEED, autotune: bool = True,
                 local_sort: bool = True, tune_cache: str | None = None, lexical_minimizers: bool = False):
        self.lib = load()
        cfg = _Config()
        self.lib.hsk_config_default(C.byref(cfg))
        cfg.device, cfg.hbm_budget, cfg.hist_len = device, hbm_budget, hist_len
        cfg.n_buckets, cfg.max_chunk_kmers, cfg.seed, cfg.autotune = n_buckets, max_chunk_kmers, seed, int(autotune)
        cfg.local_sort = int(local_sort)
        cfg.tune_cache = tune_cache.encode() if tune_cache else None
        cfg.minimizer_order = 1 if lexical_minimizers else 0
        h = C.c_void_p()
        rc = self.lib.hsk_create(C.byref(h), C.byref(cfg))
        if rc != HSK_OK:
            raise HskError(rc, "hsk_create failed (no usable CUDA device?)")
        self.h = h
        self._pending = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.hsk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc: int):
        if rc != HSK_OK:
            raise HskError(rc, self.lib.hsk_last_error(self.h).decode())

    # ---- plain path -----------------------------------------------------------
    def count(self, reads, offsets, k: int, m: int, lo: int, hi: int, copy: bool = True) -> CountResult:
        """Host arrays in, host arrays out (copies inside the call).  With
        copy=False only the scalars are returned; the arrays stay in the
        context's host memory until its next call."""
        reads, offsets = _u8(reads), _u64(offsets)
        r = _Result()
        self._check(self.lib.hsk_count(self.h, _ptr(reads), _ptr(offsets), offsets.size - 1, k, m,
                                       lo, hi, C.byref(r)))
        return _host_result(r, copy)

    def count_ext(self, reads, offsets, k: int, m: int, lo: int, hi: int):
        """hsk_count_ext: (CountResult, occ_offsets, occ_read, occ_pos) as numpy copies."""
        reads, offsets = _u8(reads), _u64(offsets)
        r = _ExtResult()
        self._check(self.lib.hsk_count_ext(self.h, _ptr(reads), _ptr(offsets), offsets.size - 1, k, m, lo, hi,
                                           C.byref(r)))
        res = _host_result(r.counts, True)
        np_, no = int(r.counts.n_pairs), int(r.n_occ)
        off = np.ctypeslib.as_array(C.cast(r.occ_offsets, C.POINTER(C.c_uint64)), shape=(np_ + 1,)).copy()
        if no:
            rd = np.ctypeslib.as_array(C.cast(r.occ_read, C.POINTER(C.c_uint32)), shape=(no,)).copy()
            ps = np.ctypeslib.as_array(C.cast(r.occ_pos, C.POINTER(C.c_uint32)), shape=(no,)).copy()
        else:
            rd, ps = np.zeros(0, np.uint32), np.zeros(0, np.uint32)
        return res, off, rd, ps

    def stage_ext_encode(self, read_t, pos_t, out_t, chunk_off_t, stream=None) -> int:
        """Encode n = read_t.numel() items; returns the byte length."""
        nb = C.c_uint64()
        self._check(self.lib.hsk_stage_ext_encode(self.h, _tptr(read_t), _tptr(pos_t), int(read_t.numel()),
                                                  _tptr(out_t), int(out_t.numel()), _tptr(chunk_off_t),
                                                  C.byref(nb), _stream_ptr(stream)))
        return nb.value

    def stage_ext_decode(self, in_t, n_bytes: int, chunk_off_t, n: int, read_t, pos_t, stream=None):
        self._check(self.lib.hsk_stage_ext_decode(self.h, _tptr(in_t), n_bytes, _tptr(chunk_off_t), n,
                                                  _tptr(read_t), _tptr(pos_t), _stream_ptr(stream)))

    def count_device(self, reads_t, offsets_t, k: int, m: int, lo: int, hi: int, stream=None,
                     n_bases: int | None = None) -> _Result:
        """Device tensors in (uint8 reads, int64/uint64 offsets); returns the raw
        result whose arrays are context-owned device memory."""
        r = _Result()
        nb = int(reads_t.numel()) if n_bases is None else n_bases
        self._check(self.lib.hsk_count_device(self.h, _tptr(reads_t), _tptr(offsets_t),
                                              int(offsets_t.numel()) - 1, nb, k, m, lo, hi,
                                              _stream_ptr(stream), C.byref(r)))
        return r

    def result_to_host(self, r: _Result) -> CountResult:
        n, kw = int(r.n_pairs), int(r.key_words)
        kmers = np.zeros(max(n * kw, 1), np.uint64)
        counts = np.zeros(max(n, 1), np.uint32)
        hist = np.zeros(int(r.hist_len), np.uint64)
        self._check(self.lib.hsk_result_copy(self.h, C.byref(r), _ptr(kmers), _ptr(counts), _ptr(hist),
                                             0, C.c_void_p(0)))
        kmers, counts = kmers[: n * kw], counts[:n]
        if kw == 2:
            kmers = kmers.reshape(n, 2)
        return CountResult(kmers, counts, hist, int(r.n_windows), int(r.n_distinct), int(r.max_count), kw,
                           int(r.n_chunks), int(r.n_supermers), float(r.device_ms))

    # ---- batched form ---------------------------------------------------------
    @staticmethod
    def _jobs(jobs):
        keep, arr = [], (_Job * max(len(jobs), 1))()
        for i, (reads, offsets, k, m, lo, hi) in enumerate(jobs):
            reads, offsets = _u8(reads), _u64(offsets)
            keep.append((reads, offsets))
            arr[i] = _Job(reads.ctypes.data if reads.size else None, offsets.ctypes.data,
                          offsets.size - 1, k, m, lo, hi)
        return keep, arr

    def count_batch(self, jobs, copy: bool = True) -> list[CountResult]:
        """jobs: sequence of (reads, offsets, k, m, lo, hi) host arrays."""
        keep, arr = self._jobs(jobs)
        outs = (_Result * max(len(jobs), 1))()
        self._check(self.lib.hsk_count_batch(self.h, arr, len(jobs), outs))
        return [_host_result(outs[i], copy) for i in range(len(jobs))]

    def autotune(self, jobs, max_trials: int = 16) -> dict:
        """Tune the batched/served parameters on sample jobs (see hsk_autotune)."""
        keep, arr = self._jobs(jobs)
        r = _TuneResult()
        self._check(self.lib.hsk_autotune(self.h, arr, len(jobs), max_trials, C.byref(r)))
        return {f: getattr(r, f) for f, _ in _TuneResult._fields_}

    def tune_set(self, **params):
        """Put batched/served parameters in force (missing ones keep their value)."""
        cur = self.tune_current()
        cur.update(params)
        r = _TuneResult(**{f: cur[f] for f, _ in _TuneResult._fields_})
        self._check(self.lib.hsk_tune_set(self.h, C.byref(r)))

    def tune_current(self) -> dict:
        """The batched/served parameters in force on this context."""
        r = _TuneResult()
        self._check(self.lib.hsk_tune_current(self.h, C.byref(r)))
        return {f: getattr(r, f) for f, _ in _TuneResult._fields_}

    # ---- served form ----------------------------------------------------------
    def submit(self, reads, offsets, k: int, m: int, lo: int, hi: int) -> int:
        reads, offsets = _u8(reads), _u64(offsets)
        job = _Job(reads.ctypes.data if reads.size else None, offsets.ctypes.data, offsets.size - 1,
                   k, m, lo, hi)
        t = C.c_uint64()
        self._check(self.lib.hsk_submit(self.h, C.byref(job), C.byref(t)))
        self._pending[t.value] = (reads, offsets)  # inputs stay alive until release
        return t.value

    def poll(self, ticket: int) -> bool:
        d = C.c_int()
        self._check(self.lib.hsk_poll(self.h, ticket, C.byref(d)))
        return bool(d.value)

    def wait(self, ticket: int, copy: bool = True) -> CountResult:
        r = _Result()
        self._check(self.lib.hsk_wait(self.h, ticket, C.byref(r)))
        return _host_result(r, copy)

    def times(self, ticket: int) -> tuple[float, float]:
        q, x = C.c_double(), C.c_double()
        self._check(self.lib.hsk_ticket_times(self.h, ticket, C.byref(q), C.byref(x)))
        return q.value, x.value

    def cancel(self, ticket: int):
        self._check(self.lib.hsk_cancel(self.h, ticket))

    def release(self, ticket: int):
        self._check(self.lib.hsk_release(self.h, ticket))
        self._pending.pop(ticket, None)

    # ---- stages (device tensors) ---------------------------------------------
    def stage_encode(self, reads_t, offsets_t, packed_t, invalid_t, start_t, stream=None):
        self._check(self.lib.hsk_stage_encode(self.h, _tptr(reads_t), int(reads_t.numel()), _tptr(offsets_t),
                                              int(offsets_t.numel()) - 1, _tptr(packed_t), _tptr(invalid_t),
                                              _tptr(start_t), _stream_ptr(stream)))

    def stage_windows(self, reads_t, offsets_t, k, m, valid_t, key_t, minhash_t, stream=None):
        self._check(self.lib.hsk_stage_windows(self.h, _tptr(reads_t), _tptr(offsets_t),
                                               int(offsets_t.numel()) - 1, int(reads_t.numel()), k, m,
                                               _tptr(valid_t), _tptr(key_t), _tptr(minhash_t),
                                               _stream_ptr(stream)))

    def stage_supermers(self, reads_t, offsets_t, k, m, n_buckets, bucket_kmers_t, bucket_rec_t, stream=None):
        """Returns (device pointer of records, n_records, record_words, max_kmers)."""
        recp, nrec, rw, nmax = C.c_void_p(), C.c_uint64(), C.c_int(), C.c_int()
        self._check(self.lib.hsk_stage_supermers(self.h, _tptr(reads_t), _tptr(offsets_t),
                                                 int(offsets_t.numel()) - 1, int(reads_t.numel()), k, m,
                                                 n_buckets, _tptr(bucket_kmers_t), _tptr(bucket_rec_t),
                                                 C.byref(recp), C.byref(nrec), C.byref(rw), C.byref(nmax),
                                                 _stream_ptr(stream)))
        return recp.value, nrec.value, rw.value, nmax.value

    def copy_device_words(self, dev_ptr: int, n_words: int) -> np.ndarray:
        """Copy n uint64 words at a context-owned device address to the host."""
        out = np.zeros(max(n_words, 1), np.uint64)
        r = _Result()
        r.n_pairs, r.key_words, r.kmers, r.hist_len = n_words, 1, dev_ptr, 0
        self._check(self.lib.hsk_result_copy(self.h, C.byref(r), _ptr(out), None, None, 0, C.c_void_p(0)))
        return out[:n_words]

    def stage_sort(self, keys_t, n: int, key_words: int, key_bits: int, stream=None):
        self._check(self.lib.hsk_stage_sort(self.h, _tptr(keys_t), n, key_words, key_bits, _stream_ptr(stream)))

    def stage_rle(self, sorted_t, n: int, key_words: int, lo: int, hi: int, stream=None) -> CountResult:
        r = _Result()
        self._check(self.lib.hsk_stage_rle(self.h, _tptr(sorted_t), n, key_words, lo, hi,
                                           _stream_ptr(stream), C.byref(r)))
        return self.result_to_host(r)

    def stage_order(self, keys_t, counts_t, n: int, key_words: int, key_bits: int, stream=None):
        self._check(self.lib.hsk_stage_order(self.h, _tptr(keys_t), _tptr(counts_t), n, key_words, key_bits,
                                             _stream_ptr(stream)))

    STAGES = ("S1 encode", "S2 k-mers+minimizers+count", "S3 scatter", "S4 expand+hist", "S4 radix passes",
              "S5 rle+filter+hist", "S6 order")

    def profile(self, on: bool = True):
        self._check(self.lib.hsk_profile_enable(self.h, int(on)))

    def profile_read(self, reset: bool = True) -> tuple[list[float], int]:
        ms = (C.c_double * 7)()
        passes = C.c_uint64()
        self._check(self.lib.hsk_profile_read(self.h, ms, C.byref(passes), int(reset)))
        return list(ms), int(passes.value)

    @staticmethod
    def launch_count() -> int:
        return int(load().hsk_launch_count())

    def fail_alloc_after(self, n: int):
        self._check(self.lib.hsk_debug_fail_alloc_after(self.h, n))

    def allocated(self) -> int:
        return int(self.lib.hsk_debug_allocated(self.h))

    def wait_timeout(self, spin_limit: int) -> int:
        """Run a bounded device wait on a flag nothing sets; returns the code
        (HSK_ETIMEOUT expected).  See hsk_debug_wait_timeout."""
        return int(self.lib.hsk_debug_wait_timeout(self.h, spin_limit))

    def pack_stats(self) -> dict:
        """Packed passes of the batched/served forms so far: passes, jobs they
        held, and jobs among those counted again alone."""
        a, b, c, f = C.c_uint64(), C.c_uint64(), C.c_uint64(), C.c_uint64()
        self._check(self.lib.hsk_debug_pack_stats(self.h, C.byref(a), C.byref(b), C.byref(c)))
        msg = self.lib.hsk_debug_pack_failure(self.h, C.byref(f)).decode()
        return {"passes": a.value, "sets": b.value, "alone": c.value, "failed_passes": f.value,
                "last_failure": msg}

    def last_overflow(self) -> int:
        """Keys of the last call that went through the global radix passes
        because their sub-segment did not fit the on-chip sort."""
        return int(self.lib.hsk_debug_last_overflow(self.h))
