#!/usr/bin/env python3
"""Write tests/golden/fullsize_digests.json: the oracle's exact result for every
full-size job of the long-read, short-read, batched (256 sets) and served
(2,000 requests) workloads, as digests the GPU tests compare against.

Only ``oracle`` (the plain CPU counter) and ``datagen`` (the seeded read
simulator) are used; nothing here touches the CUDA library.  Each job runs in
its own worker process (single-threaded oracle instances side by side, started
with ``spawn``), under a host-memory budget: the oracle holds 16 bytes per
window plus the reads.

Per job the file stores
  reads_sha256  -- SHA-256 of the ASCII reads followed by the offsets as
                   little-endian uint64: a run that simulates different reads
                   (a drift of the simulator between machines) fails as
                   datagen, not as counting;
  pairs_sha256  -- SHA-256 of the kept k-mers (n_pairs * key_words
                   little-endian uint64 words, ascending) followed by their
                   counts (little-endian uint32);
  hist_sha256   -- SHA-256 of the 65,536-bin histogram (little-endian uint64);
  hist_head     -- bins 0..63 of the histogram, for a readable diff;
  n_windows, n_distinct, n_pairs, max_count.

Usage: python tests/golden/make_fullsize_digests.py [--jobs long_read,short_read,batched,served]
       [--workers N] [--mem-gb G] [--limit N]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "fullsize_digests.json")
HIST_LEN = 65536


def job_list(which):
    sys.path.insert(0, ROOT)
    import datagen
    jobs = []
    if "long_read" in which:
        jobs.append(("long_read", ("long_read", ()), 1_500_000_000))
    if "short_read" in which:
        jobs.append(("short_read", ("short_read", ()), 2_000_000_000))
    if "batched" in which:
        for i, p in enumerate(datagen.batched_set_params(n_sets=256)):
            jobs.append((f"batched/{i}", ("batched_set", p), int(p[1] * p[2])))
    if "served" in which:
        for i, p in enumerate(datagen.served_request_params(n=2000)):
            jobs.append((f"served/{i}", ("served_request", p), int(p[1] * p[2])))
    return jobs


def digest_of_reads(reads, offsets):
    import numpy as np
    h = hashlib.sha256()
    h.update(memoryview(np.ascontiguousarray(reads, dtype=np.uint8)))
    h.update(memoryview(np.ascontiguousarray(offsets, dtype="<u8")))
    return h.hexdigest()


def run_job(spec):
    name, (fn, args) = spec
    sys.path.insert(0, ROOT)
    import numpy as np
    import datagen
    import oracle
    t0 = time.time()
    rs = getattr(datagen, fn)(*args)
    reads_sha = digest_of_reads(rs.reads, rs.offsets)
    r = oracle.count(rs.reads, rs.offsets, rs.k, rs.lo, rs.hi, hist_len=HIST_LEN)
    h = hashlib.sha256()
    h.update(memoryview(np.ascontiguousarray(r.kmers, dtype="<u8").reshape(-1)))
    h.update(memoryview(np.ascontiguousarray(r.counts, dtype="<u4")))
    return name, {
        "k": rs.k, "m": rs.m, "lo": rs.lo, "hi": rs.hi,
        "n_reads": rs.n_reads, "n_bases": rs.n_bases, "reads_sha256": reads_sha,
        "n_windows": r.n_windows, "n_distinct": r.n_distinct, "n_pairs": int(r.counts.size),
        "max_count": r.max_count, "pairs_sha256": h.hexdigest(),
        "hist_sha256": hashlib.sha256(memoryview(np.ascontiguousarray(r.hist, dtype="<u8"))).hexdigest(),
        "hist_head": [int(x) for x in r.hist[:64]],
        "oracle_s": round(time.time() - t0, 1),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", default="long_read,short_read,batched,served")
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--mem-gb", type=float, default=48.0)
    ap.add_argument("--limit", type=int, default=0)
    args = ap.parse_args()
    which = set(args.jobs.split(","))
    jobs = job_list(which)
    if args.limit:
        jobs = jobs[: args.limit]
    done = json.load(open(OUT)) if os.path.exists(OUT) else {"jobs": {}}
    done.setdefault("jobs", {})
    todo = [j for j in jobs if j[0] not in done["jobs"]]
    todo.sort(key=lambda j: -j[2])  # largest first
    budget = args.mem_gb * 1e9
    est = lambda bases: bases * 19.0 + 0.3e9  # reads + offsets + 16 B/window keys + output
    ctx = mp.get_context("spawn")
    t_start = time.time()
    with ctx.Pool(args.workers, maxtasksperchild=1) as pool:
        running = {}
        in_use = 0.0
        pending = list(todo)
        while pending or running:
            i = 0
            while i < len(pending) and len(running) < args.workers:
                name, spec, bases = pending[i]
                need = est(bases)
                if in_use + need <= budget or not running:
                    running[name] = (pool.apply_async(run_job, ((name, spec),)), need)
                    in_use += need
                    pending.pop(i)
                else:
                    i += 1
            time.sleep(0.5)
            for name in [n for n, (a, _) in running.items() if a.ready()]:
                a, need = running.pop(name)
                in_use -= need
                nm, d = a.get()
                done["jobs"][nm] = d
                print(f"[{time.time() - t_start:7.0f}s] {nm}: {d['n_windows']} windows, {d['n_pairs']} pairs, "
                      f"{d['oracle_s']} s", flush=True)
                tmp = OUT + ".tmp"
                done["_source"] = ("Written by tests/golden/make_fullsize_digests.py from oracle.count (the plain "
                                   "CPU counter of Sec. 2.1 / Sec. 3.1) on the datagen workloads; see that "
                                   "script's docstring for the fields.")
                done["hist_len"] = HIST_LEN
                json.dump(done, open(tmp, "w"), indent=0, sort_keys=True)
                os.replace(tmp, OUT)


if __name__ == "__main__":
    main()
