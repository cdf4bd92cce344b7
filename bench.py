#!/usr/bin/env python3
"""Benchmark: canonical k-mers counted per second on one GB300 (plain path).

One step = the whole hot path (S1 encode, S2 canonical k-mers + minimizers,
S3 supermer bucketing, S4 radix sort, S5 run-length count / filter /
histogram, S6 output order when chunked) over one synthetic read set that is
already resident in device memory.  Default workload: the long-read set
(50 Mbp genome with 2,000 repeat copies, 30x log-normal 10 kb reads, 0.5 %
substitutions + 0.1 % indels, k=31, m=17, filter [2, 8]; about 1.5 G windows).
The inputs (1.5 GB of reads) are larger than L2, so no flush is needed between
steps.

Printed JSON line: value = k-mers counted / s over all ranks; e2e = the same
through hsk_count() with pinned host buffers (copies inside the timed region);
roofline = the dominant kernel (the on-chip sub-segment sort, bound by
instruction issue; with local_sort off, the onesweep radix pass against the
measured HBM copy bandwidth); cpu_baseline = the CPU oracle on a bounded sample.  On one
GPU the line also carries "batched" (256 independent read sets through
hsk_count_batch against the same sets run one by one through hsk_count) and
"served" (a Poisson request stream through hsk_submit/hsk_wait: throughput
and p50/p99/p99.9 latency, against the plain per-job path).

--impl reference times the CPU oracle (single thread) on a bounded sample of
the same workload.  Under torchrun every rank runs an independent replica
(the path needs no collective); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "k-mers counted/s at k=31 on 1 GB300 (plain vs batched/served); p50/p99 job latency"
UNIT = "k-mers/s"

# Per-key counters of the dominant kernel from one ncu capture, keyed by the
# workload and the SHA-256 (first 16 hex digits) of the kernel's source code
# (comments stripped) at capture time; used only while that code is unchanged.
#   inst  : warp instructions issued per key (all on-chip tiers)
#   dram  : DRAM bytes read + written per key (all tiers)
#   smem_wavefronts : shared-memory wavefronts per key (all tiers); an SM's
#           shared-memory pipe processes at most one wavefront per cycle
# The commands that produced them are in profiles/.
NCU_PER_KEY = {
    # long-read workload, k=31: k_local_sort tiers 0, 1 and 2 (the heavy-hitter kernel does not
    # run at this scale), smsp__inst_executed.sum, DRAM bytes and shared-memory wavefronts
    # (l1tex__data_pipe_lsu_wavefronts_mem_shared.sum) from the 0.1-scale case (149.6 M keys)
    ("long_read", "068cb6efb5eb6836"): {"inst": 10.1611, "dram": 8.3749, "smem_wavefronts": 2.2143},
}
# Warp schedulers per SM (Blackwell): each issues at most one warp instruction
# per cycle; the issue peak is SMs (queried from the device) x this x the SM
# clock sampled during the run.
SCHEDULERS_PER_SM = 4


def source_sha(path: str) -> str:
    """SHA-256 (16 hex digits) of a CUDA source's code: comments and
    whitespace-only differences do not change it, any code change does."""
    import re
    text = open(path, encoding="utf-8").read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)   # block comments
    text = re.sub(r"//[^\n]*", "", text)                  # line comments
    text = "\n".join(" ".join(line.split()) for line in text.splitlines() if line.strip())
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def host_cpu() -> dict:
    """Core count (nproc) and CPU model of the host running the oracle."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.startswith("Model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"host_cores": os.cpu_count(), "cpu_model": model or "unknown"}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def make_workload(name: str, scale: float):
    import datagen
    if name == "long_read":
        rs = datagen.long_read(scale=scale)
        desc = "long-read: 50 Mbp genome + 2,000 repeat copies (1-20 kb, 0-2% div), 30x log-normal 10 kb reads, 0.5% sub + 0.1% indel, k=31 m=17, filter [2,8]"
    elif name == "short_read":
        rs = datagen.short_read(scale=scale)
        desc = "short-read: 100 Mbp genome (20 Mbp at 60% GC), 20x 2x150 bp pairs, 1% sub, N p=1e-4, k=55 m=21, filter [2,500]"
    elif name == "tiny":
        rs = datagen.tiny()
        desc = "tiny: 1 Mbp genome, 20,000 x 150 bp reads, 1% sub, k=31 m=17, filter [2,1000]"
    else:
        raise SystemExit(f"unknown workload {name}")
    if scale != 1.0:
        desc += f" (scale {scale})"
    return rs, desc


def e2e_parts(ctx, rs, pin_reads, pin_offs, e2e: dict, dev) -> dict:
    """What one end-to-end call is made of: the device stages inside it (CUDA
    events on its stream; S1/S2 overlap the input copy, so they include any
    wait for it), the same host->device and device->host copies timed alone,
    and the rest of the wall time (host work and synchronisation)."""
    import torch
    ctx.profile(True)
    ctx.profile_read(reset=True)
    t0 = time.perf_counter()
    ctx.count(pin_reads, pin_offs, rs.k, rs.m, rs.lo, rs.hi, copy=False)
    wall = (time.perf_counter() - t0) * 1e3
    stage_ms, _ = ctx.profile_read(reset=True)
    ctx.profile(False)

    def timed_copy(dst, src, reps=3):
        dst.copy_(src, non_blocking=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    h_in = torch.from_numpy(pin_reads)  # shares the pinned pages
    d_in = torch.empty(h_in.numel(), dtype=torch.uint8, device=dev)
    h2d_ms = timed_copy(d_in, h_in)
    del d_in
    nb_out = max(int(e2e["d2h_bytes_per_step"]), 1)
    d_out = torch.empty(nb_out, dtype=torch.uint8, device=dev)
    h_out = torch.empty(nb_out, dtype=torch.uint8).pin_memory()
    d2h_ms = timed_copy(h_out, d_out)
    del d_out, h_out
    dev_ms = float(sum(stage_ms))
    return {"wall_ms": wall, "device_stages_ms": dev_ms, "host_and_copy_out_ms": wall - dev_ms,
            "h2d_alone_ms": h2d_ms, "h2d_gbs": pin_reads.nbytes / h2d_ms / 1e6,
            "d2h_alone_ms": d2h_ms, "d2h_gbs": nb_out / d2h_ms / 1e6,
            "note": "one profiled hsk_count call; copies timed alone from/to pinned host memory"}


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
            # nvidia-smi's start-up can hold the host's driver calls for up to
            # a second; let it reach its first sample before anything is timed
            t_end = time.time() + 3.0
            while time.time() < t_end and self.proc.poll() is None and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_sample(rs, target_windows: int):
    """First reads of the workload holding about target_windows windows."""
    lens = np.diff(rs.offsets.astype(np.int64))
    w = np.maximum(lens - rs.k + 1, 0).cumsum()
    n = int(np.searchsorted(w, target_windows)) + 1
    n = min(n, rs.n_reads)
    return rs.reads[: int(rs.offsets[n])], rs.offsets[: n + 1].copy(), n


def run_cpu_oracle(rs, target_windows: int, steps: int = 1):
    import oracle
    reads, offs, n = cpu_sample(rs, target_windows)
    times = []
    nw = 0
    for _ in range(steps):
        t0 = time.perf_counter()
        r = oracle.count(reads, offs, rs.k, rs.lo, rs.hi)
        times.append(time.perf_counter() - t0)
        nw = r.n_windows
    return nw, times, n


# ---------------------------------------------------------------------------
# batched and served forms against the plain per-job path
# ---------------------------------------------------------------------------

_PINNED = []


def _pinned(rs):
    """The read set's reads and offsets copied into one page-locked host
    buffer of exactly their size (hsk_host_pin; see _unpin_all)."""
    import paper_2407_07718_gb300 as hsk
    ob = rs.offsets.size * 8
    rb = (rs.n_bases + 63) // 64 * 64
    buf = hsk.pinned_empty(ob + rb)
    offs = buf[:ob].view(np.uint64)
    offs[:] = rs.offsets
    reads = buf[ob:ob + rs.n_bases]
    reads[:] = rs.reads
    _PINNED.append(buf)
    return (reads, offs, rs.k, rs.m, rs.lo, rs.hi)


def _unpin_all():
    import paper_2407_07718_gb300 as hsk
    while _PINNED:
        hsk.host_unpin(_PINNED.pop())


def _generate(fn, params):
    """Simulate the read sets on all host cores (the simulator releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=max(1, min(32, os.cpu_count() or 1))) as ex:
        return list(ex.map(lambda p: _pinned(fn(*p)), params))


def _pct(x, q):
    return float(np.percentile(np.asarray(x), q)) if len(x) else None


def _fifo_latency(arrivals, service):
    """Latency of each job on one first-come-first-served server."""
    t, lat = 0.0, []
    for a, s in zip(arrivals, service):
        t = max(t, a) + s
        lat.append(t - a)
    return lat


def _plain_pass(ctx, jobs):
    """Run the jobs one after another through hsk_count; per-job seconds."""
    times, res = [], []
    for j in jobs:
        t0 = time.perf_counter()
        r = ctx.count(*j, copy=False)
        times.append(time.perf_counter() - t0)
        res.append(r)
    return times, res


def bench_batched(hsk, device: int, n_sets: int, scale: float, tune_trials: int = 12) -> dict:
    import datagen
    params = datagen.batched_set_params(n_sets=n_sets, scale=scale)
    t0 = time.perf_counter()
    jobs = _generate(datagen.batched_set, params)
    gen_s = time.perf_counter() - t0
    bases = sum(int(j[0].size) for j in jobs)
    with hsk.Context(device=device) as ctx:
        big = max(range(len(jobs)), key=lambda i: jobs[i][0].size)
        ctx.count(*jobs[big], copy=False)          # warm: the arena grows to the largest set
        plain_t, plain_r = _plain_pass(ctx, jobs)
        # the autotuner picks the forms' parameters on a sample of the sets
        # (every fourth one), timing candidates through hsk_count_batch
        t0 = time.perf_counter()
        tuned = ctx.autotune(jobs[::4], max_trials=tune_trials) if tune_trials else ctx.tune_current()
        tune_s = time.perf_counter() - t0
        ctx.count_batch(jobs, copy=False)           # warm: every slot grows its arena
        p0 = ctx.pack_stats()
        t0 = time.perf_counter()
        batch_r = ctx.count_batch(jobs, copy=False)
        batch_s = time.perf_counter() - t0
        p1 = ctx.pack_stats()
        packs = {key: (p1[key] - p0[key]) if isinstance(p1[key], int) else p1[key] for key in p1}
    for a, b in zip(plain_r, batch_r):
        assert (a.n_windows, a.n_distinct, a.extra["n_pairs"]) == (b.n_windows, b.n_distinct, b.extra["n_pairs"])
    del jobs
    _unpin_all()
    n = sum(r.n_windows for r in plain_r)
    plain_s = sum(plain_t)
    return {"workload": f"{n_sets} sets, genome log-uniform [0.1, 20] Mbp x {scale:g}, coverage U[10, 40]x, "
                        "150 bp reads, 1% sub, k=31 m=17, filter [2,1000]",
            "n_sets": n_sets, "n_bases": bases, "n_windows": n, "generate_s": gen_s,
            "plain": {"value": n / plain_s, "makespan_s": plain_s,
                      "job_p50_ms": _pct(plain_t, 50) * 1e3, "job_p99_ms": _pct(plain_t, 99) * 1e3},
            "batched": {"value": n / batch_s, "makespan_s": batch_s},
            "speedup": plain_s / batch_s, "unit": UNIT, "pack_stats": packs,
            "autotune": dict(tuned, tune_s=tune_s, sample="every 4th set"),
            "note": "makespans include host-to-device copies from pinned memory and result copies back"}


def _mem_available() -> int:
    """Host memory the kernel reports as available (bytes), or 0 if unknown."""
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def bench_served(hsk, device: int, n_req: int, scale: float, load: float, budget: int,
                 tune_trials: int = 8, fixed_rate: float = 0.0) -> dict:
    """The Poisson request stream, its inputs held in pinned host memory.

    The stream's inputs are generated up front.  When they would take more
    than 45 % of the host's available memory (results, the library's host
    pool and the tuner's trial batches need room beside them), the stream is
    run as consecutive blocks, each generated before it starts, at the same
    offered rate, and the latencies of all blocks are pooled; the line says how
    many blocks were used.

    The offered rate is fixed_rate requests per second when it is set (the
    workload's set arrival rate, the same in every run), else `load` times the
    saturated rate measured on the first block."""
    import datagen
    params = datagen.served_request_params(n=n_req, scale=scale)
    need = sum(int(g * c * 1.06) + 4096 for (_, g, c, _, _, _) in params)  # bases + offsets
    avail = _mem_available()
    n_blocks = 1
    if avail and need > 0.45 * avail:
        n_blocks = int(np.ceil(need / max(0.45 * avail, 4e9)))
    blocks = [params[i * len(params) // n_blocks:(i + 1) * len(params) // n_blocks] for i in range(n_blocks)]
    gen_s = plain_s = sat_s = open_s = tune_s = 0.0
    n = 0
    lat, plain_lat = [], []
    rate = None
    tuned = None
    packs = {"passes": 0, "sets": 0, "alone": 0, "failed_passes": 0, "last_failure": ""}
    with hsk.Context(device=device, hbm_budget=budget) as ctx:
        for bi, bparams in enumerate(blocks):
            t0 = time.perf_counter()
            jobs = _generate(datagen.served_request, bparams)
            gen_s += time.perf_counter() - t0
            if bi == 0:
                for kk in sorted({j[2] for j in jobs}):     # warm each key width on the largest request
                    big = max((i for i in range(len(jobs)) if jobs[i][2] == kk), key=lambda i: jobs[i][0].size)
                    ctx.count(*jobs[big], copy=False)
            plain_t, plain_r = _plain_pass(ctx, jobs)
            n_b = sum(r.n_windows for r in plain_r)
            n += n_b
            plain_s += sum(plain_t)
            if bi == 0:
                t0 = time.perf_counter()
                tuned = ctx.autotune(jobs[::20], max_trials=tune_trials) if tune_trials else ctx.tune_current()
                tune_s = time.perf_counter() - t0

            def closed_batch():
                # results are released as they are read: a completed request's
                # host arrays go back to the library's pool for later requests
                t0 = time.perf_counter()
                ts = [ctx.submit(*j) for j in jobs]
                for t in ts:
                    ctx.wait(t, copy=False)
                    ctx.release(t)
                return time.perf_counter() - t0

            closed_batch()                              # warm the slots
            p0 = ctx.pack_stats()
            sat_b = closed_batch()
            sat_s += sat_b
            if rate is None:                            # requests per second offered
                rate = fixed_rate if fixed_rate > 0 else load * len(jobs) / sat_b
            gaps = np.random.default_rng(5 + bi).exponential(1.0 / rate, len(jobs))
            arrivals = np.cumsum(gaps) - gaps[0]
            tickets = []
            t0 = time.perf_counter()
            for i, j in enumerate(jobs):
                while True:
                    d = arrivals[i] - (time.perf_counter() - t0)
                    if d <= 0:
                        break
                    time.sleep(min(d, 0.002))
                tickets.append(ctx.submit(*j))
            res = []
            for t in tickets:
                res.append(ctx.wait(t, copy=False))
                lat.append(sum(ctx.times(t)))
                ctx.release(t)
            open_s += time.perf_counter() - t0
            p1 = ctx.pack_stats()
            for key in packs:
                packs[key] = packs[key] + p1[key] - p0[key] if isinstance(p1[key], int) else p1[key]
            for a, b in zip(plain_r, res):
                assert (a.n_windows, a.n_distinct, a.extra["n_pairs"]) == (b.n_windows, b.n_distinct,
                                                                          b.extra["n_pairs"])
            plain_lat += _fifo_latency(arrivals, plain_t)
            del jobs, plain_r, res
            _unpin_all()
    return {"workload": f"{n_req} Poisson requests, genome log-normal (median 2 Mbp, sigma_ln 1, [0.05, 50] Mbp) "
                        f"x {scale:g}, coverage U[10, 30]x, 150 bp or 10 kb reads, k in {{21, 31, 55}}, filter [2,1000]",
            "n_requests": n_req, "n_windows": n, "generate_s": gen_s, "hbm_budget": budget,
            "blocks": n_blocks, "host_input_bytes": need,
            "offered_rate_per_s": rate, "rate_fixed": fixed_rate > 0,
            "load": rate * sat_s / n_req, "load_on_plain": rate * plain_s / n_req,
            "served": {"value_saturated": n / sat_s, "makespan_saturated_s": sat_s,
                       "value": n / open_s, "p50_ms": _pct(lat, 50) * 1e3, "p99_ms": _pct(lat, 99) * 1e3,
                       "p999_ms": _pct(lat, 99.9) * 1e3},
            "plain": {"value": n / plain_s, "makespan_s": plain_s,
                      "p50_ms": _pct(plain_lat, 50) * 1e3, "p99_ms": _pct(plain_lat, 99) * 1e3,
                      "p999_ms": _pct(plain_lat, 99.9) * 1e3,
                      "latency_model": "measured per-job times on one FIFO server at the same arrival times"},
            "speedup_saturated": plain_s / sat_s, "unit": UNIT, "pack_stats": packs,
            "autotune": dict(tuned, tune_s=tune_s, sample="every 20th request of the first block"),
            "note": "latency = submit to completion; copies from pinned host memory inside every job"}


def bench_second_workload(hsk, local: int, name: str, steps: int, warmup: int) -> dict:
    """Device-resident steps of a second plain workload (default: the
    short-read set at k=55 with 128-bit keys), timed like the main line."""
    import torch
    rs, desc = make_workload(name, 1.0)
    dev = torch.device("cuda", local)
    d_reads = torch.from_numpy(rs.reads).to(dev)
    d_offs = torch.from_numpy(rs.offsets.view(np.int64)).to(dev)
    stream = torch.cuda.current_stream(dev)
    with hsk.Context(device=local) as ctx:
        for _ in range(max(3, warmup)):
            r = ctx.count_device(d_reads, d_offs, rs.k, rs.m, rs.lo, rs.hi, stream=stream)
        ctx.profile(True)
        ctx.profile_read(reset=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            r = ctx.count_device(d_reads, d_offs, rs.k, rs.m, rs.lo, rs.hi, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        stage_ms, _ = ctx.profile_read(reset=True)
        out = {"workload": desc, "k": rs.k, "m": rs.m, "lo": rs.lo, "hi": rs.hi, "n_bases": rs.n_bases,
               "n_windows": int(r.n_windows), "n_pairs": int(r.n_pairs), "n_distinct": int(r.n_distinct),
               "steps": steps, "ms_per_step": ms, "value": int(r.n_windows) / (ms / 1e3), "unit": UNIT,
               "dtype": "u64" if rs.k <= 32 else "u128",
               "stages_ms_per_step": {n: v / steps for n, v in zip(hsk.Context.STAGES, stage_ms)}}
    del d_reads, d_offs
    torch.cuda.empty_cache()
    return out


def bench_extension(hsk, local: int, rs, pin_reads, pin_offs, steps: int = 2) -> dict:
    """Counting with extension information (Sec. 3.3.2) through hsk_count_ext
    on the workload's pinned host inputs, against hsk_count, and the byte cost
    of the extension payload: 8 bytes per occurrence (uint32 read + uint32
    position) against the paper's encoding (flag byte + two int8 differences,
    or the flag byte + the full pair) of the occurrences in read order, i.e.
    the consecutive kept k-mers of each read."""
    import torch
    with hsk.Context(device=local) as ctx:
        ctx.count(pin_reads, pin_offs, rs.k, rs.m, rs.lo, rs.hi, copy=False)
        ctx.count_ext(pin_reads, pin_offs, rs.k, rs.m, rs.lo, rs.hi)
        t0 = time.perf_counter()
        for _ in range(steps):
            ctx.count(pin_reads, pin_offs, rs.k, rs.m, rs.lo, rs.hi, copy=False)
        count_s = (time.perf_counter() - t0) / steps
        t0 = time.perf_counter()
        for _ in range(steps):
            res, off, rd, ps = ctx.count_ext(pin_reads, pin_offs, rs.k, rs.m, rs.lo, rs.hi)
        ext_s = (time.perf_counter() - t0) / steps
        n_occ = int(rd.size)
        order = np.lexsort((ps, rd))
        d_rd = torch.from_numpy(rd[order].view(np.int32)).cuda(local)
        d_ps = torch.from_numpy(ps[order].view(np.int32)).cuda(local)
        out = torch.empty(max(9 * n_occ, 1), dtype=torch.uint8, device=f"cuda:{local}")
        chunks = max((n_occ + hsk.EXT_CHUNK - 1) // hsk.EXT_CHUNK, 1)
        coff = torch.empty(chunks, dtype=torch.int64, device=f"cuda:{local}")
        nb = ctx.stage_ext_encode(d_rd, d_ps, out, coff)
        del out, d_rd, d_ps, coff
    torch.cuda.empty_cache()
    enc = nb + 8 * chunks
    return {"count_ms": count_s * 1e3, "count_ext_ms": ext_s * 1e3, "n_pairs": int(res.counts.size),
            "n_occ": n_occ, "payload_raw_bytes": 8 * n_occ, "payload_encoded_bytes": enc,
            "encoded_over_raw": enc / max(1, 8 * n_occ),
            "note": "hsk_count and hsk_count_ext from pinned host inputs, results copied back; encoded = "
                    "the paper's extension encoding of the occurrences in read order, plus its chunk index"}


def run_ablations(rs, local: int) -> dict:
    """Diagnostics of the bucketing on the workload's reads (device-resident):
    bucket balance (k-mers per bucket, from the S3 stage) at 256 and 4096
    buckets, a sweep of the minimizer length m with the whole count's device
    time, the supermers formed and their mean k-mers, and hash against
    lexical minimizer order (S2's time, supermers, balance; same counts)."""
    import torch
    import paper_2407_07718_gb300 as hsk
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    d_reads = torch.from_numpy(rs.reads).to(dev)
    d_offs = torch.from_numpy(rs.offsets.view(np.int64)).to(dev)
    stream = torch.cuda.current_stream(dev)
    balance, sweep = [], []
    with hsk.Context(device=local) as ctx:
        for B in (256, 4096):
            bk = torch.zeros(B, dtype=torch.int64, device=dev)
            br = torch.zeros(B + 1, dtype=torch.int64, device=dev)
            _, nrec, _, _ = ctx.stage_supermers(d_reads, d_offs, rs.k, rs.m, B, bk, br, stream=stream)
            torch.cuda.synchronize()
            v = bk.cpu().numpy().astype(np.float64)
            mean = v.mean()
            balance.append({"n_buckets": B, "m": rs.m, "kmers_per_bucket_mean": mean,
                            "max_over_mean": float(v.max() / mean), "min_over_mean": float(v.min() / mean),
                            "cv": float(v.std() / mean), "n_supermers": int(nrec)})
        for m in (11, 13, 15, 17, 19, 21):
            if m > rs.k or m > 32:
                continue
            for _ in range(2):
                r = ctx.count_device(d_reads, d_offs, rs.k, m, rs.lo, rs.hi, stream=stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 3
            e0.record(stream)
            for _ in range(reps):
                r = ctx.count_device(d_reads, d_offs, rs.k, m, rs.lo, rs.hi, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            sweep.append({"m": m, "ms_per_count": ms, "kmers_per_s": int(r.n_windows) / (ms / 1e3),
                          "n_supermers": int(r.n_supermers),
                          "kmers_per_supermer": int(r.n_windows) / max(1, int(r.n_supermers)),
                          "n_distinct": int(r.n_distinct), "n_pairs": int(r.n_pairs)})
        # E14: hash-ordered against lexically ordered minimizers (Sec. 3.2):
        # the same counts, different supermers and bucket balance, S2's cost
        order = []
        for lexical in (False, True):
            with hsk.Context(device=local, lexical_minimizers=lexical) as c2:
                B = 4096
                bk = torch.zeros(B, dtype=torch.int64, device=dev)
                br = torch.zeros(B + 1, dtype=torch.int64, device=dev)
                c2.stage_supermers(d_reads, d_offs, rs.k, rs.m, B, bk, br, stream=stream)
                torch.cuda.synchronize()
                v = bk.cpu().numpy().astype(np.float64)
                for _ in range(2):
                    r = c2.count_device(d_reads, d_offs, rs.k, rs.m, rs.lo, rs.hi, stream=stream)
                c2.profile(True)
                c2.profile_read(reset=True)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                reps = 3
                e0.record(stream)
                for _ in range(reps):
                    r = c2.count_device(d_reads, d_offs, rs.k, rs.m, rs.lo, rs.hi, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                st_ms, _ = c2.profile_read(reset=True)
                order.append({"order": "lexical" if lexical else "hash", "m": rs.m,
                              "ms_per_count": e0.elapsed_time(e1) / reps,
                              "s2_ms": st_ms[1] / reps, "stages_ms": [x / reps for x in st_ms],
                              "n_supermers": int(r.n_supermers),
                              "kmers_per_supermer": int(r.n_windows) / max(1, int(r.n_supermers)),
                              "buckets_4096_max_over_mean": float(v.max() / v.mean()),
                              "buckets_4096_cv": float(v.std() / v.mean()),
                              "n_distinct": int(r.n_distinct), "n_pairs": int(r.n_pairs),
                              "keys_off_chip": c2.last_overflow()})
        assert order[0]["n_distinct"] == order[1]["n_distinct"] and order[0]["n_pairs"] == order[1]["n_pairs"]
    return {"bucket_balance": balance, "m_sweep": sweep, "minimizer_order": order}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("HSK_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def reduce_max(pg, x: float, device) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(pg, x: float, device) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="long_read", choices=["long_read", "short_read", "tiny"])
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-windows", type=int, default=20_000_000,
                    help="windows in the oracle's bounded sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched and served measurements")
    ap.add_argument("--no-ext", action="store_true", help="skip the extension-information leg")
    ap.add_argument("--second-workload", default="short_read", choices=["short_read", "long_read", "none"],
                    help="a second plain workload reported under its own key (default: short-read, k=55)")
    ap.add_argument("--second-steps", type=int, default=5)
    ap.add_argument("--batched-sets", type=int, default=256)
    ap.add_argument("--batched-scale", type=float, default=1.0)
    ap.add_argument("--served-requests", type=int, default=2000)
    ap.add_argument("--tune-trials", type=int, default=10, help="autotuner trials before the forms (0 = none)")
    ap.add_argument("--served-scale", type=float, default=1.0)
    ap.add_argument("--served-load", type=float, default=0.7, help="offered load when --served-rate is 0")
    ap.add_argument("--served-rate", type=float, default=150.0,
                    help="Poisson arrival rate of the served stream, requests/s (0 = --served-load x saturated)")
    ap.add_argument("--served-budget", type=float, default=120e9)
    ap.add_argument("--ablations", action="store_true",
                    help="print one JSON line of bucketing diagnostics (bucket balance, m sweep) instead")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world, rank, local, pg = dist_setup()
    rs, desc = make_workload(args.workload, args.scale)
    kw = 1 if rs.k <= 32 else 2
    config = {"workload": desc, "k": rs.k, "m": rs.m, "lo": rs.lo, "hi": rs.hi, "n_reads": rs.n_reads,
              "n_bases": rs.n_bases, "l2": "inputs larger than L2 (reads %.2f GB); no flush" % (rs.n_bases / 1e9)}

    if args.ablations:
        if rank == 0:
            print(json.dumps({"ablations": run_ablations(rs, local), "config": config}))
        return

    if args.impl == "reference":
        if rank != 0:
            return
        steps = max(1, args.steps)
        # each step counts the same bounded sample (the first reads holding
        # about --cpu-windows windows); warm-up steps are not timed
        run_cpu_oracle(rs, args.cpu_windows, steps=args.warmup)
        nw, times, nreads = run_cpu_oracle(rs, args.cpu_windows, steps=steps)
        tot = sum(times)
        value = nw * steps / tot
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
                "steps": steps, "warmup": args.warmup, "ms_per_step": tot / steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64" if kw == 1 else "u128",
                "data": "synthetic", "config": config,
                "cpu_baseline": dict({"kind": "oracle", "value": value, "unit": UNIT, "cores": 1,
                                      "sample": f"first {nreads} reads of the workload ({nw} windows), single-thread C++ std::sort oracle"},
                                     **host_cpu()),
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    import paper_2407_07718_gb300 as hsk

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    d_reads = torch.from_numpy(rs.reads).to(dev)
    d_offs = torch.from_numpy(rs.offsets.view(np.int64)).to(dev)
    ctx = hsk.Context(device=local)
    stream = torch.cuda.current_stream(dev)

    res = None
    for _ in range(args.warmup):
        res = ctx.count_device(d_reads, d_offs, rs.k, rs.m, rs.lo, rs.hi, stream=stream)
    n_windows = int(res.n_windows)
    ctx.profile(True)
    ctx.profile_read(reset=True)
    launches0 = hsk.Context.launch_count()
    sampler = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    if pg is not None:
        pg.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.05)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        res = ctx.count_device(d_reads, d_offs, rs.k, rs.m, rs.lo, rs.hi, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    if pg is not None:
        pg.barrier()
    clocks = sampler.stop()
    launches = hsk.Context.launch_count() - launches0
    ms = e0.elapsed_time(e1)
    stage_ms, passes = ctx.profile_read(reset=True)
    overflow = ctx.last_overflow()
    ctx.profile(False)
    ms_max = reduce_max(pg, ms, dev)
    total_windows = reduce_sum(pg, float(n_windows) * args.steps, dev)
    value = total_windows / (ms_max / 1e3)

    # roofline of the dominant kernel
    peaks = measured_peaks()
    kb = 8 * kw
    clk_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    if passes > 0:  # global radix passes: one onesweep LSD pass reads and writes every key (HBM-bound)
        launch_ms = stage_ms[4] / passes
        bytes_per_launch = n_windows * 2 * kb
        achieved = bytes_per_launch / (launch_ms / 1e3) / 1e9 if launch_ms > 0 else 0.0
        sha = source_sha(os.path.join(ROOT, "paper_2407_07718_gb300", "csrc", "k_sort.cu"))
        cnt = NCU_PER_KEY.get((args.workload, sha))
        roofline = {"bound": "hbm", "kernel": "k_onesweep_tma (8-bit LSD pass)", "achieved": achieved,
                    "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                    "traffic": cnt["dram"] * n_windows / passes if cnt else None,
                    "peak_source": f"{peaks['source']} (MEASURED_PEAKS hbm_gbs copy bandwidth)",
                    "bytes_per_launch": bytes_per_launch, "launch_ms": launch_ms}
    else:
        # on-chip path: the sub-segment sort (k_local_sort, all tiers) reads
        # every key once and writes the kept pairs; it is bound by instruction
        # issue and shared-memory latency, so its roofline is the issue rate
        launch_ms = stage_ms[4] / args.steps
        sha = source_sha(os.path.join(ROOT, "paper_2407_07718_gb300", "csrc", "k_local.cu"))
        cnt = NCU_PER_KEY.get((args.workload, sha))
        n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak_issue = n_sms * SCHEDULERS_PER_SM * clk_mhz / 1e3  # G warp-instructions / s
        inst = cnt["inst"] * n_windows if cnt else None
        achieved = inst / (launch_ms / 1e3) / 1e9 if inst and launch_ms > 0 else None
        hbm_bytes = n_windows * kb + int(res.n_pairs) * (kb + 4)
        hbm_achieved = hbm_bytes / (launch_ms / 1e3) / 1e9 if launch_ms > 0 else 0.0
        wav = cnt.get("smem_wavefronts") * n_windows if cnt else None
        smem_peak = n_sms * clk_mhz / 1e3  # G wavefronts / s: one per SM per cycle
        smem_achieved = wav / (launch_ms / 1e3) / 1e9 if wav and launch_ms > 0 else None
        roofline = {"bound": "alu", "kernel": "k_local_sort (sub-segment sort + count in shared memory, all tiers)",
                    "achieved": achieved, "peak": peak_issue, "unit": "G warp-instructions/s",
                    "frac": achieved / peak_issue if achieved else None,
                    "traffic": cnt["dram"] * n_windows if cnt else None,
                    "peak_source": f"issue slots: {n_sms} SMs x {SCHEDULERS_PER_SM} schedulers x {clk_mhz:.0f} MHz (sampled)",
                    "inst_per_launch": inst, "launch_ms": launch_ms,
                    "smem_view": {"wavefronts_per_launch": wav, "achieved": smem_achieved, "peak": smem_peak,
                                  "unit": "G shared-memory wavefronts/s",
                                  "frac": smem_achieved / smem_peak if smem_achieved else None,
                                  "peak_source": f"{n_sms} SMs x 1 wavefront per cycle x {clk_mhz:.0f} MHz"},
                    "hbm_view": {"bytes_per_launch": hbm_bytes, "achieved": hbm_achieved, "unit": "GB/s",
                                 "frac": hbm_achieved / peaks["hbm_gbs"],
                                 "peak_source": f"{peaks['source']} (MEASURED_PEAKS hbm_gbs copy bandwidth)"}}
    roofline["passes_per_step"] = passes / args.steps
    # end-to-end algorithmic bytes per step (byte model of the whole path)
    n_sm = int(res.n_supermers)
    rec_b = 16 if kw == 1 else 32
    P = (2 * rs.k + 7) // 8
    if passes > 0:
        s45 = (n_sm * rec_b                                # S4: records read
               + n_windows * kb * (1 + 2 * P)              # keys written, P passes
               + n_windows * kb + int(res.n_pairs) * (kb + 4))  # S5: keys read, kept pairs written
    else:
        s45 = (2 * n_sm * rec_b                            # S4: records read to count, then to scatter
               + n_windows * kb * 2                        # keys written by the scatter, read on chip
               + int(res.n_pairs) * (kb + 4) * 3)          # kept pairs written, compacted (read + write)
    e2e_bytes = (rs.n_bases * (1 + 0.25 + 0.25)            # S1: ASCII in, packed + masks out
                 + 2 * rs.n_bases * 0.5                    # S2 + S3: packed + masks read twice
                 + n_sm * rec_b                            # S3 records written
                 + s45
                 + int(res.n_pairs) * (kb + 4) * 2 * P)    # S6: output pairs sorted
    step_s = ms_max / args.steps / 1e3
    roofline["end_to_end"] = {"bytes_per_step": e2e_bytes, "achieved": e2e_bytes / step_s / 1e9,
                              "frac": e2e_bytes / step_s / 1e9 / peaks["hbm_gbs"]}

    # end to end through the host API: pinned inputs, results copied back
    # (every rank: its replica's time enters the max over ranks)
    pin_reads = torch.from_numpy(rs.reads).pin_memory().numpy()
    pin_offs = torch.from_numpy(rs.offsets.view(np.int64)).pin_memory().numpy().view(np.uint64)
    # hsk_count copies the inputs in and the results (pairs + histogram) out into
    # library-owned host memory; copy=False skips the binding's extra numpy copy
    r = ctx.count(pin_reads, pin_offs, rs.k, rs.m, rs.lo, rs.hi, copy=False)  # warm
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        r = ctx.count(pin_reads, pin_offs, rs.k, rs.m, rs.lo, rs.hi, copy=False)
    dt = (time.perf_counter() - t0) / args.e2e_steps
    dt = reduce_max(pg, dt, dev)
    e2e = {"value": reduce_sum(pg, float(r.n_windows), dev) / dt, "unit": UNIT,
           "h2d_bytes_per_step": int(pin_reads.nbytes + pin_offs.nbytes),
           "d2h_bytes_per_step": int(r.extra["n_pairs"] * (kb + 4) + 65536 * 8),
           "ms_per_step": dt * 1e3}
    assert r.n_windows == n_windows
    e2e["parts"] = e2e_parts(ctx, rs, pin_reads, pin_offs, e2e, dev)

    ext_leg = None
    if rank == 0 and world == 1 and not args.no_ext:
        ext_leg = bench_extension(hsk, local, rs, pin_reads, pin_offs)
        print(json.dumps({"extension": ext_leg}), file=sys.stderr, flush=True)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        nw, times, nreads = run_cpu_oracle(rs, args.cpu_windows)
        cpu = dict({"value": nw / times[0], "unit": UNIT, "cores": 1, "kind": "oracle",
                    "sample": f"first {nreads} reads of the workload ({nw} windows), single-thread C++ std::sort oracle, {times[0]:.1f} s"},
                   **host_cpu())

    ctx.close()
    del d_reads, d_offs
    forms = {}
    def leg(name, fn):  # each extra leg is also logged to stderr as soon as it ends
        # the SM clocks over the whole leg, so that legs of different runs can be compared
        sampler_leg = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
        sampler_leg.start()
        forms[name] = fn()
        forms[name]["clocks"] = sampler_leg.stop()
        print(json.dumps({name: forms[name]}), file=sys.stderr, flush=True)

    if rank == 0 and world == 1 and args.second_workload not in ("none", args.workload):
        torch.cuda.empty_cache()
        leg(args.second_workload, lambda: bench_second_workload(hsk, local, args.second_workload, args.second_steps,
                                                                args.warmup))
    if rank == 0 and world == 1 and not args.no_forms:
        torch.cuda.empty_cache()
        leg("batched", lambda: bench_batched(hsk, local, args.batched_sets, args.batched_scale, args.tune_trials))
        leg("served", lambda: bench_served(hsk, local, args.served_requests, args.served_scale, args.served_load,
                                           int(args.served_budget), args.tune_trials, args.served_rate))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64" if kw == 1 else "u128",
                "data": "synthetic", "config": dict(config, n_windows=n_windows,
                                                     n_distinct=int(res.n_distinct), n_pairs=int(res.n_pairs),
                                                     n_supermers=n_sm, n_chunks=int(res.n_chunks),
                                                     keys_off_chip=overflow,
                                                     parallelism=f"replicas x{world}"),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": int(launches),
                "stages_ms_per_step": {n: v / args.steps for n, v in zip(hsk.Context.STAGES, stage_ms)}}
        if ext_leg is not None:
            line["extension"] = ext_leg
        line.update(forms)
        print(json.dumps(line))
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
