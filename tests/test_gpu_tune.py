"""The autotuner of the batched and served forms (hsk_autotune): it times
candidate parameters on sample jobs, applies the fastest, records them for
the jobs' class in the context and in its cache file, and a context created
later with that file applies them to a batch of the same class.  Results stay
bit-exact with the oracle under every parameter set tried."""
import numpy as np
import pytest

import datagen
import oracle
from gpu_util import assert_same_result

pytestmark = pytest.mark.gpu


def _jobs(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        g = int(np.exp(rng.uniform(np.log(5_000), np.log(80_000))))
        rs = datagen.batched_set(datagen.derive_seed(seed, i), g, float(rng.uniform(8, 20)))
        out.append((rs.reads, rs.offsets, 31, 17, 2, 1000))
    return out


def test_autotune_records_applies_and_keeps_results_exact(hsk, tmp_path):
    jobs = _jobs(24, 5)
    wants = [oracle.count(r, o, k, lo, hi) for (r, o, k, m, lo, hi) in jobs]
    cache = str(tmp_path / "tune.txt")
    with hsk.Context(tune_cache=cache) as ctx:
        before = ctx.tune_current()
        assert (before["group_div"], before["slots"]) == (3, 4)
        r = ctx.autotune(jobs, max_trials=6)
        assert 1 <= r["trials"] <= 6
        assert r["best_s"] > 0 and r["best_s"] <= r["first_s"] * 1.0001
        assert r["slots"] in (2, 3, 4, 6) and r["group_div"] in (2, 3, 4, 6)
        now = ctx.tune_current()
        for f in ("group_div", "plain_bucket_shift", "pack_bases", "pack_small", "slots"):
            assert now[f] == r[f], f
        got = ctx.count_batch(jobs)
        for i, (g, w) in enumerate(zip(got, wants)):
            assert_same_result(g, w, f"set {i} after tuning")
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1 and lines[0].startswith("u64:2^")
    # a new context reads the file and applies the entry to a batch of that class
    with hsk.Context(tune_cache=cache, autotune=True) as ctx2:
        ctx2.count_batch(jobs[:6] + jobs[6:])
        now2 = ctx2.tune_current()
        for f in ("group_div", "plain_bucket_shift", "pack_bases", "pack_small", "slots"):
            assert now2[f] == r[f], f
    # with autotune off the recorded entry is not applied
    with hsk.Context(tune_cache=cache, autotune=False) as ctx3:
        ctx3.count_batch(jobs)
        assert ctx3.tune_current()["group_div"] == 3


@pytest.mark.parametrize("param,values", [("slots", [2, 3, 6]), ("pack_bases", [256 << 20, 2 << 30]),
                                          ("pack_small", [64 << 20, 1 << 30]), ("group_div", [2, 4, 6]),
                                          ("plain_bucket_shift", [1])])
def test_every_tuning_candidate_counts_exactly(hsk, param, values):
    """Each value the tuner may pick gives the oracle's result (small sets
    packed, one set large enough to run alone)."""
    jobs = _jobs(10, 9)
    big = datagen.batched_set(datagen.derive_seed(9, 99), 600_000, 12.0)
    jobs.insert(4, (big.reads, big.offsets, 31, 17, 2, 1000))
    wants = [oracle.count(r, o, k, lo, hi) for (r, o, k, m, lo, hi) in jobs]
    with hsk.Context() as ctx:
        for v in values:
            small = {"pack_small": 4 << 20} if param != "pack_small" else {}
            ctx.tune_set(**{param: v}, **small)
            assert ctx.tune_current()[param] == v
            got = ctx.count_batch(jobs)
            for i, (g, w) in enumerate(zip(got, wants)):
                assert_same_result(g, w, f"{param}={v} set {i}")
        with pytest.raises(hsk.HskError):
            ctx.tune_set(slots=0)
