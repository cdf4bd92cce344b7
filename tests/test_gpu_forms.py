"""Batched (hsk_count_batch) and served (hsk_submit / hsk_wait) forms: every
job's result is bit-exact with the CPU oracle run on that job alone, whatever
the mix of sizes and k it shares the device with."""
import numpy as np
import pytest

import datagen
import oracle
from gpu_util import assert_same_result

pytestmark = pytest.mark.gpu

HSK_EINVAL, HSK_ECANCELED, HSK_ENOTFOUND = -1, -5, -7


def _mixed_jobs():
    """Small sets of several sizes and key widths, an empty set and reads shorter than k."""
    jobs = []
    for i, (g, cov) in enumerate([(20_000, 10.0), (200_000, 12.0), (5_000, 30.0), (80_000, 5.0)]):
        rs = datagen.batched_set(datagen.derive_seed(11, i), g, cov)
        jobs.append((rs.reads, rs.offsets, 31, 17, 2, 1000))
    for i, (k, m) in enumerate([(21, 11), (55, 21), (64, 32), (13, 7)]):
        r, o = datagen.random_reads(100 + i, 300, 0, 400, p_invalid=0.002)
        # repeated copies so that counts above 1 exist at every k
        r = np.concatenate([r, r, r])
        o = np.concatenate([o, o[1:] + o[-1], o[1:] + 2 * o[-1]])
        jobs.append((r, o, k, m, 2, 1000))
    jobs.append((np.zeros(0, np.uint8), np.zeros(1, np.uint64), 31, 17, 2, 1000))  # no reads
    r, o = datagen.random_reads(7, 50, 0, 30)                                        # all shorter than k
    jobs.append((r, o, 31, 17, 1, 1000))
    return jobs


@pytest.fixture(scope="module")
def jobs():
    return _mixed_jobs()


@pytest.fixture(scope="module")
def wants(jobs):
    return [oracle.count(r, o, k, lo, hi) for (r, o, k, m, lo, hi) in jobs]


def test_count_batch_matches_oracle_per_job(hsk, jobs, wants):
    with hsk.Context() as ctx:
        got = ctx.count_batch(jobs)
        assert len(got) == len(jobs)
        for i, (g, w) in enumerate(zip(got, wants)):
            assert_same_result(g, w, f"batch job {i}")
        # a second batch on the same (now warm) slots gives the same bytes
        again = ctx.count_batch(jobs[::-1])
        for i, (g, w) in enumerate(zip(again, wants[::-1])):
            assert_same_result(g, w, f"batch job {i} (reversed)")


def test_count_batch_same_as_plain_calls(hsk, jobs, wants):
    with hsk.Context() as ctx:
        plain = [ctx.count(*j) for j in jobs]
        batch = ctx.count_batch(jobs)
    for i, (p, b) in enumerate(zip(plain, batch)):
        assert_same_result(b, p, f"job {i}")


def test_count_batch_rejects_bad_job_before_running(hsk, jobs):
    bad = list(jobs[:3]) + [(jobs[0][0], jobs[0][1], 0, 1, 2, 1000)]
    with hsk.Context() as ctx:
        with pytest.raises(hsk.HskError) as e:
            ctx.count_batch(bad)
        assert e.value.code == HSK_EINVAL
        assert ctx.count_batch([]) == []


def test_count_batch_reports_failing_job(hsk, jobs, wants):
    r, o = jobs[0][0], jobs[0][1].copy()
    o[3], o[4] = o[4], o[3]  # offsets no longer monotone: the job fails, the others still run
    with hsk.Context() as ctx:
        with pytest.raises(hsk.HskError) as e:
            ctx.count_batch([jobs[1], (r, o, 31, 17, 2, 1000), jobs[2]])
        assert e.value.code == HSK_EINVAL
        assert "job 1" in str(e.value)
        # the context stays usable
        assert_same_result(ctx.count_batch([jobs[2]])[0], wants[2], "after failure")


def test_submit_wait_release_matches_oracle(hsk, jobs, wants):
    with hsk.Context() as ctx:
        tickets = [ctx.submit(*j) for j in jobs]
        for i in np.random.default_rng(0).permutation(len(jobs)):
            assert_same_result(ctx.wait(tickets[i]), wants[i], f"served job {i}")
        for t in tickets:
            assert ctx.poll(t)
            q, x = ctx.times(t)
            assert q >= 0 and x >= 0
            ctx.release(t)
        with pytest.raises(hsk.HskError) as e:
            ctx.wait(tickets[0])
        assert e.value.code == HSK_ENOTFOUND


def test_cancel_queued_job(hsk, jobs, wants):
    """A job still queued can be cancelled; one already taken by a slot runs to the end."""
    big = datagen.batched_set(datagen.derive_seed(12, 0), 2_000_000, 30.0)
    with hsk.Context() as ctx:
        # occupy the slots, then queue a job behind them
        blockers = [ctx.submit(big.reads, big.offsets, 31, 17, 2, 1000) for _ in range(8)]
        t = ctx.submit(*jobs[1])
        try:
            ctx.cancel(t)
            cancelled = True
        except hsk.HskError as e:
            assert e.code == HSK_EINVAL  # it had already started
            cancelled = False
        if cancelled:
            with pytest.raises(hsk.HskError) as e:
                ctx.wait(t)
            assert e.value.code == HSK_ECANCELED
        else:
            assert_same_result(ctx.wait(t), wants[1], "not cancelled")
        want_big = None
        for b in blockers:
            r = ctx.wait(b)
            if want_big is None:
                want_big = r
            else:
                assert_same_result(r, want_big, "blocker")
            ctx.release(b)
        ctx.release(t)


def test_served_under_small_budget_runs_jobs_one_at_a_time(hsk, jobs, wants):
    """With a budget below two jobs' estimates, admission still completes every job."""
    with hsk.Context(hbm_budget=256 << 20) as ctx:
        tickets = [ctx.submit(*j) for j in jobs[:4]]
        for i, t in enumerate(tickets):
            assert_same_result(ctx.wait(t), wants[i], f"budget job {i}")
            ctx.release(t)
