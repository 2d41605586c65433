"""EP-adapt host side (Section 4.2): the asynchronous partition job and the
switch/fallback policy, with host-side fault injection.  No GPU needed."""
import threading
import time

import numpy as np
import pytest

import workloads as W
import paper_1605_02043_gb300 as E
from paper_1605_02043_gb300 import adapt as A

KEYS = ("block_ptr", "edge_perm", "vert_ptr", "vert_list", "relabel")


@pytest.fixture(scope="module")
def mesh():
    n = 1 << 14
    src, dst = W.knn_mesh(n, 4, 0)
    return n, src, dst


def test_job_result_matches_synchronous_partition(mesh):
    n, src, dst = mesh
    ref = E.Schedule.partition(src, dst, n, 256).arrays()
    jobs = [E.PartitionJob(src, dst, n, 256, threads=t) for t in (1, 4)]  # two at once
    for j in jobs:
        assert j.wait(60)
        a = j.take().arrays()
        for key in KEYS:
            assert np.array_equal(a[key], ref[key]), key
        assert j.seconds > 0
        with pytest.raises(E.EpError) as ei:  # handed over once only
            j.take()
        assert ei.value.code == -1
        j.close()


def test_job_copies_its_input(mesh):
    n, src, dst = mesh
    ref = E.Schedule.partition(src, dst, n, 128).arrays()
    s, d = src.copy(), dst.copy()
    j = E.PartitionJob(s, d, n, 128)
    s[:] = 0  # caller reuses its buffers at once
    d[:] = 0
    assert j.wait(60)
    assert np.array_equal(j.take().arrays()["edge_perm"], ref["edge_perm"])
    j.close()


def test_job_invalid_arguments_fail_at_start(mesh):
    n, src, dst = mesh
    for args in ((src, dst, n, 0), (src, dst, 3, 256)):
        with pytest.raises(E.EpError) as ei:
            E.PartitionJob(*args)
        assert ei.value.code == -1


def test_injected_failure(mesh):
    n, src, dst = mesh
    j = E.PartitionJob(src, dst, n, 256, test=E.JOB_TEST_FAIL)
    assert j.wait(10)
    with pytest.raises(E.EpError) as ei:
        j.take()
    assert ei.value.code == -2 and "injected" in str(ei.value)
    j.close()


def test_held_job_is_cancelled_promptly(mesh):
    n, src, dst = mesh
    j = E.PartitionJob(src, dst, n, 256, test=E.JOB_TEST_HOLD)
    assert not j.wait(0.2)
    with pytest.raises(E.EpError) as ei:
        j.take()  # still running
    assert ei.value.code == -1
    t0 = time.monotonic()
    j.cancel()
    assert j.wait(5)
    assert time.monotonic() - t0 < 1.0
    with pytest.raises(E.EpError) as ei:
        j.take()
    assert ei.value.code == -6
    j.close()


def test_cancel_stops_a_real_partition():
    n = 1 << 17
    src, dst = W.knn_mesh(n, 4, 1)
    t0 = time.monotonic()
    full = E.PartitionJob(src, dst, n, 256, threads=1)
    assert full.wait(120)
    t_full = time.monotonic() - t0
    full.take()
    full.close()
    j = E.PartitionJob(src, dst, n, 256, threads=1)
    time.sleep(0.02)
    j.cancel()
    assert j.wait(60)
    with pytest.raises(E.EpError) as ei:
        j.take()
    assert ei.value.code == -6
    assert j.seconds < 0.5 * t_full
    j.close()


def test_free_while_running_joins(mesh):
    n, src, dst = mesh
    j = E.PartitionJob(src, dst, n, 256, test=E.JOB_TEST_HOLD)
    t0 = time.monotonic()
    j.close()  # cancels and joins
    assert time.monotonic() - t0 < 1.0


def test_wait_from_several_threads(mesh):
    n, src, dst = mesh
    j = E.PartitionJob(src, dst, n, 256, test=E.JOB_TEST_HOLD)
    seen = []

    def waiter():
        seen.append(j.wait(10))

    ts = [threading.Thread(target=waiter) for _ in range(3)]
    for t in ts:
        t.start()
    time.sleep(0.1)
    j.cancel()
    for t in ts:
        t.join()
    assert seen == [True, True, True]
    j.close()


# ------------------------------------------------------------------ policy
def test_policy_keeps_a_faster_schedule():
    P = A.Policy()
    for ms in (1.0, 1.2, 0.8):
        P.add_default(ms)
    assert P.job_ended(True)
    assert P.phase == A.TRIAL
    assert P.trial_done(0.5)
    assert P.phase == A.OPTIMISED and P.trial_ms == 0.5


def test_policy_reverts_a_slower_schedule():
    P = A.Policy()
    P.add_default(1.0)
    P.job_ended(True)
    assert not P.trial_done(1.01)
    assert P.phase == A.REVERTED


def test_policy_margin_and_history():
    P = A.Policy(margin=0.1, history=2)
    for ms in (100.0, 1.0, 1.0):  # only the last two count
        P.add_default(ms)
    assert P.reference_ms() == 1.0
    P.job_ended(True)
    assert P.trial_done(1.09)  # within 10%
    Q = A.Policy(margin=-0.5)
    Q.add_default(1.0)
    Q.job_ended(True)
    assert not Q.trial_done(0.6)  # must be twice as fast


def test_policy_without_default_timing_keeps_trial():
    P = A.Policy()
    P.job_ended(True)
    assert P.trial_done(123.0) and P.phase == A.OPTIMISED


def test_policy_failed_job_stays_on_default():
    P = A.Policy()
    assert not P.job_ended(False, "boom")
    assert P.phase == A.FAILED and P.error == "boom"
    assert not P.job_ended(True)  # a late result is ignored
    with pytest.raises(RuntimeError):
        P.trial_done(1.0)
