"""EP-adapt on the GPU (Section 4.2): the state carried across a schedule
swap (and back, on a forced fallback) must equal the oracle's, whatever the
partition job did (finished, failed by injection, or still running when the
application ends)."""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1605_02043_gb300 as E  # noqa: E402
from paper_1605_02043_gb300 import adapt as A  # noqa: E402

RTOL = 1e-5
TAU = 1e-3


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def case():
    n = 1 << 16
    src, dst = W.knn_mesh(n, 4, 0)
    x0 = W.flux_state(n, 5, 0)
    w = W.flux_weights(src.size, 0)
    return n, src, dst, x0, w


def drive(R, calls, per_call, wait_job_after=None):
    for c in range(calls):
        R.step(TAU, steps=per_call)
        if c == wait_job_after and R.job is not None:
            R.job.wait(120)
            R.poll()
    R.finish()


def check_state(R, case, T):
    n, src, dst, x0, w = case
    x = torch.empty(5, n, device="cuda")
    R.state(x)
    xT, _ = O.flux_steps(src, dst, x0, w, T, TAU)
    assert rel_l2(x.cpu().numpy(), xT) <= RTOL


def make(case, **kw):
    n, src, dst, x0, w = case
    return A.AdaptiveFlux(src, dst, n, 256, torch.from_numpy(x0).float().cuda(),
                          torch.from_numpy(w).float().cuda(), **kw)


def test_swap_to_partitioned_schedule(case):
    R = make(case, margin=10.0)  # keep it whatever the timing noise
    drive(R, calls=6, per_call=2, wait_job_after=1)
    assert R.phase == A.OPTIMISED
    assert R.switch_step in (2, 4) and R.partition_seconds > 0
    assert R.cur is R.optimised
    assert R.policy.default_ms and R.policy.trial_ms > 0
    check_state(R, case, 12)
    R.close()


def test_forced_fallback_goes_back(case):
    R = make(case, margin=-0.999)  # the trial can never be fast enough
    drive(R, calls=6, per_call=2, wait_job_after=1)
    assert R.phase == A.REVERTED and R.cur is R.default
    check_state(R, case, 12)
    R.close()


def test_failed_job_stays_on_default(case):
    R = make(case, job_test=E.JOB_TEST_FAIL)
    drive(R, calls=4, per_call=2, wait_job_after=0)
    assert R.phase == A.FAILED and "injected" in R.policy.error
    assert R.cur is R.default
    check_state(R, case, 8)
    R.close()


def test_application_ends_before_the_job(case):
    R = make(case, job_test=E.JOB_TEST_HOLD)
    drive(R, calls=3, per_call=2)
    assert R.phase == A.DEFAULT and R.cur is R.default
    check_state(R, case, 6)
    R.close()  # stops the partition thread
    assert R.job is None
