"""The multi-threaded FP64 CPU baseline (oracle/cpu_fair.c) against the
NumPy oracle: same steps to rounding, on several thread counts.  No GPU."""
import numpy as np
import pytest

import oracle as O
import workloads as W

if O.build_fair() is None:
    pytest.skip("no OpenMP compiler", allow_module_level=True)


@pytest.mark.parametrize("threads", [1, 3, 0])
@pytest.mark.parametrize("D", [1, 5, 8])
def test_fair_cpu_matches_oracle(threads, D):
    src, dst = W.knn_mesh(3000, 4, 2)
    src[:5] = dst[:5]  # self loops contribute nothing
    x0 = W.flux_state(3000, D, 1).astype(np.float64)
    w = W.flux_weights(src.size, 1)
    F = O.FairCpu(src, dst, 3000, D)
    x = x0.copy()
    out, used = F.steps(x, w, 3, 1e-2, threads)
    xT, fT = O.flux_steps(src, dst, x0, w, 3, 1e-2)
    assert used >= 1 and (threads == 0 or used == threads)
    np.testing.assert_allclose(x, xT, rtol=0, atol=1e-12)
    np.testing.assert_allclose(out, fT, rtol=0, atol=1e-12)
