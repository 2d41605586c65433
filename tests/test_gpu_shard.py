"""A schedule split over G shards and run on one GPU, the halo sums exchanged
every step (GPU only).

Shard g runs its blocks as its own schedule with the halo declared; after
every step the shards' halo sums are summed on the device (the stand-in for
the all-reduce across GPUs) and written back.  The gathered state after T
steps must match the FP64 oracle's unsharded steps (parity.py bounds), and
the exchange must matter: without it the halo vertices go wrong.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1605_02043_gb300 as E  # noqa: E402
from paper_1605_02043_gb300.shard import ShardedFlux  # noqa: E402
from parity import check_state  # noqa: E402


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.mark.parametrize("n,C,G,stages", [(4096, 256, 2, 3), (4096, 128, 4, 0), (30000, 512, 8, 3),
                                          (30000, 256, 2, 2)])
def test_sharded_steps_match_oracle(n, C, G, stages):
    src, dst = W.knn_mesh(n, 4, 5)
    S = E.Schedule.partition(src, dst, n, C)
    x0 = W.flux_state(n, 5, 2)
    w = W.flux_weights(src.size, 2)
    T, tau = 4, 1e-3
    R = ShardedFlux(S, src, dst, n, 5, G)
    for Sg in R.S:
        Sg.set_pipeline(stages)
    assert R.halo.ids.size > 0
    R.load(cuda(x0), cuda(w))
    for _ in range(T):
        R.step(tau)
    R.finish(tau)
    x = R.gather(cuda(x0))
    xT, _ = O.flux_steps(src, dst, x0, w, T, tau)
    check_state(x, xT, x0, T, f"x (G={G})")
    for Sg in R.S:
        assert Sg.check_errors() == 0


def test_exchange_is_needed():
    n, C, G = 4096, 256, 2
    src, dst = W.knn_mesh(n, 4, 5)
    S = E.Schedule.partition(src, dst, n, C)
    x0 = W.flux_state(n, 5, 2)
    w = W.flux_weights(src.size, 2)
    R = ShardedFlux(S, src, dst, n, 5, G, reduce=lambda bufs: None)  # no exchange
    R.load(cuda(x0), cuda(w))
    R.step(1e-3)
    R.finish(1e-3)
    x = R.gather(cuda(x0)).cpu().numpy()
    xT, _ = O.flux_steps(src, dst, x0, w, 1, 1e-3)
    h = R.halo.ids
    interior = np.setdiff1d(np.arange(n), h)
    # after one step the vertices of one shard only are right; halo vertices
    # miss the other shards' sums
    err_i = np.abs(x[:, interior] - xT[:, interior]).max()
    err_h = np.abs(x[:, h] - xT[:, h]).max()
    assert err_i < 1e-5 and err_h > 1e-4, (err_i, err_h)
