"""Bounded waits of the pipelined kernels (GPU only).

The test hook ep_debug_stall leaves one stage of every persistent CUDA block
unfilled, so the consumers' wait for it runs out (nothing ever arrives on
that barrier).  No fault and no hang: the launch gives up after its wait
limit, sets the error word, and returns; ep_check_errors must report
EP_ETIMEOUT, and the same schedule must then run cleanly and match the
oracle, which shows the context and the schedule's state stayed usable.
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
from paper_1605_02043_gb300._lib import EpError  # noqa: E402

RTOL = 1e-5
EP_ETIMEOUT = -4


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.fixture(scope="module")
def mesh():
    # many more schedule blocks than persistent CUDA blocks, so every CUDA
    # block reaches the stalled stage index
    n = 1 << 16
    src, dst = W.knn_mesh(n, 4, 0)
    S = E.Schedule.partition(src, dst, n, 64)
    return n, src, dst, S


@pytest.mark.parametrize("stall", [0, 2])
def test_forward_wait_expires_then_recovers(mesh, stall):
    n, src, dst, S = mesh
    S.set_pipeline(3)
    x0 = W.flux_state(n, 5, 0)
    w = W.flux_weights(src.size, 0)
    S.debug_stall(stall)
    x = cuda(x0)
    S.run(x, cuda(w), None, steps=1, tau=1e-3)
    with pytest.raises(EpError) as ei:
        S.check_errors()
    assert ei.value.code == EP_ETIMEOUT
    assert S.check_errors() == 0  # reading the word clears it
    S.debug_stall(-1)
    x = cuda(x0)
    out = torch.zeros_like(x)
    S.run(x, cuda(w), out, steps=2, tau=1e-3)
    torch.cuda.synchronize()
    xT, fT = O.flux_steps(src, dst, x0, w, 2, 1e-3)
    assert rel_l2(x.cpu().numpy(), xT) <= RTOL
    assert rel_l2(out.cpu().numpy(), fT) <= RTOL
    assert S.check_errors() == 0


def test_adjoint_wait_expires_then_recovers(mesh):
    n, src, dst, S = mesh
    S.set_pipeline(3)
    x0 = W.flux_state(n, 5, 0)
    w = W.flux_weights(src.size, 0)
    g = W.loss_weights(n, 5, 1)
    S.debug_stall(1)
    lam = cuda(g)
    gw = torch.zeros(src.size, device="cuda")
    S.run_adjoint(cuda(x0), cuda(w), lam, gw, steps=1, tau=1e-3)
    with pytest.raises(EpError) as ei:
        S.check_errors()
    assert ei.value.code == EP_ETIMEOUT
    S.debug_stall(-1)
    lam = cuda(g)
    gw.zero_()
    S.run_adjoint(cuda(x0), cuda(w), lam, gw, steps=2, tau=1e-3)
    dx, dw = O.flux_adjoint(src, dst, x0, w, 2, 1e-3, g)
    assert rel_l2(lam.cpu().numpy(), dx) <= RTOL
    assert rel_l2(gw.cpu().numpy(), dw) <= RTOL
    assert S.check_errors() == 0
