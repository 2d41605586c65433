"""Pins for the oracle's FP64 edge kernels, time stepping and adjoint (CPU only).

* Two-node closed form of the flux f = w (x_v - x_u) / (1 + |x_v - x_u|^2),
  hand-computed (tests/golden/flux_two_node.txt).
* Antisymmetry: every task adds f to u and -f to v, so sum_v out_v = 0.
* Task-order and orientation invariance.
* Small-state limit: f -> w (x_v - x_u), so out -> -L_w x with L_w the weighted
  graph Laplacian (scipy.sparse.csgraph.laplacian).
* SpMV: the bipartite data-affinity kernel of Section 5.2 equals
  scipy.sparse.csr_matrix @ x.
* Adjoint: central finite differences (h = 1e-3, FP64) on 64 random
  coordinates of the 4096-node mesh, and the dot-product identity.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import laplacian

import oracle as O
import workloads as W
from conftest import read_golden


def test_flux_two_node_closed_form():
    g = read_golden("flux_two_node.txt")
    xu = np.array(g["xu"][0], np.float64) / 4.0
    xv = np.array(g["xv"][0], np.float64) / 4.0
    w = g["w"][0][0] / 4.0
    fu = np.array(g["out_u"][0], np.float64) / 4.0
    x = np.stack([xu, xv], axis=1)
    out = O.flux([0], [1], x, [w])
    assert np.allclose(out[:, 0], fu, atol=0, rtol=1e-15)
    assert np.allclose(out[:, 1], -fu, atol=0, rtol=1e-15)


@pytest.fixture(scope="module")
def mesh():
    src, dst = W.knn_mesh(4096, 4, 0)
    x = W.flux_state(4096, 5, 0).astype(np.float64)
    w = W.flux_weights(src.size, 0).astype(np.float64)
    return src, dst, x, w


def test_flux_antisymmetry(mesh):
    src, dst, x, w = mesh
    out = O.flux(src, dst, x, w)
    assert np.abs(out.sum(axis=1)).max() < 1e-10
    assert np.abs(out).max() > 0.1


def test_flux_order_and_orientation_invariance(mesh):
    src, dst, x, w = mesh
    out = O.flux(src, dst, x, w)
    rng = np.random.default_rng(5)
    p = rng.permutation(src.size)
    flip = rng.random(src.size) < 0.5
    s2 = np.where(flip, dst, src)[p]
    d2 = np.where(flip, src, dst)[p]
    out2 = O.flux(s2, d2, x, w[p])
    assert np.allclose(out, out2, rtol=0, atol=1e-12)


def test_flux_small_state_is_laplacian(mesh):
    src, dst, _, w = mesh
    n = 4096
    eps = 1e-5
    x = eps * W.flux_state(n, 3, 4).astype(np.float64)
    A = sp.coo_matrix((w, (src, dst)), shape=(n, n))
    A = (A + A.T).tocsr()
    L = laplacian(A)
    out = O.flux(src, dst, x, w)
    ref = -(L @ x.T).T
    assert np.abs(out - ref).max() < 1e-6 * np.abs(ref).max()


def test_flux_steps_tau_zero_and_one_step(mesh):
    src, dst, x, w = mesh
    xT, out = O.flux_steps(src, dst, x, w, 3, 0.0)
    assert np.array_equal(xT, x)
    x1, out1 = O.flux_steps(src, dst, x, w, 1, 1e-3)
    assert np.allclose(x1, x + 1e-3 * O.flux(src, dst, x, w), rtol=0, atol=1e-15)


def test_spmv_matches_scipy():
    r, c = W.rmat(scale=10, m_draws=20000, seed=2)
    n = 1 << 10
    x, w = W.spmv_inputs(n, r.size, 0)
    y = O.spmv(r, c, x, w, n)
    A = sp.csr_matrix((w.astype(np.float64), (r, c)), shape=(n, n))
    assert np.allclose(y, A @ x.astype(np.float64), rtol=1e-13, atol=1e-13)


def test_adjoint_finite_differences(mesh):
    src, dst, x, w = mesh
    T, tau = 10, 1e-3
    g = W.loss_weights(4096, 5, 1)
    dx, dw = O.flux_adjoint(src, dst, x, w, T, tau, g)

    def loss(xx, ww):
        xT, _ = O.flux_steps(src, dst, xx, ww, T, tau)
        return float(np.sum(g * xT))

    rng = np.random.default_rng(2)
    h = 1e-3
    # the differenced loss carries float64 rounding of about eps |L| / h in
    # absolute terms: the check is |fd - adj| <= 1e-6 |adj| + 4 eps |L| / h
    ROUND = np.finfo(np.float64).eps * abs(loss(x, w)) / h
    errs = []
    for _ in range(32):
        c = int(rng.integers(0, 5))
        v = int(rng.integers(0, 4096))
        xp, xm = x.copy(), x.copy()
        xp[c, v] += h
        xm[c, v] -= h
        fd = (loss(xp, w) - loss(xm, w)) / (2 * h)
        errs.append(abs(fd - dx[c, v]) / (1e-6 * abs(dx[c, v]) + 4 * ROUND))
    for _ in range(32):
        e = int(rng.integers(0, src.size))
        wp, wm = w.copy(), w.copy()
        wp[e] += h
        wm[e] -= h
        fd = (loss(x, wp) - loss(x, wm)) / (2 * h)
        errs.append(abs(fd - dw[e]) / (1e-6 * abs(dw[e]) + 4 * ROUND))
    assert max(errs) <= 1.0, max(errs)


def test_adjoint_dot_product(mesh):
    # <J v, g> = <v, J^T g> for the linearised T-step map, via directional FD
    src, dst, x, w = mesh
    T, tau = 4, 1e-3
    g = W.loss_weights(4096, 5, 3)
    rng = np.random.default_rng(11)
    vx = rng.standard_normal(x.shape)
    vw = rng.standard_normal(w.shape)
    dx, dw = O.flux_adjoint(src, dst, x, w, T, tau, g)
    h = 1e-4
    xp, _ = O.flux_steps(src, dst, x + h * vx, w + h * vw, T, tau)
    xm, _ = O.flux_steps(src, dst, x - h * vx, w - h * vw, T, tau)
    jv = np.sum(g * (xp - xm)) / (2 * h)
    jtg = np.sum(vx * dx) + np.sum(vw * dw)
    assert abs(jv - jtg) < 1e-7 * abs(jtg)
