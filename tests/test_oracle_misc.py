"""Pins of the Philox generator (published known-answer vectors), the
Gaussian streams (moments), the closed-form eigenpairs (against LAPACK) and
the dense adjoint gradients (against central finite differences)."""
import os

import numpy as np
import pytest

import ttinputs as ti
from oracle import philox, closed_forms as cf, adjoint, tt

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(v, 16) for v in line.split()])
    rows = np.array(rows, dtype=np.uint64)
    out = philox.philox4x32_10(rows[:, 0:4], rows[:, 4:6])
    assert np.array_equal(out.astype(np.uint64), rows[:, 6:10])


def test_gaussian_stream_moments_and_independence():
    g = philox.gaussian(400000, seed=7, stream=3)
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1.0) < 0.01
    assert abs(np.mean(g ** 4) - 3.0) < 0.05
    h = philox.gaussian(400000, seed=7, stream=4)
    assert abs(np.corrcoef(g, h)[0, 1]) < 0.01
    # prefix property: a stream does not depend on how many elements are drawn
    assert np.array_equal(philox.gaussian(10, 7, 3), g[:10])


def test_sketch_factor_variance():
    S = philox.sketch_factors([64] * 4, 200, seed=0)
    v = np.var(np.concatenate([s.ravel() for s in S]))
    assert abs(v - 200.0 ** (-1 / 4)) < 0.02 * 200.0 ** (-1 / 4)


@pytest.mark.parametrize("n", [5, 16, 64])
def test_laplacian_eigenpairs(n):
    lam, Q = cf.laplacian_eig(n)
    L = ti.laplacian_1d(n)
    assert np.allclose(np.sort(lam), np.linalg.eigvalsh(L), rtol=1e-12)
    assert np.allclose(L @ Q, Q * lam, atol=1e-9 * lam.max())
    assert np.allclose(Q.T @ Q, np.eye(n), atol=1e-12)


@pytest.mark.parametrize("n", [6, 64])
def test_convdiff_eigenpairs(n):
    lam, V = cf.convdiff_eig(n)
    M = ti.laplacian_1d(n) + 10 * ti.central_difference_1d(n)
    ref = np.sort(np.linalg.eigvals(M).real)
    assert np.allclose(np.sort(lam), ref, rtol=1e-9)
    Vn = V / np.linalg.norm(V, axis=0)
    assert np.max(np.abs(M @ Vn - Vn * lam)) < 1e-8 * np.max(np.abs(lam))


def test_kron_sum_dense_solve():
    # n = 4 would make L + 10 B defective (zero super-diagonal when n + 1 = 5)
    mats = [ti.laplacian_1d(6) + 10 * ti.central_difference_1d(6), ti.laplacian_1d(3)]
    b = np.random.default_rng(0).standard_normal(18)
    A = np.kron(mats[0], np.eye(3)) + np.kron(np.eye(6), mats[1])
    assert np.allclose(cf.kron_sum_solve_dense(mats, b), np.linalg.solve(A, b), rtol=1e-10)
    assert np.allclose(cf.kron_sum_apply_dense(mats, b), A @ b, rtol=1e-12)


def test_dense_adjoint_vs_finite_differences():
    d, n = 3, 5
    rng = np.random.default_rng(1)
    theta = rng.uniform(0.5, 2.0, size=d)
    L = ti.laplacian_1d(n)
    b = ti.random_tt([n] * d, [1, 2, 2, 1], seed=2)
    xt = ti.random_tt([n] * d, [1, 2, 2, 1], seed=3)
    loss, dth, dcores, _, _ = adjoint.loss_and_grads(theta, L, b, xt)
    h = 1e-5
    for k in range(d):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (adjoint.loss_and_grads(tp, L, b, xt)[0] - adjoint.loss_and_grads(tm, L, b, xt)[0]) / (2 * h)
        assert np.isclose(dth[k], fd, rtol=1e-5)
    for k in range(d):
        for idx in [(0, 1, 0), (b[k].shape[0] - 1, n - 1, b[k].shape[2] - 1)]:
            bp = [c.copy() for c in b]
            bm = [c.copy() for c in b]
            bp[k][idx] += h
            bm[k][idx] -= h
            fd = (adjoint.loss_and_grads(theta, L, bp, xt)[0]
                  - adjoint.loss_and_grads(theta, L, bm, xt)[0]) / (2 * h)
            assert np.isclose(dcores[k][idx], fd, rtol=1e-5, atol=1e-9)


def test_tt_dot_grad_matches_dense_and_fd():
    # the TT restatement against the dense gradient of <X, Y> (interfaces of y
    # built from full tensors) and against central differences
    ns = [3, 4, 2, 3]
    x = ti.random_tt(ns, [1, 2, 3, 2, 1], seed=11)
    y = ti.random_tt(ns, [1, 3, 2, 2, 1], seed=12)
    G = adjoint.dot_grad(x, y)
    X = tt.full(x)
    for k in range(len(ns)):
        left = np.ones((1, 1))
        for c in y[:k]:
            left = (left @ c.reshape(c.shape[0], -1)).reshape(-1, c.shape[2])
        right = np.ones((1, 1))
        for c in reversed(y[k + 1:]):
            right = (c.reshape(-1, c.shape[2]) @ right.T).reshape(c.shape[0], -1).T
        Xk = X.reshape(left.shape[0], ns[k], right.shape[0])
        dense = np.einsum("xiy,xa,yc->aic", Xk, left, right)
        assert np.allclose(G[k], dense, atol=1e-12)
    h = 1e-6
    for k, idx in [(0, (0, 1, 2)), (2, (1, 0, 1)), (3, (1, 2, 0))]:
        yp = [c.copy() for c in y]
        ym = [c.copy() for c in y]
        yp[k][idx] += h
        ym[k][idx] -= h
        fd = (tt.dot(x, yp) - tt.dot(x, ym)) / (2 * h)
        assert np.isclose(G[k][idx], fd, rtol=1e-7, atol=1e-10)


def test_tt_local_dots_match_dense_mode_products():
    ns = [4, 3, 5]
    x = ti.random_tt(ns, [1, 2, 3, 1], seed=13)
    y = ti.random_tt(ns, [1, 3, 2, 1], seed=14)
    rng = np.random.default_rng(15)
    mats = [rng.standard_normal((n, n)) for n in ns]
    out = adjoint.local_dots(x, y, mats)
    X, Y = tt.full(x).reshape(ns), tt.full(y).reshape(ns)
    for k in range(3):
        MY = np.moveaxis(np.tensordot(mats[k], Y, axes=([1], [k])), 0, k)
        assert np.isclose(out[k], np.sum(X * MY), rtol=1e-12)
    # a Kronecker-sum term with M = identity gives <x, y> in every position
    ones = adjoint.local_dots(x, y, [np.eye(n) for n in ns])
    assert np.allclose(ones, tt.dot(x, y), rtol=1e-12)
