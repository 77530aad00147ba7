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
