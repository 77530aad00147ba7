"""Pins of the oracle's STTA (Section 3.3): for d = 2 the recovery is the
generalized Nystrom approximation T X (Y^T T X)^+ Y^T T of the matrix T (the
textbook formula, written out here on the matrix); a TT whose ranks are at most
the target ranks is recovered exactly; the structured sketches equal their
dense definitions; sketches are linear in the tensor; d = 1 returns the vector.
"""
import numpy as np
import pytest

import ttinputs as ti
from oracle import tt, stta


def drms(ns, r, l, seed):
    d = len(ns)
    X = ti.gaussian_drm(ns, [1] + [r] * (d - 1) + [1], seed=seed)
    Y = ti.gaussian_drm(ns, [1] + [l] * (d - 1) + [1], seed=seed + 1)
    return X, Y


def test_interfaces_against_full_tensor():
    # the dense interfaces reproduce the full tensor: T = Y_{<=mu} Y_{>mu}^T
    ns = [3, 4, 2, 3]
    Y = ti.random_tt(ns, [1, 2, 3, 2, 1], seed=3)
    full = tt.full(Y).reshape(-1)
    for mu in range(1, 4):
        Yl = stta.left_interface(Y, mu)
        Yr = stta.right_interface(Y, mu)
        assert np.allclose(Yl @ Yr.T, full.reshape(Yl.shape[0], -1), atol=1e-13)


def test_d2_is_generalized_nystrom():
    n1, n2, r, l = 9, 7, 3, 5
    T = np.random.default_rng(4).standard_normal((n1, n2))
    X, Y = drms([n1, n2], r, l, seed=10)
    Psi, Omega = stta.sketch_dense(T, [n1, n2], X, Y)
    cores = stta.recover(Psi, Omega)
    approx = tt.full(cores).reshape(n1, n2)
    Xm = X[1][:, :, 0].T          # X_{>1}: n2 x r
    Ym = Y[0][0]                  # Y_{<=1}: n1 x l
    gn = (T @ Xm) @ np.linalg.pinv(Ym.T @ T @ Xm) @ (Ym.T @ T)
    assert np.allclose(approx, gn, atol=1e-12 * np.abs(T).max())


@pytest.mark.parametrize("ns,ranks", [([4, 5, 3, 4], [1, 2, 3, 2, 1]),
                                      ([3, 3, 3, 3, 3], [1, 3, 4, 4, 2, 1])])
def test_exact_recovery_of_low_rank_tt(ns, ranks):
    T = ti.random_tt(ns, ranks, seed=7)
    X = ti.gaussian_drm(ns, [1] + ranks[1:-1] + [1], seed=20)   # target ranks = T's ranks
    Y = ti.gaussian_drm(ns, [1] + [k + 2 for k in ranks[1:-1]] + [1], seed=21)
    Psi, Omega = stta.sketch(T, X, Y)
    cores = stta.recover(Psi, Omega)
    assert tt.ranks(cores) == ranks
    err = np.linalg.norm(tt.full(cores) - tt.full(T)) / np.linalg.norm(tt.full(T))
    assert err <= 1e-10, err


def test_structured_sketch_equals_definition():
    ns = [3, 4, 2, 3]
    T = ti.random_tt(ns, [1, 3, 4, 2, 1], seed=8)
    X, Y = drms(ns, 2, 4, seed=30)
    Pd, Od = stta.sketch_dense(tt.full(T), ns, X, Y)
    Ps, Os = stta.sketch(T, X, Y)
    for a, b in zip(Pd, Ps):
        assert a.shape == b.shape
        assert np.allclose(a, b, atol=1e-13 * max(1.0, np.abs(a).max()))
    for a, b in zip(Od, Os):
        assert np.allclose(a, b, atol=1e-13 * max(1.0, np.abs(a).max()))


def test_sketches_are_linear():
    ns = [3, 4, 3]
    A = ti.random_tt(ns, [1, 2, 3, 1], seed=9)
    B = ti.random_tt(ns, [1, 3, 2, 1], seed=10)
    X, Y = drms(ns, 2, 5, seed=40)
    Pd, Od = stta.sketch_dense(tt.full(A) * 0.7 - 1.3 * tt.full(B), ns, X, Y)
    Ps, Os = stta.sketch_sum([(0.7, A), (-1.3, B)], X, Y)
    for a, b in zip(Pd + Od, Ps + Os):
        assert np.allclose(a, b, atol=1e-13 * max(1.0, np.abs(a).max()))


def test_d1_returns_the_vector():
    v = np.random.default_rng(5).standard_normal(11)
    core = [v.reshape(1, 11, 1)]
    X = [np.ones((1, 11, 1))]
    Y = [np.ones((1, 11, 1))]
    Psi, Omega = stta.sketch(core, X, Y)
    assert Omega == []
    assert np.allclose(tt.full(stta.recover(Psi, Omega)), v, atol=0)


def test_rank_deficient_sketch_uses_the_cutoff():
    # target rank 4 above the tensor's rank 2: Omega is rank deficient; the
    # pseudo-inverse with its cutoff still recovers the tensor
    ns = [4, 5, 4]
    T = ti.random_tt(ns, [1, 2, 2, 1], seed=11)
    X, Y = drms(ns, 4, 7, seed=50)
    Psi, Omega = stta.sketch(T, X, Y)
    assert np.linalg.matrix_rank(Omega[0], tol=1e-10 * np.abs(Omega[0]).max()) == 2
    cores = stta.recover(Psi, Omega)
    err = np.linalg.norm(tt.full(cores) - tt.full(T)) / np.linalg.norm(tt.full(T))
    assert err <= 1e-9, err
