"""Pins of the oracle's exponential-sum preconditioner and TT-sPGMRES
(Section 4, Algorithm 5): the sum against 1/z on its interval; P^{-1} by mode
products against the matrix exponential of the whole Kronecker sum (scipy
expm of the dense operator); the spectrum of P^{-1} A against the closed-form
Laplacian eigenvalues; and the preconditioned solve against a dense solve."""
import numpy as np
import pytest
import scipy.linalg as sla

import ttinputs as ti
from oracle import tt, precond as pc, philox, closed_forms as cf


@pytest.mark.parametrize("a,b", [(1.0, 100.0), (39.4, 1.1e4), (1.0, 1e6)])
@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-8])
def test_exp_sum_accuracy(a, b, tol):
    alpha, beta = pc.exp_sum_coefficients(a, b, tol)
    z = np.geomspace(a, b, 5000)
    assert np.abs(z * pc.exp_sum(z, alpha, beta) - 1.0).max() <= tol
    assert np.all(alpha > 0) and np.all(beta > 0)


def test_precond_is_the_exp_sum_of_the_kronecker_sum():
    # E(A_0) with A_0 the dense Kronecker sum, each exponential by scipy expm
    # of the whole n^d x n^d matrix, against the mode-product form
    ns = [4, 3, 5]
    mats = [ti.laplacian_1d(n) + 3.0 * ti.central_difference_1d(n) for n in ns]
    A0 = tt.op_full(ti.kron_sum_operator(mats))
    alpha, beta = pc.exp_sum_coefficients(20.0, 400.0, 1e-2)
    x = ti.random_tt(ns, [1, 2, 3, 1], seed=3)
    got = tt.full(pc.apply_precond(x, mats, alpha, beta))
    want = sum(a * (sla.expm(-bi * A0) @ tt.full(x)) for a, bi in zip(alpha, beta))
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    # a single mode product leaves the ranks unchanged
    assert tt.ranks(pc.mode_product(x, [np.eye(n) for n in ns])) == tt.ranks(x)


def test_preconditioned_spectrum():
    # A_0 = sum of 1-D Laplacians (symmetric): P^{-1} A_0 has eigenvalues
    # lambda E(lambda), within tol of 1 on the interval covering the spectrum
    d, n = 3, 6
    lam, _ = cf.laplacian_eig(n)
    a, b = d * lam[0], d * lam[-1]
    alpha, beta = pc.exp_sum_coefficients(a, b, 1e-2)
    L = ti.laplacian_1d(n)
    A0 = tt.op_full(ti.kron_sum_operator([L] * d))
    Pinv = sum(al * sla.expm(-bi * A0) for al, bi in zip(alpha, beta))
    ev = np.linalg.eigvals(Pinv @ A0)
    assert np.abs(ev - 1.0).max() <= 1e-2


def test_spgmres_solves_in_few_iterations():
    d, n = 3, 16
    w = ti.workload("laplace_fp64", d=d, n=n)
    lam, _ = cf.laplacian_eig(n)
    alpha, beta = pc.exp_sum_coefficients(d * lam[0], d * lam[-1], 1e-2)
    L = ti.laplacian_1d(n)
    S = philox.sketch_factors(w.ns, 40, 0)
    drm = philox.drm_cores(w.ns, [1, 60, 60, 1], 1)
    x, info = pc.tt_spgmres(w.op, w.b, [L] * d, alpha, beta, S, drm, 20, 1e-8, 1e-10, 50)
    xd = cf.kron_sum_solve_dense([L] * d, tt.full(w.b))
    assert info["iters"] <= 8
    assert np.linalg.norm(tt.full(x) - xd) / np.linalg.norm(xd) <= 1e-6
