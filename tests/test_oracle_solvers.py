"""Pins of the oracle's solvers: the least-squares step against the normal
equations and the SVD pseudo-inverse, and whole solves against dense
fast-diagonalisation solutions of the Kronecker-sum systems (closed form)."""
import numpy as np
import pytest

import ttinputs as ti
from oracle import tt, solvers, philox, closed_forms as cf


def test_sketched_lstsq_matches_pinv_and_normal_equations():
    rng = np.random.default_rng(0)
    W = rng.standard_normal((40, 7))
    c = rng.standard_normal(40)
    y, res = solvers.sketched_lstsq(W, c)
    assert np.allclose(y, np.linalg.solve(W.T @ W, W.T @ c), rtol=1e-10)
    assert np.allclose(y, np.linalg.pinv(W) @ c, rtol=1e-10)
    assert np.isclose(res, np.linalg.norm(W @ y - c))
    # exact fit when c is in the range
    y2, res2 = solvers.sketched_lstsq(W, W @ np.arange(7.0))
    assert np.allclose(y2, np.arange(7.0)) and res2 < 1e-12


def _setup(w, seed_s=0, seed_drm=1):
    p = w.params
    S = philox.sketch_factors(w.ns, p["s"], seed_s)
    ells = [1] + [p["rmax"] + p["oversample"]] * (w.d - 1) + [1]
    return S, philox.drm_cores(w.ns, ells, seed_drm)


def test_tt_sgmres_laplace_small_vs_dense():
    w = ti.workload("laplace_fp64", d=3, n=8)
    p = w.params
    S, drm = _setup(w)
    x, info = solvers.solve(w.op, w.b, S, drm, p["maxit"], 1e-8, 1e-10, p["rmax"],
                            p["oversample"])
    xd = cf.kron_sum_solve_dense([ti.laplacian_1d(8)] * 3, tt.full(w.b))
    A = tt.op_full(w.op)
    assert np.linalg.norm(A @ tt.full(x) - tt.full(w.b)) / np.linalg.norm(tt.full(w.b)) <= 1e-8
    assert np.linalg.norm(tt.full(x) - xd) / np.linalg.norm(xd) < 1e-7
    assert info["true_res"] <= 1e-8


def test_laplace_fp64_full_config_vs_closed_form():
    # d=4, n=16: the dense tensor (65536 entries) fits, so the fast
    # diagonalisation gives the exact solution
    w = ti.workload("laplace_fp64")
    p = w.params
    S, drm = _setup(w)
    x, info = solvers.solve(w.op, w.b, S, drm, p["maxit"], p["tol"], p["round_tol"], p["rmax"],
                            p["oversample"], stop_safety=0.01)
    xd = cf.kron_sum_solve_dense([ti.laplacian_1d(16)] * 4, tt.full(w.b))
    assert info["true_res"] <= p["tol"]
    assert np.linalg.norm(tt.full(x) - xd) / np.linalg.norm(xd) <= 1e-5
    assert info["cycles"][0]["iters"] <= p["maxit"]


def test_convdiff_small_sketched_vs_true_residual_gap():
    # the sketched residual tracks the true one within a factor 10 (Section 5.2.3)
    w = ti.workload("convdiff", d=4, n=12, maxit=60)
    p = w.params
    S, drm = _setup(w)
    x, info = solvers.tt_sgmres(w.op, w.b, S, drm, p["maxit"], 1e-6, 1e-8, p["rmax"],
                                p["oversample"], final_tol=1e-10)
    A = tt.op_full(w.op)
    bf = tt.full(w.b)
    true = np.linalg.norm(A @ tt.full(x) - bf) / np.linalg.norm(bf)
    sk = info["res_hist"][-1]
    assert true / sk < 10.0 and sk / true < 10.0
    M = ti.laplacian_1d(12) + 10 * ti.central_difference_1d(12)
    xd = cf.kron_sum_solve_dense([M] * 4, bf)
    assert np.linalg.norm(tt.full(x) - xd) / np.linalg.norm(xd) < 1e-3


def test_tt_gmres_reference_solver():
    w = ti.workload("convdiff", d=3, n=7, maxit=60)
    x, info = solvers.tt_gmres(w.op, w.b, 60, 1e-9, 1e-12)
    M = ti.laplacian_1d(7) + 10 * ti.central_difference_1d(7)
    xd = cf.kron_sum_solve_dense([M] * 3, tt.full(w.b))
    assert np.linalg.norm(tt.full(x) - xd) / np.linalg.norm(xd) < 1e-7


def test_true_residual_norm_exact():
    w = ti.workload("convdiff", d=3, n=6)
    x = ti.random_tt(w.ns, [1, 2, 2, 1], seed=11)
    A = tt.op_full(w.op)
    expect = np.linalg.norm(tt.full(w.b) - A @ tt.full(x))
    assert np.isclose(solvers.true_residual_norm(w.op, x, w.b), expect, rtol=1e-12)


def test_full_orthogonalisation_gives_arnoldi():
    # l = maxit and no truncation (RTO at tolerance 0 with the rank cap above
    # every representation rank is exact): the basis is orthonormal and
    # A v_k = sum_{i <= k+1} h_{i,k} v_i holds (the Arnoldi relation of
    # Section 3.4); with l = 1 the basis is not orthogonal
    w = ti.workload("convdiff", d=3, n=5, rank=2)
    ns = w.ns
    S = philox.sketch_factors(ns, 20, 0)
    drm = philox.drm_cores(ns, [1, 400, 400, 1], 1)
    A = tt.op_full(w.op)
    x, info = solvers.tt_sgmres(w.op, w.b, S, drm, 8, 1e-14, 0.0, 400, oversample=0, ell=8)
    V = np.array([tt.full(v) for v in info["V"]])
    k = info["iters"]
    assert np.abs(V @ V.T - np.eye(len(V))).max() <= 1e-10
    H = info["H"]
    for j in range(min(k, len(V) - 1)):
        lhs = A @ V[j]
        rhs = sum(H[i, j] * V[i] for i in range(j + 2))
        assert np.linalg.norm(lhs - rhs) <= 1e-10 * np.linalg.norm(lhs)
    _, info1 = solvers.tt_sgmres(w.op, w.b, S, drm, 8, 1e-14, 0.0, 400, oversample=0, ell=1)
    V1 = np.array([tt.full(v) for v in info1["V"]])
    assert np.abs(V1 @ V1.T - np.eye(len(V1))).max() > 1e-3


def test_partial_orthogonalisation_solves():
    # l = 3 on the small convection-diffusion system: the restarted solve
    # reaches the tolerance and matches the dense solution
    w = ti.workload("convdiff", d=3, n=8)
    p = w.params
    S, drm = _setup(w)
    x, info = solvers.solve(w.op, w.b, S, drm, 40, 1e-8, 1e-10, p["rmax"], p["oversample"],
                            ell=3, stop_safety=0.01)
    A = tt.op_full(w.op)
    xd = np.linalg.solve(A, tt.full(w.b))
    assert info["true_res"] <= 1e-8
    assert np.linalg.norm(tt.full(x) - xd) / np.linalg.norm(xd) <= 1e-6
