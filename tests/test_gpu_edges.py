"""Degenerate and mixed cases of the GPU path against the oracle or closed
forms: a TF32 matvec whose cores split between the tensor-core kernel (mode
size a multiple of 4) and the CUDA-core GEMM, a zero right-hand side, a right-
hand side that is an eigenvector (the Krylov space is exact after one step), the
rounding of a sum that cancels to zero, and a batch of one right-hand side."""
import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import tt as ott, solvers as osol, closed_forms as cf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_09471_gb300 as g
    return g


def test_tf32_matvec_mixed_core_paths(g):
    # n = 12 and 16 take the tensor-core kernel, n = 9 and 5 the CUDA-core GEMM
    ns = [12, 9, 16, 5]
    op = ti.kron_sum_operator([ti.laplacian_1d(n) + 10 * ti.central_difference_1d(n) for n in ns])
    x = ti.random_tt(ns, [1, 7, 66, 9, 1], seed=51)
    ref = ott.matvec(op, x)
    y = g.tt_matvec(g.op_to_device(op, torch.float32), g.TT.from_numpy(x, torch.float32), mode=2)
    for a, b in zip(y.numpy(), ref):
        assert np.linalg.norm(a - b) <= 3e-5 * np.linalg.norm(b)


def test_zero_right_hand_side_is_rejected(g):
    w = ti.workload("laplace_fp64", d=3, n=8)
    zero = [np.zeros_like(c) for c in w.b]
    with pytest.raises(g.TTError):
        g.tt_sgmres_solve(g.op_to_device(w.op), g.TT.from_numpy(zero), maxit=10, tol=1e-6, rmax=8)


@pytest.mark.parametrize("mode", [0, 1])
def test_eigenvector_right_hand_side_one_step(g, mode):
    # b = q (rank-1 tensor of eigenvectors): A q = mu q, so x = q / mu and the
    # Krylov space is exact after one step (h_{2,1} = 0 up to rounding); A is
    # symmetric positive definite, so ||x - q/mu|| <= ||b - A x|| / lambda_min(A)
    d, n = 4, 16
    lam, V = cf.laplacian_eig(n)
    js = [0, 3, 7, 1]
    q = ti.rank_one_tt([V[:, j] for j in js])
    mu = sum(lam[j] for j in js)
    op = ti.kron_sum_operator([ti.laplacian_1d(n)] * d)
    x, info = g.tt_sgmres_solve(g.op_to_device(op), g.TT.from_numpy(q), maxit=20, tol=1e-6,
                                rmax=8, mode=mode, s=40, stop_safety=0.01)
    assert info["status"] == 0 and info["cycles"] == 1
    # ||A q - h q|| is at the rounding level of h: the first step ends on a
    # breakdown (the Krylov space {q} is invariant under A)
    assert info["breakdowns"] == 1 and info["iters"] == 1
    r = osol.true_residual_norm(op, x.numpy(), q)
    err = np.linalg.norm(ott.full(x.numpy()) - ott.full(q) / mu)
    assert err <= 1.01 * r / (d * lam[0]) + 1e-15
    assert err <= 1e-5 / mu


@pytest.mark.parametrize("mode", [0, 1])
def test_rounding_of_a_cancelling_sum_is_zero(g, mode):
    ns = [6, 5, 7]
    x = ti.random_tt(ns, [1, 3, 4, 1], seed=52)
    X = g.TT.from_numpy(x, g.mode_dtype(mode))
    y = g.tt_round_rand([X, X], [1.0, -1.0], 1e-8, 10, 4, seed=2, mode=mode)
    for c in y.numpy():
        assert np.all(np.isfinite(c))
    nrm = ott.norm(y.numpy())
    assert nrm <= (1e-12 if mode == 0 else 1e-5) * ott.norm(x)


def test_batch_of_one_converges_like_single_solve(g):
    # one right-hand side through the worker pool (narrow QR plan, worker
    # stream) against the single-solve path: both reach the tolerance by the
    # oracle's exact residual, in nearly the same number of iterations
    w = ti.workload("convdiff", d=4, n=12, maxit=60)
    op = g.op_to_device(w.op)
    b = g.TT.from_numpy(w.b)
    kw = dict(maxit=60, tol=1e-6, rmax=64, mode=0, s=120, stop_safety=0.01, r_sol=64,
              oversample=10)
    (xb, ib), = g.tt_sgmres_solve_batched(op, [b], nworkers=4, **kw)
    xs, is_ = g.tt_sgmres_solve(op, b, **kw)
    assert ib["status"] == 0 and is_["status"] == 0
    for x, info in ((xb, ib), (xs, is_)):
        r = osol.true_residual_norm(w.op, x.numpy(), w.b) / ott.norm(w.b)
        assert r <= 1e-6
        assert abs(r - info["true_res"]) <= 1e-2 * r + 1e-14
    assert abs(ib["iters"] - is_["iters"]) <= 2


@pytest.mark.parametrize("mode,ell", [(0, 3), (2, 2)])
def test_partial_orthogonalisation(g, mode, ell):
    # each new vector orthogonalised against the last ell basis vectors
    # (Section 3.4): the restarted solve reaches the tolerance by the oracle's
    # exact FP64 residual
    w = ti.workload("convdiff", d=4, n=12, maxit=40)
    op = g.op_to_device(w.op)
    b = g.TT.from_numpy(w.b)
    x, info = g.tt_sgmres_solve(op, b, maxit=40, tol=1e-6, rmax=64, mode=mode, s=80,
                                stop_safety=0.01, r_sol=64, oversample=10, max_restarts=8,
                                ell=ell)
    assert info["status"] == 0, info
    r = osol.true_residual_norm(w.op, x.numpy(), w.b) / ott.norm(w.b)
    assert r <= 1e-6
    assert abs(r - info["true_res"]) <= 1e-2 * r + 1e-14
