"""GPU parity of the adjoint path (the differentiable solve): the backward
contractions against the oracle's TT restatements, the operator builder and
transpose against the input generator and the oracle, and the gradients of
``||x(theta, b) - x_t||^2`` against the oracle's dense gradient (tiny grids),
central finite differences of the library's own FP64 solves, and at the
differentiable workload's full size (d=12, n=64, FP32 contractions).

Tolerances: backward contractions 1e-12 (FP64) and 2e-5 (FP32) relative, the
same as the forward kernels; gradients 1e-6 relative against the dense oracle
with FP64 solves at tol 1e-12, and 1e-4 against finite differences (the bar the
differentiable workload sets)."""
import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import tt as ott, adjoint as oadj

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_09471_gb300 as g
    return g


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


TOL = {0: 1e-12, 1: 2e-5}


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("ns,rx,ry", [([5, 6, 4, 3], [1, 3, 7, 2, 1], [1, 2, 5, 4, 1]),
                                      ([9], [1, 1], [1, 1]),
                                      ([16, 16, 16], [1, 40, 33, 1], [1, 4, 70, 1])])
def test_dot_grad_parity(g, mode, ns, rx, ry):
    x = ti.random_tt(ns, rx, seed=21)
    y = ti.random_tt(ns, ry, seed=22)
    dt = g.mode_dtype(mode)
    out = g.tt_dot_grad(g.TT.from_numpy(x, dt), g.TT.from_numpy(y, dt), mode=mode)
    ref = oadj.dot_grad(x, y)
    for a, b in zip(out, ref):
        assert a.shape == b.shape
        assert rel(a.double().cpu().numpy(), b) <= TOL[mode]


@pytest.mark.parametrize("mode", [0, 1])
def test_local_dots_parity(g, mode):
    ns = [7, 5, 8, 6]
    x = ti.random_tt(ns, [1, 4, 9, 3, 1], seed=23)
    y = ti.random_tt(ns, [1, 2, 6, 5, 1], seed=24)
    rng = np.random.default_rng(25)
    mats = [rng.standard_normal((n, n)) for n in ns]
    dt = g.mode_dtype(mode)
    out = g.tt_local_dots(g.TT.from_numpy(x, dt), g.TT.from_numpy(y, dt),
                          [torch.as_tensor(m, dtype=dt, device="cuda") for m in mats], mode=mode)
    ref = oadj.local_dots(x, y, mats)
    scale = ott.norm(x) * ott.norm(y) * max(np.linalg.norm(m, 2) for m in mats)
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 10 * TOL[mode] * scale


@pytest.mark.parametrize("d", [1, 2, 5])
def test_kron_sum_op_and_transpose(g, d):
    n = 6
    rng = np.random.default_rng(26)
    theta = rng.uniform(0.5, 2.0, size=d)
    M = rng.standard_normal((n, n))
    ref = ti.kron_sum_operator([t * M for t in theta])
    Md = torch.as_tensor(M, device="cuda")
    op = g.tt_kron_sum_op([Md] * d, theta)
    for a, b in zip(op, ref):
        assert a.shape == b.shape
        assert np.allclose(a.cpu().numpy(), b, atol=1e-15, rtol=0)
    opT = g.tt_op_transpose(op)
    for a, b in zip(opT, ott.transpose_op(ref)):
        assert np.array_equal(a.cpu().numpy(), b)


SOLVE64 = dict(maxit=60, tol=1e-12, rmax=60, mode=0, s=120, stop_safety=0.01, r_sol=60,
               oversample=10, max_restarts=6)


def test_solve_loss_gradients_vs_dense_oracle(g):
    d, n = 3, 8
    rng = np.random.default_rng(27)
    theta = rng.uniform(0.5, 2.0, size=d)
    L = ti.laplacian_1d(n)
    b = ti.random_tt([n] * d, [1, 3, 2, 1], seed=28)
    xt = ti.random_tt([n] * d, [1, 2, 3, 1], seed=29)
    loss_ref, dth_ref, db_ref, _, _ = oadj.loss_and_grads(theta, L, b, xt)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    bc = [torch.as_tensor(c, device="cuda").requires_grad_(True) for c in b]
    xc = [torch.as_tensor(c, device="cuda").requires_grad_(True) for c in xt]
    loss = g.solve_loss(th, torch.as_tensor(L, device="cuda"), bc, xc, **SOLVE64)
    loss.backward()
    assert abs(loss.item() - loss_ref) <= 1e-8 * abs(loss_ref)
    assert rel(th.grad.numpy(), dth_ref) <= 1e-6
    for t, r in zip(bc, db_ref):
        assert rel(t.grad.cpu().numpy(), r) <= 1e-6
    # dL/dx_t = -2 (x - x_t) projected on x_t's cores: check one entry by FD of the dense loss
    k, idx, h = 1, (1, 3, 2), 1e-6
    xp = [c.copy() for c in xt]
    xm = [c.copy() for c in xt]
    xp[k][idx] += h
    xm[k][idx] -= h
    fd = (oadj.loss_and_grads(theta, L, b, xp)[0] - oadj.loss_and_grads(theta, L, b, xm)[0]) / (2 * h)
    assert np.isclose(xc[k].grad[idx].item(), fd, rtol=1e-5, atol=1e-9)


def test_solve_loss_at_the_solution_does_not_cancel(g):
    # x_t = the exact solution (dense solve, compressed by the oracle's TT-SVD):
    # the loss is ||x - x*||^2 for the FP64 solve at tol 1e-12 (relative error
    # <= kappa 1e-12, kappa ~ 32 here), far below the ~1e-16 ||x*||^2 that
    # <x,x> - 2 <x,x*> + <x*,x*> would leave, with either sign, after cancelling
    from oracle import closed_forms as cf, rounding as ornd
    d, n = 3, 8
    theta = np.array([0.7, 1.3, 1.9])
    L = ti.laplacian_1d(n)
    b = ti.random_tt([n] * d, [1, 3, 2, 1], seed=30)
    xs = cf.kron_sum_solve_dense([t * L for t in theta], ott.full(b))
    cores = [np.eye(n).reshape(1, n, n), np.eye(n * n).reshape(n, n, n * n),
             xs.reshape(n * n, n, 1)]
    xt = ornd.tt_svd_round(cores, 0.0)
    assert np.allclose(ott.full(xt), xs, rtol=0, atol=1e-13 * np.abs(xs).max())
    th = torch.tensor(theta, dtype=torch.float64)
    bc = [torch.as_tensor(c, device="cuda") for c in b]
    xc = [torch.as_tensor(c, device="cuda") for c in xt]
    loss = g.solve_loss(th, torch.as_tensor(L, device="cuda"), bc, xc, **SOLVE64).item()
    assert 0.0 <= loss <= 1e-18 * float(np.sum(xs ** 2)), loss


def test_solve_loss_gradients_vs_finite_differences(g):
    # d=5, n=16: central differences of the library's own FP64 solves.  The
    # solutions are capped at rank 60, which floors the true residual near 5e-8
    # here; with that floor a step of 1e-4 leaves ~1e-4 of noise in the
    # difference quotient (measured), so this check uses h = 1e-3 (truncation
    # error of the central difference near 1e-6 relative)
    d, n = 5, 16
    rng = np.random.default_rng(30)
    theta = rng.uniform(0.5, 2.0, size=d)
    Ld = torch.as_tensor(ti.laplacian_1d(n), device="cuda")
    b = [torch.as_tensor(c, device="cuda") for c in ti.random_tt([n] * d, [1, 3, 3, 3, 3, 1], seed=31)]
    # x_t on the solution's scale (1 / lambda_min of A), so the loss is sensitive to theta
    lam_min = theta.sum() * 4.0 * (n + 1) ** 2 * np.sin(np.pi / (2 * (n + 1))) ** 2
    xt_np = ti.random_tt([n] * d, [1, 2, 2, 2, 2, 1], seed=32)
    xt_np[0] = xt_np[0] / lam_min
    xt = [torch.as_tensor(c, device="cuda") for c in xt_np]
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    bc = [c.clone().requires_grad_(True) for c in b]
    loss = g.solve_loss(th, Ld, bc, xt, **SOLVE64)
    loss.backward()

    def f(thv, bcores):
        with torch.no_grad():
            return g.solve_loss(torch.tensor(thv, dtype=torch.float64), Ld, bcores, xt, **SOLVE64).item()

    h = 1e-3
    for k in (0, 3):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (f(tp, b) - f(tm, b)) / (2 * h)
        assert abs(th.grad[k].item() - fd) <= 1e-4 * abs(fd)
    k, idx = 2, (1, 5, 2)
    bp = [c.clone() for c in b]
    bm = [c.clone() for c in b]
    bp[k][idx] += h
    bm[k][idx] -= h
    fd = (f(theta, bp) - f(theta, bm)) / (2 * h)
    assert abs(bc[k].grad[idx].item() - fd) <= 1e-4 * abs(fd) + 1e-10


def test_differentiable_workload_full_size_fp32(g):
    # d=12, n=64, theta ~ U[0.5, 2], b and x_t random TT rank 4; forward and
    # adjoint solves in FP32 mode (FP64 refinement), asked for 1e-8; theta_1
    # against central differences (h = 1e-4) of FP64 solves at tol 1e-11
    # (measured agreement 2e-6 to 7e-6)
    w = ti.workload("differentiable")
    p = w.params
    theta = w.extra["theta"]
    Ld = torch.as_tensor(w.extra["L"], device="cuda")
    b = [torch.as_tensor(c, device="cuda") for c in w.b]
    xt = [torch.as_tensor(c, device="cuda") for c in w.extra["x_target"]]
    kw = dict(maxit=p["maxit"], tol=1e-8, rmax=p["rmax"], s=p["s"], r_sol=p["r_sol"],
              oversample=p["oversample"], stop_safety=0.1, max_restarts=8)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    loss = g.solve_loss(th, Ld, b, xt, mode=g.MODE_FP32, **kw)
    loss.backward()
    info = g.solve_loss.last
    assert info["last_info"]["true_res"] <= 2e-6
    assert info["last_adjoint_info"]["true_res"] <= 2e-6

    kw64 = dict(kw, mode=0, tol=1e-11)

    def f(thv):
        with torch.no_grad():
            return g.solve_loss(torch.tensor(thv, dtype=torch.float64), Ld, b, xt, **kw64).item()

    h = 1e-4
    for k in (0,):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (f(tp) - f(tm)) / (2 * h)
        assert abs(th.grad[k].item() - fd) <= 1e-4 * abs(fd)
