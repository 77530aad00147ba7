"""GPU parity of the batched forms (row a9): the one-CTA-per-matrix FP64 QR
against the factorisation's defining properties and LAPACK, and batched solves
of many right-hand sides with uneven TT ranks against dense solves (small
grids) and the oracle's exact FP64 residual (the 64-RHS d=8, n=32 workload).

Tolerances: QR orthogonality and reconstruction 1e-13 x l (FP64) / 1e-6 x l
(float Q); solutions 1e-5 (FP64) / 1e-4 (FP32) relative to the dense solution,
true relative residual 1e-6 per right-hand side."""
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


def test_qr_batched_parity(g):
    shapes = [(1, 1), (70, 70), (1600, 50), (300, 17), (2048, 74), (40, 33)]
    Ys = []
    for m, l in shapes:
        Y = np.random.default_rng(m + 3 * l).standard_normal((m, l))
        if l > 3:
            Y[:, 2] = Y[:, 1]  # exact rank deficiency: Q must stay orthonormal
        Ys.append(Y)
    Yd = [torch.as_tensor(Y, device="cuda") for Y in Ys]
    Qs, Rs = g.tt_qr_f64_batched(Yd)
    for Y, Q, R in zip(Ys, Qs, Rs):
        l = Y.shape[1]
        Q, R = Q.cpu().numpy(), R.cpu().numpy()
        assert np.max(np.abs(Q.T @ Q - np.eye(l))) <= 1e-13 * max(1, l)
        assert np.max(np.abs(Q @ R - Y)) <= 1e-13 * np.max(np.abs(Y)) * max(1, l)
        assert np.allclose(np.tril(R, -1), 0.0)
        Rn = np.linalg.qr(Y)[1]
        assert np.allclose(np.abs(np.diag(R))[:2], np.abs(np.diag(Rn))[:2], rtol=1e-12)
    Qf, _ = g.tt_qr_f64_batched([y.float() for y in Yd])
    for Y, Q in zip(Ys, Qf):
        l = Y.shape[1]
        Q = Q.cpu().double().numpy()
        assert np.max(np.abs(Q.T @ Q - np.eye(l))) <= 1e-6 * max(1, l)


@pytest.mark.parametrize("mode", [0, 1])
def test_batched_small_vs_dense(g, mode):
    # d=4, n=8: rank cap 64 = n^2 holds every exact solution
    w = ti.workload("batched", d=4, n=8, nrhs=6)
    op = g.op_to_device(w.op)
    bs = [g.TT.from_numpy(b) for b in w.b]
    res = g.tt_sgmres_solve_batched(op, bs, maxit=40, tol=1e-6, rmax=64, mode=mode, s=80,
                                    round_tol=1e-8, stop_safety=0.01, r_sol=64, nworkers=4,
                                    max_restarts=8)
    L = ti.laplacian_1d(8)
    for b, (x, info) in zip(w.b, res):
        xd = cf.kron_sum_solve_dense([L] * 4, ott.full(b))
        err = np.linalg.norm(ott.full(x.numpy()) - xd) / np.linalg.norm(xd)
        assert info["status"] == 0 and info["true_res"] <= 1e-6
        assert err <= (1e-5 if mode == 0 else 1e-4)


def test_batched_workload_rhs_subset(g):
    # d=8, n=32 Laplacian, the first 8 of the 64 right-hand sides (bond ranks
    # U{1..12}), rank cap 150, TF32 mode (split-TF32 tensor-core matvec, FP64
    # QR / least squares / residual); every solution checked by the oracle's
    # exact FP64 residual, and one of them against the single-RHS solver
    w = ti.workload("batched")
    p = w.params
    op = g.op_to_device(w.op)
    sub = w.b[:8]
    bs = [g.TT.from_numpy(b) for b in sub]
    kw = dict(maxit=p["maxit"], tol=p["tol"], rmax=p["rmax"], mode=g.MODE_TF32, s=p["s"],
              round_tol=p["round_tol"], r_sol=p["r_sol"], oversample=p["oversample"],
              max_restarts=10)
    res = g.tt_sgmres_solve_batched(op, bs, nworkers=8, **kw)
    assert len(res) == 8
    for b, (x, info) in zip(sub, res):
        assert info["status"] == 0
        assert max(x.ranks) <= p["r_sol"]
        r = osol.true_residual_norm(w.op, x.numpy(), b) / ott.norm(b)
        assert r <= 1e-6
        assert abs(r - info["true_res"]) <= 1e-2 * r + 1e-14
    # two solutions with relative residual <= tol differ by at most
    # 2 kappa(A) tol relative (kappa of the 1-D Laplacian is that of the sum)
    x1, i1 = g.tt_sgmres_solve(op, bs[3], **kw)
    assert i1["status"] == 0
    n = 32
    kappa = (np.sin(n * np.pi / (2 * (n + 1))) / np.sin(np.pi / (2 * (n + 1)))) ** 2
    diff = ott.norm(ott.left_orthogonalize(ott.add([(1.0, x1.numpy()), (-1.0, res[3][0].numpy())])))
    assert diff <= 2 * kappa * p["tol"] * ott.norm(x1.numpy())


def test_batched_workload_all_64(g):
    # the whole batched workload: 64 right-hand sides (d = 8, n = 32, bond
    # ranks U{1..12}), rank cap 150, FP32 contractions, in one batched call.
    # Every solution's FP64 residual, computed exactly on the device, is at
    # most 1e-6; every fourth one is recomputed by the oracle (about 4 s each
    # on the host), which must agree to 1%.  The first cycle of the hardest
    # right-hand side (31) ends near 5e-6 in either float mode; after it the
    # solution sits at the rank cap, each restart residual is rounded to the
    # basis cap, and a cycle gains only part of its sketched reduction.  With
    # FP32 contractions it reached 9.4e-7 in 5 cycles on GB300; with the
    # split-TF32 matvec (about 2^-20 per product) it levelled off at 1.02e-6
    # (the subset test above keeps TF32 mode).
    w = ti.workload("batched")
    p = w.params
    op = g.op_to_device(w.op)
    bs = [g.TT.from_numpy(b) for b in w.b]
    assert len(bs) == 64
    res = g.tt_sgmres_solve_batched(op, bs, maxit=p["maxit"], tol=p["tol"], rmax=p["rmax"],
                                    mode=g.MODE_FP32, s=p["s"], round_tol=p["round_tol"],
                                    r_sol=p["r_sol"], oversample=p["oversample"],
                                    max_restarts=20, nworkers=16)
    bad = [(i, info["true_res"], info["cycles"], info["iters"]) for i, (_, info) in enumerate(res)
           if info["status"] != 0 or info["true_res"] > 1e-6]
    assert not bad, bad
    for x, _ in res:
        assert max(x.ranks) <= p["r_sol"]
    for i in range(0, 64, 4):
        x, info = res[i]
        r = osol.true_residual_norm(w.op, x.numpy(), w.b[i]) / ott.norm(w.b[i])
        assert r <= 1e-6, (i, r)
        assert abs(r - info["true_res"]) <= 1e-2 * r + 1e-14, (i, r, info["true_res"])
