"""GPU parity at the large-rank workload's sizes (d = 20 modes of n = 128, the
Laplacian Kronecker sum, rank cap 128) and its full solve, through the C ABI.

d = 20 is past the 16 cores one tensor-core matvec launch takes, so the TF32
matvec runs in two launches; n = 128 gives operator slices of n R = 256 rows
(two M tiles).  Kernel parity is element by element against the FP64 oracle on
random inputs of small rank (cheap for the oracle) at the full d and n; the
full solve is checked with the oracle's exact FP64 residual.

Tolerances as in ``test_gpu_kernels``: FP64 1e-12, FP32 2e-5, split TF32 3e-5
relative per kernel."""
import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import tt as ott, rounding as ornd, solvers as osol

pytestmark = pytest.mark.gpu

D, N = 20, 128
TOL = {0: 1e-12, 1: 2e-5, 2: 3e-5}


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_09471_gb300 as g
    return g


def dev_tt(g, cores, mode):
    return g.TT.from_numpy(cores, dtype=g.mode_dtype(mode))


def rel_err(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def tt_rel_diff(a_cores, b_cores):
    diff = ott.add([(1.0, a_cores), (-1.0, b_cores)])
    return ott.norm(ott.left_orthogonalize(diff)) / ott.norm(b_cores)


def ragged_ranks(d, hi, seed):
    return ti.uneven_ranks(d, 1, hi, seed)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_matvec_parity_d20_n128(g, mode):
    # dense random operator cores at positions 1 (first launch) and 17 (second
    # launch of the tensor-core path) exercise every operator entry
    op = ti.kron_sum_operator([ti.laplacian_1d(N)] * D)
    rng = np.random.default_rng(21)
    for k in (1, 17):
        op[k] = rng.standard_normal(op[k].shape)
    x = ti.random_tt([N] * D, ragged_ranks(D, 12, 22), seed=23)
    ref = ott.matvec(op, x)
    y = g.tt_matvec(g.op_to_device(op, g.mode_dtype(mode)), dev_tt(g, x, mode), mode=mode)
    assert y.ranks == ott.ranks(ref)
    for k, (a, b) in enumerate(zip(y.numpy(), ref)):
        assert rel_err(a, b) <= TOL[mode], k


def test_matvec_tc_equals_fp32_d20_rank128(g):
    # the full basis rank: every core of the tensor-core result against the
    # FP32 CUDA-core result of the same inputs (both checked against the oracle
    # above at small rank); cores 0, 10 and 19 also against the oracle
    op = ti.kron_sum_operator([ti.laplacian_1d(N)] * D)
    x = ti.random_tt([N] * D, [1] + [128] * (D - 1) + [1], seed=24)
    opd = g.op_to_device(op, torch.float32)
    xd = dev_tt(g, x, 1)
    y2 = g.tt_matvec(opd, xd, mode=2).numpy()
    y1 = g.tt_matvec(opd, xd, mode=1).numpy()
    for k in range(D):
        assert rel_err(y2[k], y1[k]) <= 2 * TOL[2], k
    for k in (0, 10, 19):
        # the oracle's matvec works core by core: one core pair gives that core
        G = ott.matvec([op[k]], [x[k]])[0]
        assert rel_err(y2[k], G) <= TOL[2], k


@pytest.mark.parametrize("mode", [0, 1])
def test_sketch_parity_d20_n128(g, mode):
    from oracle import philox as oph
    x = ti.random_tt([N] * D, ragged_ranks(D, 12, 25), seed=26)
    S = oph.sketch_factors([N] * D, 200, seed=0)
    ref = ott.sketch_kr_fast(x, S)
    out = g.tt_sketch(dev_tt(g, x, mode), [torch.as_tensor(f, dtype=g.mode_dtype(mode),
                                                           device="cuda") for f in S], mode=mode)
    assert rel_err(out.cpu().numpy(), ref) <= 10 * TOL[mode]


@pytest.mark.parametrize("mode", [0, 1])
def test_dot_parity_d20_n128(g, mode):
    x = ti.random_tt([N] * D, ragged_ranks(D, 12, 27), seed=28)
    y = ti.random_tt([N] * D, ragged_ranks(D, 12, 29), seed=30)
    ref = ott.dot(x, y)
    out = g.tt_dot(dev_tt(g, x, mode), dev_tt(g, y, mode), mode=mode).item()
    assert abs(out - ref) <= 10 * TOL[mode] * ott.norm(x) * ott.norm(y)


@pytest.mark.parametrize("mode", [0, 1])
def test_round_rand_parity_d20_n128_same_drm(g, mode):
    terms = [(0.9, ti.random_tt([N] * D, ragged_ranks(D, 9, 31), seed=32)),
             (-0.4, ti.random_tt([N] * D, ragged_ranks(D, 9, 33), seed=34))]
    rmax, p, eps = 12, 6, 1e-3
    drm = ti.gaussian_drm([N] * D, [1] + [rmax + p] * (D - 1) + [1], seed=35)
    trunc = "sequential" if mode == 0 else "simultaneous"
    ref = ornd.rto_round(terms, drm, eps=eps, rmax=rmax, oversample=p, truncation=trunc)
    y = g.tt_round_rand([dev_tt(g, X, mode) for _, X in terms], [a for a, _ in terms], eps, rmax,
                        p, drm=[torch.as_tensor(c, dtype=g.mode_dtype(mode), device="cuda")
                                for c in drm], mode=mode)
    assert y.ranks == ott.ranks(ref)
    assert tt_rel_diff(y.numpy(), ref) <= (1e-10 if mode == 0 else 1e-4)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("n", [32, N])
def test_round_rand_d20_solver_steps(g, mode, n):
    # The solver's first two roundings Round(A v - h v) at d = 20, with the
    # DRM it draws (capacity ranks 138, entries of variance 1/(138 n 138)).
    # The right partial contractions of such a DRM shrink by about l/138^2 per
    # core, and the operator's cores mix entries of size (n+1)^2 with identity
    # blocks: the float modes must keep their precision over the 19 bonds.
    # Both sides round the same inputs: the device matvec A v (in a float mode
    # it carries the FP32 conditioning error of L applied to smooth vectors,
    # up to kappa(L) 2^-24 ~ 4e-4 at n = 128, which is the matvec's own error)
    # and v as the mode stores it.
    from oracle import philox as oph
    w = ti.workload("large_rank", n=n)
    op = w.op
    drm64 = oph.drm_cores(w.ns, [1] + [138] * (D - 1) + [1], 0)
    drm = [torch.as_tensor(c, dtype=g.mode_dtype(mode), device="cuda") for c in drm64]
    opd = g.op_to_device(op, g.mode_dtype(mode))
    v = ott.scale(w.b, 1.0 / ott.norm(w.b))
    tol = 1e-10 if mode == 0 else 1e-5
    for step, eps in enumerate((0.0, 1e-8)):
        V = dev_tt(g, v, mode)
        AV = g.tt_matvec(opd, V, mode=mode)
        av, vs = AV.numpy(), V.numpy()
        h = ott.dot(av, vs)
        ref = ornd.rto_round([(1.0, av), (-h, vs)], drm64, eps=eps, rmax=128, oversample=10,
                             truncation="sequential" if mode == 0 else "simultaneous")
        y = g.tt_round_rand([AV, V], [1.0, -h], eps, 128, 10, drm=drm, mode=mode)
        if mode == 0:
            assert y.ranks == ott.ranks(ref), step
        assert tt_rel_diff(y.numpy(), ref) <= tol, step
        v = ott.scale(ref, 1.0 / ott.norm(ref))


def solve_large_rank(g, mode, **over):
    w = ti.workload("large_rank")
    p = dict(w.params)
    p.update(over)
    x, info = g.tt_sgmres_solve(g.op_to_device(w.op), g.TT.from_numpy(w.b), maxit=p["maxit"],
                                tol=p["tol"], rmax=p["rmax"], mode=mode, s=p["s"], eta=p["eta"],
                                stop_safety=0.1, r_sol=p["r_sol"], oversample=p["oversample"],
                                seed=0, max_restarts=p.get("max_restarts", 8))
    return w, x, info


@pytest.mark.parametrize("mode", [1, 2])
def test_large_rank_full_solve(g, mode):
    # d = 20, n = 128, b random TT rank 8 (||b|| ~ 1), rank cap 128, m <= 100,
    # s = 200, oversampling 10, tol 1e-6; the residual is recomputed exactly by
    # the oracle in FP64 (about a minute on the host)
    w, x, info = solve_large_rank(g, mode)
    assert info["status"] == 0, info
    assert info["max_rank"] <= w.params["rmax"]
    assert max(x.ranks) <= w.params["r_sol"]
    res = osol.true_residual_norm(w.op, x.numpy(), w.b) / ott.norm(w.b)
    assert res <= 1e-6
    assert abs(res - info["true_res"]) <= 1e-2 * res
