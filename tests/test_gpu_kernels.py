"""GPU parity of each kernel of the hot path against the FP64 oracle, through
the C ABI: Philox Gaussian stream, TT matvec, Khatri-Rao sketch, TT inner
product, FP64 Householder QR, sketched least squares and randomized rounding.

Tolerances: FP64 mode 1e-12 relative per kernel; FP32 mode 2e-5 relative
(float32 accumulation over at most a few thousand terms); TF32 mode 3e-5: the
tensor-core matvec splits each operand into two TF32 parts and keeps three
products, so each product carries at most about 2^-20 relative error (plain
TF32 would be 2^-11 = 4.9e-4) before the same float32 accumulation."""
import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import tt as ott, rounding as ornd, solvers as osol, philox as oph, closed_forms as cf

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 2e-5
TF32_TOL = 3e-5   # split TF32 (hi*hi + lo*hi + hi*lo) with FP32 accumulation
BF16_TOL = 1e-4   # split BF16: bf16 hi + lo (8 + 8 significant bits), ~2^-17 per product


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


def tol_of(g, mode):
    return {0: F64_TOL, 1: F32_TOL, 2: TF32_TOL, 3: BF16_TOL}[mode]


def tt_rel_diff(a_cores, b_cores):
    """||a - b|| / ||b|| in exact TT arithmetic (oracle)."""
    diff = ott.add([(1.0, a_cores), (-1.0, b_cores)])
    return ott.norm(ott.left_orthogonalize(diff)) / ott.norm(b_cores)


def test_gaussian_stream_matches_oracle(g):
    for seed, stream, count in [(0, 1024, 1000), (7, 3, 4097), (2**40 + 5, 2**33 + 1, 33)]:
        dev = g.tt_gaussian(count, seed, stream, std=0.5, mode=g.MODE_FP64).cpu().numpy()
        ref = oph.gaussian(count, seed, stream, std=0.5)
        assert np.max(np.abs(dev - ref)) <= 1e-13 * np.max(np.abs(ref))
    f32 = g.tt_gaussian(100, 3, 9, mode=g.MODE_FP32).cpu().numpy()
    assert np.allclose(f32, oph.gaussian(100, 3, 9), rtol=1e-6, atol=1e-6)
    assert g.tt_gaussian(0, 1, 1).numel() == 0


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("d,n,ranks", [(2, 70, [1, 67, 1]), (3, 17, [1, 5, 66, 1]),
                                       (4, 9, [1, 1, 3, 2, 1]), (1, 5, [1, 1])])
def test_matvec_parity(g, mode, d, n, ranks):
    M = ti.laplacian_1d(n) + 10 * ti.central_difference_1d(n)
    op = ti.kron_sum_operator([M] * d)
    # a dense random operator core in the middle exercises every operator entry
    if d >= 3:
        op[1] = np.random.default_rng(1).standard_normal(op[1].shape)
    x = ti.random_tt([n] * d, ranks, seed=2)
    ref = ott.matvec(op, x)
    y = g.tt_matvec(g.op_to_device(op, g.mode_dtype(mode)), dev_tt(g, x, mode), mode=mode)
    assert y.ranks == ott.ranks(ref)
    for a, b in zip(y.numpy(), ref):
        assert rel_err(a, b) <= tol_of(g, mode)


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("d,n,ranks", [(3, 64, [1, 64, 37, 1]), (3, 16, [1, 5, 100, 1]),
                                       (4, 32, [1, 1, 3, 130, 1]), (2, 128, [1, 9, 1]),
                                       (3, 12, [1, 7, 3, 1])])
def test_matvec_parity_tensor_cores(g, mode, d, n, ranks):
    # n a multiple of 4 takes the tcgen05 path in TF32 mode (two N tiles when
    # the rank exceeds 64, two M tiles when n R > 128)
    M = ti.laplacian_1d(n) + 10 * ti.central_difference_1d(n)
    op = ti.kron_sum_operator([M] * d)
    op[1] = np.random.default_rng(3).standard_normal(op[1].shape)
    x = ti.random_tt([n] * d, ranks, seed=4)
    ref = ott.matvec(op, x)
    # mode 2 split TF32; mode 3 split BF16 (a 64-wide K chunk per step, so
    # n = 12 and 16 are one partial chunk and 128 two full ones)
    y = g.tt_matvec(g.op_to_device(op, torch.float32), dev_tt(g, x, mode), mode=mode)
    assert y.ranks == ott.ranks(ref)
    for a, b in zip(y.numpy(), ref):
        assert rel_err(a, b) <= tol_of(g, mode)


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_matvec_full_size_eigenvector(g, mode):
    # d=10, n=64 (the convection-diffusion workload's operator): A q = lambda q
    # exactly for a rank-1 tensor of eigenvectors; sampled entries are checked.
    d, n = 10, 64
    lam, V = cf.convdiff_eig(n)
    V = V / np.linalg.norm(V, axis=0)
    js = [0, 3, 63, 10, 31, 2, 5, 40, 12, 7]
    q = ti.rank_one_tt([V[:, j] for j in js])
    op = ti.kron_sum_operator([ti.laplacian_1d(n) + 10 * ti.central_difference_1d(n)] * d)
    y = g.tt_matvec(g.op_to_device(op, g.mode_dtype(mode)), dev_tt(g, q, mode), mode=mode)
    yc = y.numpy()
    mu = sum(lam[j] for j in js)
    rng = np.random.default_rng(0)
    scale = mu * np.prod([np.max(np.abs(V[:, j])) for j in js])
    for _ in range(50):
        idx = rng.integers(0, n, size=d)
        assert abs(ott.entry(yc, idx) - mu * ott.entry(q, idx)) <= 50 * tol_of(g, mode) * scale


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("s,ns,ranks", [(100, [16] * 4, [1, 4, 7, 3, 1]),
                                        (67, [70, 3, 65], [1, 65, 2, 1]),
                                        (1, [5, 5], [1, 2, 1])])
def test_sketch_parity(g, mode, s, ns, ranks):
    x = ti.random_tt(ns, ranks, seed=4)
    S = ti.khatri_rao_factors(ns, s, seed=5)
    ref = ott.sketch_kr_fast(x, S)
    out = g.tt_sketch(dev_tt(g, x, mode), [torch.as_tensor(f, dtype=g.mode_dtype(mode),
                                                           device="cuda") for f in S], mode=mode)
    assert rel_err(out.cpu().numpy(), ref) <= 10 * tol_of(g, mode)


def test_sketch_full_size_rank_one(g):
    ns = [64] * 10
    rng = np.random.default_rng(3)
    us = [rng.standard_normal(n) / 8 for n in ns]
    S = oph.sketch_factors(ns, 160, seed=0)
    expect = np.prod(np.stack([Sk @ u for Sk, u in zip(S, us)]), axis=0)
    out = g.tt_sketch(dev_tt(g, ti.rank_one_tt(us), 0),
                      [torch.as_tensor(f, device="cuda") for f in S], mode=0)
    assert rel_err(out.cpu().numpy(), expect) <= F64_TOL


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_dot_parity(g, mode):
    ns = [13, 64, 7, 30]
    x = ti.random_tt(ns, [1, 5, 70, 3, 1], seed=6)
    y = ti.random_tt(ns, [1, 2, 9, 65, 1], seed=7)
    ref = ott.dot(x, y)
    out = g.tt_dot(dev_tt(g, x, mode), dev_tt(g, y, mode), mode=mode).item()
    scale = ott.norm(x) * ott.norm(y)
    assert abs(out - ref) <= 10 * tol_of(g, mode) * scale


@pytest.mark.parametrize("m,l", [(1, 1), (70, 70), (4736, 74), (300, 17), (64, 64), (9000, 130),
                                 (17664, 138), (40, 33)])
def test_qr_f64(g, m, l):
    rng = np.random.default_rng(m + l)
    Y = rng.standard_normal((m, l))
    if l > 3:
        Y[:, 2] = Y[:, 1]  # exact rank deficiency: Q must stay orthonormal
    Yd = torch.as_tensor(Y, device="cuda")
    Q, R = g.tt_qr_f64(Yd)
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    assert np.max(np.abs(Q.T @ Q - np.eye(l))) <= 1e-13 * max(1, l)
    assert np.max(np.abs(Q @ R - Y)) <= 1e-13 * np.max(np.abs(Y)) * max(1, l)
    assert np.allclose(np.tril(R, -1), 0.0)
    Rn = np.linalg.qr(Y)[1]
    assert np.allclose(np.abs(np.diag(R))[:2], np.abs(np.diag(Rn))[:2], rtol=1e-12)
    # float32 input, float32 Q
    Qf, Rf = g.tt_qr_f64(Yd.float())
    Qf = Qf.cpu().double().numpy()
    assert np.max(np.abs(Qf.T @ Qf - np.eye(l))) <= 1e-6 * max(1, l)


@pytest.mark.parametrize("s,k", [(100, 1), (160, 80), (40, 40)])
def test_lstsq_parity(g, s, k):
    rng = np.random.default_rng(s + k)
    W = rng.standard_normal((s, k)) @ np.diag(np.logspace(0, -6, k))
    c = rng.standard_normal(s)
    y_ref, r_ref = osol.sketched_lstsq(W, c)
    y, r = g.tt_lstsq_f64(torch.as_tensor(W, device="cuda"), torch.as_tensor(c, device="cuda"))
    assert abs(r.item() - r_ref) <= 1e-10 * np.linalg.norm(c)
    assert rel_err(W @ y.cpu().numpy(), W @ y_ref) <= 1e-9


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_round_rand_identity_tol0(g, mode):
    ns = [6, 9, 5, 7]
    x = ti.random_tt(ns, [1, 3, 7, 4, 1], seed=8)
    xd = dev_tt(g, x, mode)
    drm = ti.gaussian_drm(ns, [1, 40, 40, 40, 1], seed=9)
    y = g.tt_round_rand([xd, xd, xd], [1.0, 1.0, -1.0], 0.0, 40, 10,
                        drm=[torch.as_tensor(c, dtype=g.mode_dtype(mode), device="cuda") for c in drm],
                        mode=mode)
    assert tt_rel_diff(y.numpy(), x) <= 10 * tol_of(g, mode)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("eps,rmax,p", [(1e-6, 30, 10), (1e-2, 30, 5), (0.0, 4, 3), (1e-8, 2, 0)])
def test_round_rand_parity_same_drm(g, mode, eps, rmax, p):
    ns = [8, 70, 5, 9]
    terms = [(0.7, ti.random_tt(ns, [1, 4, 9, 5, 1], seed=10)),
             (-1.3, ti.random_tt(ns, [1, 3, 12, 2, 1], seed=11))]
    L = [1, rmax + p, rmax + p, rmax + p, 1]
    drm = ti.gaussian_drm(ns, L, seed=12)
    # FP64 mode truncates bond by bond (TT-SVD sweep); the float modes truncate
    # all bonds from the same tensor (the oracle's "simultaneous" reading)
    trunc = "sequential" if mode == 0 else "simultaneous"
    ref = ornd.rto_round(terms, drm, eps=eps, rmax=rmax, oversample=p, truncation=trunc)
    y = g.tt_round_rand([dev_tt(g, X, mode) for _, X in terms], [a for a, _ in terms], eps, rmax, p,
                        drm=[torch.as_tensor(c, dtype=g.mode_dtype(mode), device="cuda") for c in drm],
                        mode=mode)
    assert y.ranks == ott.ranks(ref)
    # the represented tensors agree (cores may differ by orthogonal factors)
    tol = 1e-10 if mode == 0 else 1e-4
    assert tt_rel_diff(y.numpy(), ref) <= tol
    if mode == 0:
        # cores 2..d right-orthogonal after the sequential sweep
        for c in y.numpy()[1:]:
            Mx = c.reshape(c.shape[0], -1)
            assert np.max(np.abs(Mx @ Mx.T - np.eye(Mx.shape[0]))) <= 1e-12


def test_round_rand_philox_drm_matches_oracle(g):
    ns = [5, 7, 6]
    terms = [(1.0, ti.random_tt(ns, [1, 5, 6, 1], seed=13)), (0.5, ti.random_tt(ns, [1, 4, 3, 1], seed=14))]
    rmax, p, seed = 3, 2, 77
    drm = oph.drm_cores(ns, [1, rmax + p, rmax + p, 1], seed)
    ref = ornd.rto_round(terms, drm, eps=0.0, rmax=rmax, oversample=p)
    y = g.tt_round_rand([dev_tt(g, X, 0) for _, X in terms], [a for a, _ in terms], 0.0, rmax, p,
                        seed=seed, mode=0)
    assert tt_rel_diff(y.numpy(), ref) <= 1e-10


def test_round_rand_full_size_sum_of_rank_ones(g):
    # d=10, n=64 sum whose exact TT rank is 6 at every bond: rounding at
    # tolerance 1e-10 must return rank 6 and the same tensor (checked on samples)
    d, n = 10, 64
    rng = np.random.default_rng(5)
    terms = [(float(rng.uniform(0.5, 2)), ti.rank_one_tt([rng.standard_normal(n) for _ in range(d)]))
             for _ in range(6)]
    y = g.tt_round_rand([dev_tt(g, X, 0) for _, X in terms], [a for a, _ in terms], 1e-10, 64, 10,
                        seed=3, mode=0)
    assert max(y.ranks) == 6
    yc = y.numpy()
    for _ in range(30):
        idx = rng.integers(0, n, size=d)
        ref = sum(a * ott.entry(X, idx) for a, X in terms)
        scale = sum(abs(a) * abs(ott.entry(X, idx)) for a, X in terms)
        assert abs(ott.entry(yc, idx) - ref) <= 1e-8 * scale


def test_bad_arguments_raise(g):
    x = dev_tt(g, ti.random_tt([4, 4], [1, 2, 1], seed=0), 0)
    with pytest.raises(g.TTError):
        g.tt_dot(x, dev_tt(g, ti.random_tt([4, 5], [1, 2, 1], seed=0), 0))
    with pytest.raises(g.TTError):
        g.tt_round_rand([x], [1.0], -1.0, 4, 2)


def test_round_rand_fp64_large_bond_identity(g):
    # a bond of 144 columns: the FP64 Jacobi SVD of the truncation keeps V in
    # global scratch (A and V together exceed shared memory); tolerance 0
    # must return the tensor
    ns = [12, 12, 12, 12]
    x = ti.random_tt(ns, [1, 12, 50, 12, 1], seed=41)
    X = g.TT.from_numpy(x)
    y = g.tt_round_rand([X, X, X], [1.0, 1.0, -1.0], 0.0, 150, 10, seed=3, mode=0)
    assert tt_rel_diff(y.numpy(), x) <= 1e-12


@pytest.mark.parametrize("m,l", [(33792, 264), (6000, 200)])
def test_qr_f64_wide_rows_in_global_memory(g, m, l):
    # row blocks too large for shared memory: the cooperative factorisation
    # keeps them in global memory (the exact residual check of a rank-128 TT
    # with a rank-8 right-hand side factorises 264 columns)
    rng = np.random.default_rng(m + l)
    Y = rng.standard_normal((m, l))
    Y[:, 5] = Y[:, 3]
    Yd = torch.as_tensor(Y, device="cuda")
    Q, R = g.tt_qr_f64(Yd)
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    assert np.max(np.abs(Q.T @ Q - np.eye(l))) <= 1e-13 * l
    assert np.max(np.abs(Q @ R - Y)) <= 1e-13 * np.max(np.abs(Y)) * l
    Qf, _ = g.tt_qr_f64(Yd.float())
    Qf = Qf.cpu().double().numpy()
    assert np.max(np.abs(Qf.T @ Qf - np.eye(l))) <= 1e-6 * l


@pytest.mark.parametrize("mode", [0, 1])
def test_sketch_factors_match_oracle_philox(g, mode):
    # the Khatri-Rao factors the solver draws (Philox streams 1024 + k,
    # variance s^(-1/d)) against the oracle's independent Philox + Box-Muller
    ns, s = [16, 5, 64, 9], 100
    S = g.tt_sketch_factors(ns, s, seed=7, mode=mode)
    ref = oph.sketch_factors(ns, s, seed=7)
    for a, b in zip(S, ref):
        assert a.shape == (s, b.shape[1])
        tol = 1e-13 if mode == 0 else 1e-6
        assert np.max(np.abs(a.double().cpu().numpy() - b)) <= tol * np.max(np.abs(b))
    with pytest.raises(g.TTError):
        g.tt_sketch_factors(ns, 0, seed=7, mode=mode)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("seed", [0, 1])
def test_round_rand_float_truncation_vs_sequential_tt_svd(g, mode, seed):
    # T = X + delta Y with X of TT rank 5 and a tail delta ||Y|| = 1e-3 ||X||:
    # at eps = 1e-2 both the float modes' rule (all bonds from one
    # left-orthogonal tensor, per-bond eps ||T|| / (d - 1)) and the oracle's
    # sequential TT-SVD (per-bond eps ||T|| / sqrt(d - 1)) keep rank 5 at every
    # bond, and each result lies within eps ||T|| of T, so the two lie within
    # 2 eps ||T|| of each other (plus FP32 rounding, well below 1e-5)
    ns = [12, 70, 8, 33]
    X = ti.random_tt(ns, [1, 5, 5, 5, 1], seed=60 + seed)
    Y = ti.random_tt(ns, [1, 3, 3, 3, 1], seed=70 + seed)
    delta = 1e-3 * ott.norm(X) / ott.norm(Y)
    terms = [(1.0, X), (delta, Y)]
    eps, rmax, p = 1e-2, 20, 4
    drm = ti.gaussian_drm(ns, [1] + [rmax + p] * 3 + [1], seed=80 + seed)
    ref = ornd.rto_round(terms, drm, eps=eps, rmax=rmax, oversample=p, truncation="sequential")
    y = g.tt_round_rand([dev_tt(g, c, mode) for _, c in terms], [a for a, _ in terms], eps, rmax,
                        p, drm=[torch.as_tensor(c, dtype=torch.float32, device="cuda")
                                for c in drm], mode=mode)
    assert y.ranks == ott.ranks(ref) == [1, 5, 5, 5, 1]
    T = ott.add(terms)
    assert tt_rel_diff(y.numpy(), T) <= eps + 1e-5
    assert tt_rel_diff(y.numpy(), ref) <= 2 * eps + 1e-5



@pytest.mark.parametrize("mode", [1, 2])
def test_round_rand_float_truncation_wide_bond(g, mode):
    # Sketch rank l = 170 + 10 = 180 at both bonds: the FP64 Gram matrix (l^2
    # doubles) no longer fits in shared memory, so its Cholesky factor is formed
    # in global memory, and the Jacobi rotations V live in global scratch.  X has
    # TT rank 170 (Gaussian cores: singular values within ~15x of each other),
    # the tail delta ||Y|| = 1e-4 ||X|| lies below eps ||T|| / (d - 1) = 5e-4 ||T||,
    # so both truncation rules keep rank 170 and agree within 2 eps
    ns = [220, 3, 220]
    X = ti.random_tt(ns, [1, 170, 170, 1], seed=64)
    Y = ti.random_tt(ns, [1, 10, 10, 1], seed=65)
    delta = 1e-4 * ott.norm(X) / ott.norm(Y)
    terms = [(1.0, X), (delta, Y)]
    eps, rmax, p = 1e-3, 200, 10
    drm = ti.gaussian_drm(ns, [1, rmax + p, rmax + p, 1], seed=66)
    ref = ornd.rto_round(terms, drm, eps=eps, rmax=rmax, oversample=p, truncation="sequential")
    y = g.tt_round_rand([dev_tt(g, c, mode) for _, c in terms], [a for a, _ in terms], eps, rmax,
                        p, drm=[torch.as_tensor(c, dtype=torch.float32, device="cuda")
                                for c in drm], mode=mode)
    assert y.ranks == ott.ranks(ref) == [1, 170, 170, 1]
    T = ott.add(terms)
    assert tt_rel_diff(y.numpy(), T) <= eps + 1e-5
    assert tt_rel_diff(y.numpy(), ref) <= 2 * eps + 1e-5

def test_tf32_contractions_ragged_ranks(g):
    # TF32 mode runs the sketch steps, Gram sweeps and the rounding's
    # contractions on the tcgen05 grouped GEMM (split TF32, FP32 accumulation)
    # once a problem is large enough: ragged bond ranks 1, 9, 65, 74, 130 give
    # partial tiles in every dimension, transposed problems and split-K
    ns = [16, 32, 8, 64, 12]
    ranks = [1, 9, 65, 74, 130, 1]
    x = ti.random_tt(ns, ranks, seed=90)
    y = ti.random_tt(ns, [1, 12, 70, 66, 9, 1], seed=91)
    X, Y = dev_tt(g, x, 2), dev_tt(g, y, 2)
    S = ti.khatri_rao_factors(ns, 160, seed=92)
    out = g.tt_sketch(X, [torch.as_tensor(f, dtype=torch.float32, device="cuda") for f in S],
                      mode=2)
    assert rel_err(out.cpu().numpy(), ott.sketch_kr_fast(x, S)) <= 10 * TF32_TOL
    dv = g.tt_dot(X, Y, mode=2).item()
    assert abs(dv - ott.dot(x, y)) <= 10 * TF32_TOL * ott.norm(x) * ott.norm(y)
    drm = ti.gaussian_drm(ns, [1, 80, 80, 80, 80, 1], seed=93)
    terms = [(1.0, x), (-0.5, y)]
    ref = ornd.rto_round(terms, drm, eps=1e-6, rmax=70, oversample=10,
                         truncation="simultaneous")
    r = g.tt_round_rand([X, Y], [1.0, -0.5], 1e-6, 70, 10,
                        drm=[torch.as_tensor(c, dtype=torch.float32, device="cuda") for c in drm],
                        mode=2)
    assert r.ranks == ott.ranks(ref)
    assert tt_rel_diff(r.numpy(), ref) <= 1e-4
