"""Pins of the oracle's exact TT arithmetic against independent constructions:
Kronecker products built by ``np.kron``, dense matrix algebra, closed-form
eigenpairs of the 1-D model matrices, and the explicit Khatri-Rao sketch."""
import numpy as np
import pytest

import ttinputs as ti
from oracle import tt, closed_forms as cf


def kron_all(vs):
    out = np.ones(1)
    for v in vs:
        out = np.kron(out, v)
    return out


def dense_kron_sum(mats):
    """``sum_k I x .. x M_k x .. x I`` built with ``np.kron`` (mode 1 slowest)."""
    ns = [M.shape[0] for M in mats]
    N = int(np.prod(ns))
    A = np.zeros((N, N))
    for k, M in enumerate(mats):
        term = np.ones((1, 1))
        for j, n in enumerate(ns):
            term = np.kron(term, M if j == k else np.eye(n))
        A += term
    return A


def test_full_rank_one_is_kron():
    rng = np.random.default_rng(0)
    vs = [rng.standard_normal(n) for n in (3, 4, 2, 5)]
    assert np.allclose(tt.full(ti.rank_one_tt(vs)), kron_all(vs), rtol=0, atol=1e-14)


def test_full_sum_of_rank_ones():
    rng = np.random.default_rng(1)
    a = [rng.standard_normal(n) for n in (3, 4, 2)]
    b = [rng.standard_normal(n) for n in (3, 4, 2)]
    s = tt.add([(2.0, ti.rank_one_tt(a)), (-0.5, ti.rank_one_tt(b))])
    assert tt.ranks(s) == [1, 2, 2, 1]
    assert np.allclose(tt.full(s), 2.0 * kron_all(a) - 0.5 * kron_all(b), atol=1e-14)


def test_operator_cores_give_kron_sum():
    mats = [ti.laplacian_1d(3), ti.laplacian_1d(4) + 10 * ti.central_difference_1d(4),
            ti.central_difference_1d(2)]
    A = tt.op_full(ti.kron_sum_operator(mats))
    assert np.allclose(A, dense_kron_sum(mats), rtol=1e-15, atol=1e-12)
    assert np.allclose(tt.op_full(tt.transpose_op(ti.kron_sum_operator(mats))), A.T, atol=1e-12)


@pytest.mark.parametrize("d,n,ranks", [(1, 6, [1, 1]), (2, 5, [1, 3, 1]), (4, 3, [1, 2, 3, 2, 1])])
def test_matvec_matches_dense(d, n, ranks):
    mats = [ti.laplacian_1d(n) + 10 * ti.central_difference_1d(n)] * d
    op = ti.kron_sum_operator(mats)
    x = ti.random_tt([n] * d, ranks, seed=3)
    y = tt.matvec(op, x)
    R = [c.shape[0] for c in op] + [1]
    assert tt.ranks(y) == [a * b for a, b in zip(R, ranks)]  # ranks multiply
    assert np.allclose(tt.full(y), dense_kron_sum(mats) @ tt.full(x), rtol=1e-13, atol=1e-10)


def test_matvec_laplacian_eigenvector_any_size():
    # exact closed form A q = (sum lambda_j) q at a size with no dense form
    d, n = 10, 64
    lam, Q = cf.laplacian_eig(n)
    js = [1, 5, 63, 0, 17, 33, 2, 8, 40, 11]
    q = ti.rank_one_tt([Q[:, j] for j in js])
    op = ti.kron_sum_operator([ti.laplacian_1d(n)] * d)
    y = tt.matvec(op, q)
    mu = sum(lam[j] for j in js)
    rng = np.random.default_rng(0)
    for _ in range(20):
        idx = rng.integers(0, n, size=d)
        assert np.isclose(tt.entry(y, idx), mu * tt.entry(q, idx), rtol=1e-11,
                          atol=1e-12 * mu * np.max(np.abs(Q)) ** d)


def test_dot_matches_dense_and_orthonormality():
    x = ti.random_tt([4, 3, 5], [1, 2, 3, 1], seed=5)
    y = ti.random_tt([4, 3, 5], [1, 3, 1, 1], seed=6)
    assert np.isclose(tt.dot(x, y), tt.full(x) @ tt.full(y), rtol=1e-13)
    lam, Q = cf.laplacian_eig(16)
    a = ti.rank_one_tt([Q[:, 1], Q[:, 2], Q[:, 3], Q[:, 4]])
    b = ti.rank_one_tt([Q[:, 1], Q[:, 2], Q[:, 5], Q[:, 4]])
    assert abs(tt.dot(a, a) - 1.0) < 1e-13 and abs(tt.dot(a, b)) < 1e-13
    assert np.isclose(tt.norm(x), np.linalg.norm(tt.full(x)), rtol=1e-13)


def test_sketch_equals_explicit_khatri_rao():
    ns = [3, 4, 2, 3]
    x = ti.random_tt(ns, [1, 2, 3, 2, 1], seed=7)
    S = ti.khatri_rao_factors(ns, 9, seed=0)
    dense = tt.sketch_dense(tt.full(x), S)
    # explicit rows built with np.kron independently of sketch_dense
    rows = np.stack([kron_all([Sk[j] for Sk in S]) for j in range(9)])
    assert np.allclose(dense, rows @ tt.full(x), atol=1e-14)
    assert np.allclose(tt.sketch_kr(x, S), dense, rtol=1e-13, atol=1e-14)
    assert np.allclose(tt.sketch_kr_fast(x, S), dense, rtol=1e-13, atol=1e-14)


def test_sketch_rank_one_closed_form():
    rng = np.random.default_rng(2)
    ns = [64] * 10
    us = [rng.standard_normal(n) for n in ns]
    S = ti.khatri_rao_factors(ns, 40, seed=1)
    expect = np.prod(np.stack([Sk @ u for Sk, u in zip(S, us)]), axis=0)
    assert np.allclose(tt.sketch_kr_fast(ti.rank_one_tt(us), S), expect, rtol=1e-12)


def test_sketch_preserves_norm_in_expectation():
    # variance s^{-1/d} per entry gives E ||S x||^2 = ||x||^2 (Section 3.1)
    ns = [5, 5, 5]
    x = ti.random_tt(ns, [1, 2, 2, 1], seed=8)
    ratios = []
    for seed in range(400):
        S = ti.khatri_rao_factors(ns, 40, seed=seed)
        ratios.append(np.sum(tt.sketch_kr_fast(x, S) ** 2) / tt.norm(x) ** 2)
    assert abs(np.mean(ratios) - 1.0) < 0.1


def test_orthogonalize_keeps_tensor():
    x = ti.random_tt([3, 4, 5, 2], [1, 3, 4, 2, 1], seed=9)
    for f, side in ((tt.left_orthogonalize, "L"), (tt.right_orthogonalize, "R")):
        y = f(x)
        assert np.allclose(tt.full(y), tt.full(x), atol=1e-14)
        cores = y[:-1] if side == "L" else y[1:]
        for c in cores:
            r0, n, r1 = c.shape
            M = c.reshape(r0 * n, r1) if side == "L" else c.reshape(r0, n * r1).T
            assert np.allclose(M.T @ M, np.eye(M.shape[1]), atol=1e-13)


def test_bad_inputs_raise():
    x = ti.random_tt([3, 3], [1, 2, 1], seed=0)
    with pytest.raises(ValueError):
        tt.check_tt([x[0][:, :, :1], x[1]])
    with pytest.raises(ValueError):
        ti.random_tt([3, 3], [2, 2, 1], seed=0)


def test_tt_row_sketch_rank1_is_khatri_rao():
    # rank-1 rows are Khatri-Rao rows: the same factors give the same sketch
    ns = [4, 3, 5, 2]
    x = ti.random_tt(ns, [1, 2, 3, 2, 1], seed=21)
    S = ti.khatri_rao_factors(ns, 9, seed=22)
    Y = [Sk[:, None, :, None] for Sk in S]
    assert np.allclose(tt.sketch_tt_rows(x, Y), tt.sketch_kr(x, S), rtol=1e-13, atol=1e-15)


def test_tt_row_sketch_against_dense_rows():
    ns = [3, 4, 3]
    x = ti.random_tt(ns, [1, 2, 3, 1], seed=23)
    Y = ti.tt_row_sketch(ns, 7, 3, seed=24)
    assert np.allclose(tt.sketch_tt_rows(x, Y), tt.sketch_tt_rows_dense(tt.full(x), Y),
                       rtol=1e-12, atol=1e-14)


def test_tt_row_sketch_preserves_norms_in_expectation():
    # E ||S x||^2 = ||x||^2: the mean over 400 independent sketches is within
    # five standard errors of 1
    ns = [3, 3, 3, 3]
    x = ti.random_tt(ns, [1, 2, 2, 2, 1], seed=25)
    nx = tt.norm(x) ** 2
    r = np.array([np.sum(tt.sketch_tt_rows(x, ti.tt_row_sketch(ns, 4, 3, seed=100 + t)) ** 2) / nx
                  for t in range(400)])
    assert abs(r.mean() - 1.0) <= 5 * r.std() / np.sqrt(len(r))
