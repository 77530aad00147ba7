"""Pins of the oracle's roundings: identities at tolerance 0, the TT-SVD error
bound ``||T - T~|| <= eps ||T||`` (Section 2.2), ranks equal to matrix ranks of
the unfoldings, the partial contractions against their dense definition, and
the randomized rounding against TT-SVD (a heuristic ratio only: the RTO error
bound is probabilistic, so that comparison is the one unpinned part)."""
import numpy as np
import pytest

import ttinputs as ti
from oracle import tt, rounding as rnd
from oracle import tt as ott


def unfolding_ranks(full, ns, tol=1e-10):
    out = []
    for mu in range(1, len(ns)):
        M = full.reshape(int(np.prod(ns[:mu])), -1)
        s = np.linalg.svd(M, compute_uv=False)
        out.append(int(np.sum(s > tol * s[0])))
    return out


def test_truncation_rank_rule():
    s = np.array([4.0, 2.0, 1.0, 0.5])
    assert rnd.truncation_rank(s, 0.0) == 4
    assert rnd.truncation_rank(s, 0.5) == 3
    assert rnd.truncation_rank(s, np.sqrt(1.25)) == 2
    assert rnd.truncation_rank(s, 10.0) == 1
    assert rnd.truncation_rank(s, 0.0, rmax=2) == 2


def test_tt_svd_identity_and_minimal_ranks():
    ns = [3, 4, 3, 2]
    x = ti.random_tt(ns, [1, 2, 3, 2, 1], seed=1)
    z = tt.add([(1.0, x), (1.0, x), (-1.0, x)])        # rank 3r representation
    y = rnd.tt_svd_round(z, eps=1e-12)
    assert np.allclose(tt.full(y), tt.full(x), atol=1e-13)
    assert tt.ranks(y)[1:-1] == unfolding_ranks(tt.full(x), ns)


@pytest.mark.parametrize("eps", [1e-1, 1e-3, 1e-6])
def test_tt_svd_error_bound(eps):
    ns = [4, 4, 4, 4]
    z = tt.add([(1.0, ti.random_tt(ns, [1, 3, 4, 3, 1], seed=s)) for s in range(4)])
    y = rnd.tt_svd_round(z, eps=eps)
    err = np.linalg.norm(tt.full(y) - tt.full(z))
    assert err <= eps * np.linalg.norm(tt.full(z)) * (1 + 1e-10)


def test_right_partial_contractions_dense():
    ns = [3, 2, 4, 3]
    X = ti.random_tt(ns, [1, 2, 3, 2, 1], seed=2)
    R = ti.gaussian_drm(ns, [1, 2, 2, 3, 1], seed=3)
    W = rnd.right_partial_contractions(X, R)

    def right_interface(cores, mu):
        # X_{>mu}: rows (i_{mu+1}..i_d), cols r_mu, built from the dense tail
        tail = cores[mu:]
        r = tail[0].shape[0]
        cols = []
        for a in range(r):
            e = [tail[0][a:a + 1]] + tail[1:]
            cols.append(tt.full(e))
        return np.stack(cols, axis=1)

    for mu in range(1, 4):
        expect = right_interface(X, mu).T @ right_interface(R, mu)
        assert np.allclose(W[mu], expect, atol=1e-13)


def test_rto_identity_at_tolerance_zero():
    ns = [4, 5, 3, 4, 3]
    x = ti.random_tt(ns, [1, 3, 4, 4, 2, 1], seed=4)
    terms = [(1.0, x), (1.0, x), (-1.0, x)]
    drm = ti.gaussian_drm(ns, [1, 40, 40, 40, 40, 1], seed=5)
    y = rnd.rto_round(terms, drm, eps=0.0, rmax=40, oversample=10)
    assert np.allclose(tt.full(y), tt.full(x), atol=1e-13 * np.linalg.norm(tt.full(x)))
    # cores 2..d right-orthogonal after the truncation sweep
    for c in y[1:]:
        M = c.reshape(c.shape[0], -1)
        assert np.allclose(M @ M.T, np.eye(M.shape[0]), atol=1e-12)


def test_rto_tolerance_and_rank_cap():
    ns = [4, 4, 4, 4]
    z = [(0.7, ti.random_tt(ns, [1, 3, 4, 3, 1], seed=s)) for s in range(3)]
    zf = sum(a * tt.full(X) for a, X in z)
    drm = ti.gaussian_drm(ns, [1, 50, 50, 50, 1], seed=6)
    for eps in (1e-2, 1e-6):
        y = rnd.rto_round(z, drm, eps=eps, rmax=50, oversample=10)
        # l >= representation rank here, so the sketch is exact and the
        # TT-SVD bound applies to the truncation sweep
        assert np.linalg.norm(tt.full(y) - zf) <= eps * np.linalg.norm(zf) * (1 + 1e-8)
    y = rnd.rto_round(z, drm, eps=0.0, rmax=2, oversample=2)
    assert max(tt.ranks(y)) <= 2


def test_rto_scale_of_drm_irrelevant():
    ns = [3, 4, 3]
    x = ti.random_tt(ns, [1, 3, 3, 1], seed=7)
    w = ti.random_tt(ns, [1, 2, 2, 1], seed=8)
    drm = ti.gaussian_drm(ns, [1, 4, 4, 1], seed=9)
    drm2 = [c * 7.5 for c in drm]
    a = rnd.rto_round([(1.0, x), (0.3, w)], drm, eps=0.0, rmax=2, oversample=1)
    b = rnd.rto_round([(1.0, x), (0.3, w)], drm2, eps=0.0, rmax=2, oversample=1)
    assert np.allclose(tt.full(a), tt.full(b), atol=1e-13)


@pytest.mark.parametrize("eps", [1e-1, 1e-3])
def test_rto_equals_tt_svd_when_the_sketch_rank_covers_the_tensor(eps):
    # sketch ranks l >= the sum's representation ranks: the randomized range
    # finder reproduces the sum exactly (the DRM contractions have full column
    # rank with probability one); with no singular value below the threshold
    # the truncation keeps it, and the result is the oracle's TT-SVD rounding
    # of the same tensor: same ranks, same tensor to rounding
    ns = [4, 5, 4, 3]
    z = [(0.7 - 0.3 * s, ti.random_tt(ns, [1, 3, 4, 2, 1], seed=20 + s)) for s in range(3)]
    drm = ti.gaussian_drm(ns, [1, 70, 70, 70, 1], seed=30)
    y = rnd.rto_round(z, drm, eps=eps, rmax=60, oversample=10)
    ref = rnd.tt_svd_round(tt.add(z), eps=eps, rmax=60)
    assert tt.ranks(y) == tt.ranks(ref)
    yf, rf = tt.full(y), tt.full(ref)
    assert np.linalg.norm(yf - rf) <= 1e-10 * np.linalg.norm(rf)


def test_rto_truncation_matches_tt_svd_across_a_spectral_gap():
    # T = X + delta Y with X of TT rank (3, 4, 2) and ||delta Y|| = 1e-8 ||X||,
    # rounded at eps = 1e-4: both truncation sweeps (right-to-left after the
    # randomized left sweep, and the oracle's left-to-right TT-SVD) drop exactly
    # the tail, so they keep X's ranks and agree to the size of the tail
    ns = [4, 5, 4, 3]
    X = ti.random_tt(ns, [1, 3, 4, 2, 1], seed=40)
    Y = ti.random_tt(ns, [1, 2, 3, 2, 1], seed=41)
    delta = 1e-8 * tt.norm(X) / tt.norm(Y)
    z = [(1.0, X), (delta, Y)]
    drm = ti.gaussian_drm(ns, [1, 70, 70, 70, 1], seed=42)
    y = rnd.rto_round(z, drm, eps=1e-4, rmax=60, oversample=10)
    ref = rnd.tt_svd_round(tt.add(z), eps=1e-4, rmax=60)
    assert tt.ranks(y) == tt.ranks(ref) == [1, 3, 4, 2, 1]
    yf, rf = tt.full(y), tt.full(ref)
    assert np.linalg.norm(yf - rf) <= 1e-7 * np.linalg.norm(rf)


def test_rto_vs_tt_svd_heuristic():
    # parity unpinned beyond this heuristic: randomized error within 10x of
    # the deterministic truncation error at equal rank, over 20 seeds
    ns = [6, 6, 6, 6]
    z = [(1.0, ti.random_tt(ns, [1, 4, 6, 4, 1], seed=s)) for s in range(3)]
    full = tt.add(z)
    zf = tt.full(full)
    ref = rnd.tt_svd_round(full, rmax=5)
    e_ref = np.linalg.norm(tt.full(ref) - zf)
    ratios = []
    for seed in range(20):
        drm = ti.gaussian_drm(ns, [1, 12, 12, 12, 1], seed=100 + seed)
        y = rnd.rto_round(z, drm, eps=0.0, rmax=5, oversample=5)
        ratios.append(np.linalg.norm(tt.full(y) - zf) / e_ref)
    assert np.median(ratios) < 10.0


@pytest.mark.parametrize("eps", [3e-1, 1e-1, 1e-3])
def test_simultaneous_truncation_error_bound_and_identity(eps):
    # the bond-by-bond telescoping bound: ||T - T~|| <= sum of dropped tails
    # <= eps ||T|| with per-bond threshold eps ||T|| / (d - 1)
    ns = [4, 5, 4, 3, 4]
    z = [(1.0, ti.random_tt(ns, [1, 4, 6, 5, 3, 1], seed=s)) for s in range(3)]
    X = ttm_left(tt.add(z))
    y = rnd.truncate_simultaneous(X, eps=eps)
    err = np.linalg.norm(tt.full(y) - tt.full(X))
    assert err <= eps * np.linalg.norm(tt.full(X)) * (1 + 1e-10)
    # tolerance 0: nothing is dropped
    y0 = rnd.truncate_simultaneous(X, eps=0.0)
    assert np.allclose(tt.full(y0), tt.full(X), atol=1e-12 * np.linalg.norm(tt.full(X)))
    # a small tolerance removes only the roundoff directions: the ranks become
    # the exact unfolding ranks (the Gram matrices resolve singular values down
    # to about sqrt(machine eps) of the largest, so 1e-6 is "small" here)
    y1 = rnd.truncate_simultaneous(X, eps=1e-6)
    assert tt.ranks(y1)[1:-1] == unfolding_ranks(tt.full(X), ns)


def ttm_left(cores):
    return tt.left_orthogonalize(cores)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_simultaneous_equals_sequential_tt_svd_with_a_spectral_gap(seed):
    # T = X + delta Y with X of TT rank 4 and delta ||Y|| = 1e-14 ||X||: every
    # bond spectrum has four singular values of order ||X|| and the rest below
    # 1e-13 of them.  A tolerance inside that gap makes the truncation rank 4
    # for both rules (each bond's threshold, eps ||T|| / (d - 1) for the
    # simultaneous rule and eps ||T|| / sqrt(d - 1) for the sequential TT-SVD,
    # lies far above the tail and far below the kept values), so the two must
    # keep the same ranks and the same tensor up to the dropped tail.
    rng = np.random.default_rng(seed)
    ns = [5, 6, 4, 7, 5]
    X = ti.random_tt(ns, [1, 4, 4, 4, 4, 1], seed=10 + seed)
    Y = ti.random_tt(ns, [1, 3, 3, 3, 3, 1], seed=20 + seed)
    delta = 1e-14 * ott.norm(X) / ott.norm(Y)
    T = ott.left_orthogonalize(ott.add([(1.0, X), (delta, Y)]))
    eps = 1e-8 * float(rng.uniform(0.5, 2.0))
    a = rnd.truncate_simultaneous(T, eps=eps)
    b = rnd.tt_svd_round(T, eps=eps)
    assert ott.ranks(a) == ott.ranks(b) == [1, 4, 4, 4, 4, 1]
    diff = ott.norm(ott.left_orthogonalize(ott.add([(1.0, a), (-1.0, b)])))
    assert diff <= 1e-12 * ott.norm(T)
    # and both are within the tolerance of T itself
    for c in (a, b):
        err = ott.norm(ott.left_orthogonalize(ott.add([(1.0, c), (-1.0, T)])))
        assert err <= eps * ott.norm(T)
