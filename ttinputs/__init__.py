"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only *builds input data*: the 1-D matrices of the paper's model
problems, their rank-2 Kronecker-sum TT operators, random TT right-hand sides,
Gaussian Khatri-Rao sketch factors and Gaussian TT-DRM cores drawn with NumPy's
seeded generator.  It holds none of the solver's arithmetic (no contraction,
sketch, rounding, orthogonalisation or least-squares step) and imports neither
the oracle nor the CUDA package, so both sides can consume the same inputs.

Layouts (row-major, C order), used by every consumer:

* TT vector core k: ``[r_{k-1}, n_k, r_k]`` with ``r_0 = r_d = 1``
  (eq. ``tt-format``, Section 2.2).
* TT operator core k: ``[R_{k-1}, n_out, n_in, R_k]`` (eq. ``operator
  tt-format``, Section 2.2).
* Full-tensor index ``(i_1, ..., i_d)`` with ``i_1`` slowest, so the
  Kronecker-sum term with ``M`` in position k acts on mode k.
* Khatri-Rao sketch factor k: ``[s, n_k]`` (Section 3.1).
* TT-DRM core k: ``[l_{k-1}, n_k, l_k]`` (Definition "Random Gaussian
  TT-Tensor", Section 3.3).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "laplacian_1d",
    "central_difference_1d",
    "paper_convdiff_1d",
    "kron_sum_operator",
    "random_tt",
    "rank_one_tt",
    "khatri_rao_factors",
    "gaussian_drm",
    "uneven_ranks",
    "birth_death_generator",
    "markov_operator",
    "markov_precond_blocks",
    "Workload",
    "workload",
]


def laplacian_1d(n: int) -> np.ndarray:
    """``(n+1)^2 * tridiag(-1, 2, -1)``: the SPD 1-D Dirichlet Laplacian on a
    grid of ``n`` interior points with spacing ``h = 1/(n+1)``."""
    h2 = float(n + 1) ** 2
    L = np.zeros((n, n))
    idx = np.arange(n)
    L[idx, idx] = 2.0 * h2
    L[idx[:-1], idx[:-1] + 1] = -h2
    L[idx[1:], idx[1:] - 1] = -h2
    return L


def central_difference_1d(n: int) -> np.ndarray:
    """``(n+1)/2 * tridiag(-1, 0, +1)``: the central-difference first
    derivative (sub-diagonal -1, super-diagonal +1)."""
    c = float(n + 1) / 2.0
    B = np.zeros((n, n))
    idx = np.arange(n - 1)
    B[idx, idx + 1] = c
    B[idx + 1, idx] = -c
    return B


def paper_convdiff_1d(n: int, K: float = 1e-2, w: float = 1e-2) -> np.ndarray:
    """The paper's 1-D convection-diffusion block ``L + D_i`` on [-1, 1]
    (Section 5.1.1): ``K/h^2 tridiag(1,-2,1) + w/h bidiag(-1, 1)`` with
    ``h = 2/(n+1)``."""
    h = 2.0 / (n + 1)
    idx = np.arange(n)
    L = np.zeros((n, n))
    L[idx, idx] = -2.0
    L[idx[:-1], idx[:-1] + 1] = 1.0
    L[idx[1:], idx[1:] - 1] = 1.0
    D = np.zeros((n, n))
    D[idx, idx] = -1.0
    D[idx[:-1], idx[:-1] + 1] = 1.0
    return (K / h**2) * L + (w / h) * D


def kron_sum_operator(mats) -> list:
    """Rank-2 TT operator of the Kronecker sum ``sum_k I x .. x M_k x .. x I``.

    Cores (shape ``[R_{k-1}, n, n, R_k]``): first ``[M_1, I]``, middle
    ``[[I, 0], [M_k, I]]``, last ``[I; M_d]``.  Each path through the rank
    indices picks ``M`` in exactly one position, so the product of cores is the
    Kronecker sum.  ``d == 1`` gives the single core ``[[M_1]]``.
    """
    mats = [np.asarray(M, dtype=np.float64) for M in mats]
    d = len(mats)
    cores = []
    for k, M in enumerate(mats):
        n = M.shape[0]
        eye = np.eye(n)
        if d == 1:
            c = M.reshape(1, n, n, 1).copy()
        elif k == 0:
            c = np.zeros((1, n, n, 2))
            c[0, :, :, 0] = M
            c[0, :, :, 1] = eye
        elif k == d - 1:
            c = np.zeros((2, n, n, 1))
            c[0, :, :, 0] = eye
            c[1, :, :, 0] = M
        else:
            c = np.zeros((2, n, n, 2))
            c[0, :, :, 0] = eye
            c[1, :, :, 0] = M
            c[1, :, :, 1] = eye
        cores.append(c)
    return cores


def random_tt(ns, ranks, seed: int, dtype=np.float64) -> list:
    """Random TT with i.i.d. Gaussian cores.

    ``ranks`` has ``d+1`` entries with ``ranks[0] == ranks[-1] == 1``.  Core k
    is ``N(0, 1) / sqrt(r_{k-1} n_k)``; this deterministic per-core scale
    gives ``E ||x||^2 = 1`` for every rank profile (the "normalised" right-hand
    side, up to the random fluctuation of the norm).
    """
    ranks = list(ranks)
    if len(ranks) != len(ns) + 1 or ranks[0] != 1 or ranks[-1] != 1:
        raise ValueError("ranks must have d+1 entries with r_0 = r_d = 1")
    rng = np.random.default_rng(seed)
    cores = []
    for k, n in enumerate(ns):
        c = rng.standard_normal((ranks[k], n, ranks[k + 1]))
        c /= np.sqrt(ranks[k] * n)
        cores.append(c.astype(dtype))
    return cores


def rank_one_tt(vectors) -> list:
    """TT of rank 1 whose core k is the vector ``vectors[k]``."""
    return [np.asarray(v, dtype=np.float64).reshape(1, -1, 1).copy() for v in vectors]


def khatri_rao_factors(ns, s: int, seed: int) -> list:
    """Gaussian factors ``S_k in R^{s x n_k}`` with i.i.d. ``N(0, s^{-1/d})``
    entries (variance ``s^{-1/d}``, Section 3.1)."""
    d = len(ns)
    std = float(s) ** (-0.5 / d)
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((s, n)) * std for n in ns]


def tt_row_sketch(ns, s: int, R: int, seed: int) -> list:
    """Cores ``[s][R_{k-1}][n_k][R_k]`` of s independent Gaussian TT rows of
    rank R (R_0 = R_d = 1): entries N(0, 1/R_k), the first core scaled by
    ``s^{-1/2}``, so that ``E ||S x||^2 = ||x||^2``.  R = 1 gives Khatri-Rao rows."""
    rng = np.random.default_rng(seed)
    d = len(ns)
    out = []
    for k, n in enumerate(ns):
        a = 1 if k == 0 else R
        b = 1 if k == d - 1 else R
        Yk = rng.standard_normal((s, a, n, b)) / np.sqrt(b)
        if k == 0:
            Yk = Yk / np.sqrt(s)
        out.append(Yk)
    return out


def gaussian_drm(ns, ells, seed: int) -> list:
    """Gaussian TT-DRM cores ``[l_{k-1}, n_k, l_k]`` with variance
    ``1/(l_{k-1} n_k l_k)`` (Definition "Random Gaussian TT-Tensor").
    ``ells`` has ``d+1`` entries with ``ells[0] == ells[-1] == 1``."""
    rng = np.random.default_rng(seed)
    out = []
    for k, n in enumerate(ns):
        a, b = ells[k], ells[k + 1]
        out.append(rng.standard_normal((a, n, b)) / np.sqrt(a * n * b))
    return out


def uneven_ranks(d: int, lo: int, hi: int, seed: int) -> list:
    """Bond ranks drawn i.i.d. uniformly from ``lo..hi`` (inclusive), with
    ``r_0 = r_d = 1``."""
    rng = np.random.default_rng(seed)
    inner = rng.integers(lo, hi + 1, size=d - 1).tolist()
    return [1] + [int(r) for r in inner] + [1]


def birth_death_generator(n: int, rng) -> np.ndarray:
    """Generator (row convention, rows sum to zero) of a random walk on states
    0..n-1: rate eta_k from k to k+1 and mu_k from k to k-1, each drawn
    i.i.d. uniformly from [1, 2] (Section 5.1.2)."""
    eta = rng.uniform(1.0, 2.0, size=n - 1)
    mu = rng.uniform(1.0, 2.0, size=n - 1)
    Q = np.zeros((n, n))
    for k in range(n - 1):
        Q[k, k + 1] = eta[k]
        Q[k + 1, k] = mu[k]
    Q[np.arange(n), np.arange(n)] = -Q.sum(axis=1)
    return Q


def markov_operator(d: int, n: int, seed: int, sync_rate: float = 0.1):
    """TT operator of the steady-state system of d coupled random walks
    (Section 5.1.2), in the rank-one-normalised form
    ``A = -G_c + 1 1^T / n^d`` with ``G_c = (Q + W - D)^T`` the generator in
    column convention (``G_c pi = 0`` at steady state):

    * ``Q = sum_k I x .. x Q_k x .. x I`` with Q_k from
      :func:`birth_death_generator` (drawn in mode order from ``seed``);
    * for every pair of neighbouring systems (k, k+1) the joint transition from
      (n-2, n-2) to (n-1, n-1) at rate ``sync_rate`` (W) and its diagonal
      outflow (D), i.e. ``sync_rate (M x M - E x E)`` in column convention with
      ``M = e_{n-1} e_{n-2}^T`` and ``E = e_{n-2} e_{n-2}^T``;
    * the rank-one term ``1 1^T / n^d = (J/n) x .. x (J/n)``, J all ones.

    ``A rho = 1`` has the solution ``rho = n^d pi`` with pi the steady-state
    distribution.  Cores ``[R_{k-1}, n, n, R_k]`` with ranks 5 (channels: 0
    all terms closed, 1 none opened, 2 and 3 a synchronisation's W and D parts
    opened at the previous mode, 4 the rank-one term).  Returns the cores and
    the d matrices Q_k (row convention)."""
    rng = np.random.default_rng(seed)
    Qs = [birth_death_generator(n, rng) for _ in range(d)]
    eye = np.eye(n)
    M = np.zeros((n, n))
    M[n - 1, n - 2] = 1.0
    E = np.zeros((n, n))
    E[n - 2, n - 2] = 1.0
    J = np.ones((n, n)) / n
    cores = []
    for k in range(d):
        Rl = 1 if k == 0 else 5
        Rr = 1 if k == d - 1 else 5
        c = np.zeros((Rl, n, n, Rr))
        # left index: 0 closed, 1 none opened, 2 W open, 3 D open, 4 rank-one
        # (the first core's single row acts as both "none opened" and the
        # start of the rank-one channel)
        left = {0: 0, 1: 1, 2: 2, 3: 3, 4: 4} if k > 0 else {1: 0, 4: 0}
        last = k == d - 1
        def put(a, b, mat):
            if a in left:
                c[left[a], :, :, 0 if last else b] += mat
        single = -Qs[k].T
        put(0, 0, eye)
        put(1, 0, single)
        if not last:
            put(1, 1, eye)
            put(1, 2, -sync_rate * M)
            put(1, 3, sync_rate * E)
        put(2, 0, M)
        put(3, 0, E)
        put(4, 4, J)
        if last:
            # the channels that are still open close here
            pass
        cores.append(c)
    return cores, Qs


def markov_precond_blocks(Qs, shift_frac: float = 1.0):
    """Input data of the exponential-sum preconditioner of the Markov system:
    the blocks ``A_k = -Q_k^T + (sigma / d) I`` of the shifted independent part
    ``-Q^T + sigma I`` (the Kronecker sum of the systems' generators ignoring
    the synchronisations, shifted off its zero eigenvalue), with sigma a
    fraction of the smallest spectral gap among the systems, and the
    interval ``[sigma, sigma + sum_k lambda_max(-Q_k)]`` that holds the
    Kronecker sum's spectrum (the walks are reversible, so each -Q_k has real
    eigenvalues).  The default shift is the whole gap: a smaller one lowers
    the FP64 iteration count a little (6 against 9 at d = 5, n = 32) but
    amplifies the near-null direction by 1/sigma, which the float modes'
    products cannot resolve (TF32 stalled near 5e-6 at a third of the gap).
    Returns ``(blocks, a, b)``."""
    d = len(Qs)
    gaps, tops = [], []
    for Q in Qs:
        ev = np.sort(np.linalg.eigvals(-Q.T).real)
        gaps.append(ev[1])
        tops.append(ev[-1])
    sigma = shift_frac * min(gaps)
    blocks = [-Q.T + (sigma / d) * np.eye(Q.shape[0]) for Q in Qs]
    return blocks, sigma, sigma + sum(tops)


class Workload:
    """One synthetic linear system ``A x = b`` in TT format plus the solver
    parameters it is quoted with."""

    def __init__(self, name, op, b, params, extra=None):
        self.name = name
        self.op = op
        self.b = b
        self.params = dict(params)
        self.extra = dict(extra or {})

    @property
    def d(self):
        return len(self.op)

    @property
    def ns(self):
        return [c.shape[1] for c in self.op]


def workload(name: str, **over) -> Workload:
    """The five named model problems (sizes may be overridden for small
    test variants, e.g. ``workload('convdiff', d=4, n=16)``).

    * ``laplace_fp64``  d=4, n=16, ``A = sum_k L_k``, b = all ones (rank 1),
      m<=50, s=100, rounding tol 1e-8, rmax 40, tol 1e-6, FP64.
    * ``convdiff``  d=10, n=64, ``A = sum_k (L + 10 B)_k`` (rank 2), b random
      TT rank 4, rmax 64, m<=80, s=160, oversampling 10, mixed precision.
    * ``large_rank``  d=20, n=128, ``A = sum_k L_k``, b random TT rank 8,
      rmax 128, oversampling 10, m<=100, s=200, FP32 contractions.
    * ``batched``  d=8, n=32, 64 right-hand sides with bond ranks U{1..12},
      m<=100, s=200, rank cap 150 (basis and solution): the solutions of these
      rough right-hand sides need it for a 1e-6 residual (caps 40, 64, 100 left
      most of them above 1e-6, and 128 some of those with ranks near 12).
    * ``markov``  d=5, n=32 coupled random walks (Section 5.1.2), the
      rank-one-normalised steady-state system ``(-G_c + 1 1^T / n^d) rho = 1``
      (see :func:`markov_operator`), b = all ones (rank 1), rmax 64, m<=100;
      solved with the exponential-sum preconditioner of
      :func:`markov_precond_blocks`.
    * ``differentiable``  d=12, n=64, ``A(theta) = sum_k theta_k L_k`` with
      ``theta_k ~ U[0.5, 2]``, b and x_target random TT rank 4, rmax 64.
      x_target is scaled by ``1 / lambda_min(A(theta))`` (the largest gain of
      ``A^{-1}`` on a unit right-hand side), so that it has the solution's
      order of magnitude and the loss is sensitive to theta.
    """
    if name == "laplace_fp64":
        d, n = over.get("d", 4), over.get("n", 16)
        op = kron_sum_operator([laplacian_1d(n)] * d)
        b = rank_one_tt([np.ones(n)] * d)
        params = dict(maxit=50, s=100, tol=1e-6, round_tol=1e-8, rmax=40, oversample=10,
                      mode="fp64", r_sol=40)
        return Workload(name, op, b, {**params, **over.get("params", {})})
    if name == "convdiff":
        d, n = over.get("d", 10), over.get("n", 64)
        M = laplacian_1d(n) + 10.0 * central_difference_1d(n)
        op = kron_sum_operator([M] * d)
        r = over.get("rank", 4)
        b = random_tt([n] * d, [1] + [r] * (d - 1) + [1], seed=over.get("seed", 2))
        maxit = over.get("maxit", 80)
        params = dict(maxit=maxit, s=2 * maxit, tol=1e-6, rmax=64, oversample=10, mode="mixed",
                      eta=0.1, r_sol=64)
        return Workload(name, op, b, {**params, **over.get("params", {})})
    if name == "large_rank":
        d, n = over.get("d", 20), over.get("n", 128)
        op = kron_sum_operator([laplacian_1d(n)] * d)
        r = over.get("rank", 8)
        b = random_tt([n] * d, [1] + [r] * (d - 1) + [1], seed=over.get("seed", 2))
        maxit = over.get("maxit", 100)
        params = dict(maxit=maxit, s=2 * maxit, tol=1e-6, rmax=128, oversample=10, mode="fp32",
                      eta=0.1, r_sol=128)
        return Workload(name, op, b, {**params, **over.get("params", {})})
    if name == "batched":
        d, n = over.get("d", 8), over.get("n", 32)
        nrhs = over.get("nrhs", 64)
        op = kron_sum_operator([laplacian_1d(n)] * d)
        bs = [random_tt([n] * d, uneven_ranks(d, 1, 12, seed=1000 + i), seed=1000 + i)
              for i in range(nrhs)]
        maxit = over.get("maxit", 100)
        params = dict(maxit=maxit, s=2 * maxit, tol=1e-6, round_tol=1e-8, rmax=150, oversample=10,
                      mode="mixed", r_sol=150)
        return Workload(name, op, bs, {**params, **over.get("params", {})})
    if name == "markov":
        d, n = over.get("d", 5), over.get("n", 32)
        op, Qs = markov_operator(d, n, seed=over.get("seed", 5))
        b = rank_one_tt([np.ones(n)] * d)
        maxit = over.get("maxit", 100)
        params = dict(maxit=maxit, s=2 * maxit, tol=1e-6, rmax=64, oversample=10, mode="mixed",
                      eta=0.1, r_sol=64)
        return Workload(name, op, b, {**params, **over.get("params", {})}, extra=dict(Q=Qs))
    if name == "differentiable":
        d, n = over.get("d", 12), over.get("n", 64)
        rng = np.random.default_rng(over.get("theta_seed", 4))
        theta = rng.uniform(0.5, 2.0, size=d)
        L = laplacian_1d(n)
        b = random_tt([n] * d, [1] + [4] * (d - 1) + [1], seed=over.get("seed", 2))
        xt = random_tt([n] * d, [1] + [4] * (d - 1) + [1], seed=over.get("target_seed", 3))
        lam_min = float(np.sum(theta)) * 4.0 * (n + 1) ** 2 * np.sin(np.pi / (2 * (n + 1))) ** 2
        xt[0] = xt[0] / lam_min
        op = kron_sum_operator([t * L for t in theta])
        maxit = over.get("maxit", 100)
        params = dict(maxit=maxit, s=2 * maxit, tol=1e-6, rmax=64, oversample=10, mode="fp32",
                      eta=0.1, r_sol=64)
        return Workload(name, op, b, {**params, **over.get("params", {})},
                        extra=dict(theta=theta, L=L, x_target=xt))
    raise KeyError(name)
