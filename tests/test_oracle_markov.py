"""Pins of the Markov-chain workload (Section 5.1.2): the TT operator of the
rank-one-normalised steady-state system against the generator built state by
state from the model's definition, zero row sums of that generator, its
steady state against the solution of the normalised system, the operator's
TT ranks, and the oracle's TT-sGMRES on a small instance."""
import itertools

import numpy as np
import pytest

import ttinputs as ti
from oracle import tt as ott, solvers as osol, philox as oph


def dense_generator(Qs, n, rate=0.1):
    """Row-convention generator of d coupled random walks, enumerated state by
    state: each system moves k -> k +- 1 at the rates of its own generator;
    neighbouring systems k, k+1 both in state n-2 move together to n-1."""
    d = len(Qs)
    N = n ** d
    states = list(itertools.product(range(n), repeat=d))  # C order: mode 1 slowest
    index = {s: i for i, s in enumerate(states)}
    G = np.zeros((N, N))
    for s in states:
        i = index[s]
        for k in range(d):
            for t in (s[k] - 1, s[k] + 1):
                if 0 <= t < n:
                    u = list(s)
                    u[k] = t
                    G[i, index[tuple(u)]] += Qs[k][s[k], t]
        for k in range(d - 1):
            if s[k] == n - 2 and s[k + 1] == n - 2:
                u = list(s)
                u[k] = u[k + 1] = n - 1
                G[i, index[tuple(u)]] += rate
        G[i, i] = -G[i].sum()
    return G


@pytest.mark.parametrize("d,n", [(2, 4), (3, 4), (4, 3)])
def test_markov_operator_equals_the_model(d, n):
    op, Qs = ti.markov_operator(d, n, seed=7)
    G = dense_generator(Qs, n)
    assert np.allclose(G.sum(axis=1), 0.0, atol=1e-12)        # a generator
    assert np.all(G - np.diag(np.diag(G)) >= 0.0)
    N = n ** d
    A = -G.T + np.ones((N, N)) / N
    assert np.max(np.abs(ott.op_full(op) - A)) <= 1e-13 * np.max(np.abs(A))
    assert [c.shape[0] for c in op] + [1] == [1] + [5] * (d - 1) + [1]


def test_markov_steady_state_solves_the_normalised_system():
    d, n = 3, 5
    op, Qs = ti.markov_operator(d, n, seed=3)
    G = dense_generator(Qs, n)
    N = n ** d
    # steady state: the null vector of G^T (smallest singular vector), summing to one
    U, sv, Vt = np.linalg.svd(G.T)
    pi = Vt[-1] / Vt[-1].sum()
    assert sv[-1] <= 1e-12 * sv[0] and sv[-2] > 1e-6 * sv[0]  # irreducible: one null vector
    assert np.all(pi > 0)
    rho = np.linalg.solve(ott.op_full(op), np.ones(N))
    assert np.allclose(rho / N, pi, rtol=1e-10, atol=1e-14)
    assert abs(rho.sum() / N - 1.0) <= 1e-12


def test_markov_oracle_tt_sgmres_small():
    w = ti.workload("markov", d=4, n=6, maxit=60)
    p = w.params
    S = oph.sketch_factors(w.ns, p["s"], 0)
    drm = oph.drm_cores(w.ns, [1] + [p["rmax"] + p["oversample"]] * (w.d - 1) + [1], 0)
    x, info = osol.solve(w.op, w.b, S, drm, maxit=p["maxit"], tol=1e-8, round_tol=1e-10,
                         rmax=p["rmax"], oversample=p["oversample"], r_sol=p["r_sol"],
                         stop_safety=0.1, max_restarts=10)
    assert info["true_res"] <= 1e-8
    N = 6 ** 4
    ref = np.linalg.solve(ott.op_full(w.op), np.ones(N))
    assert np.linalg.norm(ott.full(x) - ref) <= 1e-6 * np.linalg.norm(ref)
