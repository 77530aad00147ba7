"""Exponential-sum right preconditioning and TT-sPGMRES (Section 4,
Algorithm 5), in float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

With the dominant part of the operator a Kronecker sum ``A_0 = sum_j (I x .. x
A_j x .. x I)``, the preconditioner is ``P^{-1} = E(A_0)`` for an exponential
sum ``E(z) = sum_i alpha_i exp(-beta_i z) ~ 1/z``; because the terms of a
Kronecker sum commute, ``exp(-beta A_0)`` is the Kronecker product of the
``exp(-beta A_j)``, so ``P^{-1} x = sum_i alpha_i (x multiplied in every mode j
by exp(-beta_i A_j))`` and each term keeps x's TT ranks.

Reading (the paper takes its coefficients from a procedure it does not print):
the coefficients come from the trapezoidal rule applied to
``1/z = int_R exp(t - e^t z) dt`` (the substitution s = e^t in the Laplace
integral ``int_0^inf exp(-s z) ds``), the exponentially convergent rule for
such integrands (Trefethen and Weideman, SIAM Review 2014).  For z in [a, b]
write z = a u, u in [1, kappa]; with step h and nodes t_k = k h, k0 <= k <= k1,
``1/u ~ h sum_k exp(t_k) exp(-exp(t_k) u)``, so ``alpha_k = h exp(t_k) / a`` and
``beta_k = exp(t_k) / a``.  The truncations and step follow from a target
relative accuracy tol: the lower tail is below ``u exp(t_lo)``, so
``t_lo = log(tol / kappa)``; the upper tail is ``exp(-exp(t_hi) u) / u``,
below tol at u = 1 for ``t_hi = log(log(1 / tol))``.  The integrand is
analytic in t; on the line Im t = y it is bounded by ``exp(Re t - e^{Re t} u
cos y)``, which still decays for |y| < pi/2 but ever more slowly as |y| -> pi/2,
so the strip used for the error bound has half-width pi/4 (cos y >= 1/sqrt 2).
The rule's discretisation error then decays like ``exp(-2 pi (pi/4) / h)``, and
``h = pi^2 / (2 log(1 / tol))``.  (With the full half-width pi/2 the same
derivation gives h twice as large, which measured 9-12 tol instead of tol.)
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from . import tt as ttm
from . import rounding as rnd
from . import solvers as sol


def exp_sum_coefficients(a, b, tol=1e-2):
    """``(alpha, beta)`` of an exponential sum with ``|E(z) z - 1| <~ tol`` on
    ``[a, b]`` (0 < a < b), by the trapezoidal rule described above."""
    if not (0 < a < b):
        raise ValueError("need 0 < a < b")
    kappa = b / a
    t_lo = math.log(tol / kappa)
    t_hi = math.log(math.log(1.0 / tol))
    h = math.pi ** 2 / (2.0 * math.log(1.0 / tol))
    k0 = math.floor(t_lo / h)
    k1 = math.ceil(t_hi / h)
    t = h * np.arange(k0, k1 + 1, dtype=np.float64)
    return h * np.exp(t) / a, np.exp(t) / a


def exp_sum(z, alpha, beta):
    """``E(z) = sum_i alpha_i exp(-beta_i z)``."""
    z = np.asarray(z, dtype=np.float64)
    return np.sum(alpha[:, None] * np.exp(-np.outer(beta, z.reshape(-1))), axis=0).reshape(z.shape)


def mode_product(cores, mats):
    """The TT whose core k is ``C_k x_2 M_k`` (``M_k`` acting on mode k):
    ``(M_1 x .. x M_d) x`` without changing the ranks."""
    return [np.einsum("ij,ajb->aib", M, C) for C, M in zip(cores, mats)]


def precond_matrices(A1d, alpha, beta):
    """``exp(-beta_i A_j)`` for every term i and mode j (dense, scipy expm)."""
    return [[sla.expm(-bi * A) for A in A1d] for bi in beta]


def apply_precond(cores, A1d, alpha, beta, eps=None, rmax=None, drm=None, oversample=10):
    """``P^{-1} x = sum_i alpha_i (exp(-beta_i A_1) x .. x exp(-beta_i A_d)) x``.
    Without ``drm`` the exact sum (ranks multiplied by the number of terms);
    with it, rounded by the randomized rounding to ``eps`` and ``rmax`` (the
    bounded-rank rounding of Section 4.2)."""
    E = precond_matrices(A1d, alpha, beta)
    terms = [(float(a), mode_product(cores, Ei)) for a, Ei in zip(alpha, E)]
    if drm is None:
        return ttm.add(terms)
    return rnd.rto_round(terms, drm, eps=eps or 0.0, rmax=rmax, oversample=oversample)


def tt_spgmres(op, b, A1d, alpha, beta, S, drm, maxit, tol, round_tol, rmax, oversample=10,
               r_sol=None, final_tol=None):
    """Algorithm 5 (l = 1, zero initial guess): right preconditioning,
    ``w = A P^{-1} v_k`` with ``P^{-1} v_k`` rounded to ``rmax`` (bounded-rank
    rounding), and ``x = P^{-1} (sum_i y_i v_i)``.  Returns ``(x, info)``."""
    r_sol = rmax if r_sol is None else r_sol
    final_tol = round_tol if final_tol is None else final_tol
    beta0 = ttm.norm(b)
    V = [ttm.scale(b, 1.0 / beta0)]
    Sr0 = ttm.sketch_kr_fast(b, S)
    betaS = float(np.linalg.norm(Sr0))
    Wcols, hist = [], []
    y = None
    k = 0
    for k in range(1, maxit + 1):
        z = apply_precond(V[-1], A1d, alpha, beta, eps=round_tol, rmax=rmax, drm=drm,
                          oversample=oversample)
        w = ttm.matvec(op, z)                           # A P^{-1} v_k
        Wcols.append(ttm.sketch_kr_fast(w, S))
        h = ttm.dot(w, V[-1])
        vt = rnd.rto_round([(1.0, w), (-h, V[-1])], drm, eps=round_tol, rmax=rmax,
                           oversample=oversample)
        hn = ttm.norm(vt)
        y, res = sol.sketched_lstsq(np.stack(Wcols, axis=1), Sr0)
        hist.append(res / betaS)
        if res <= tol * betaS or hn == 0.0:
            break
        V.append(ttm.scale(vt, 1.0 / hn))
    u = rnd.rto_round([(float(y[i]), V[i]) for i in range(len(y))], drm, eps=final_tol,
                      rmax=r_sol, oversample=oversample)
    x = apply_precond(u, A1d, alpha, beta, eps=final_tol, rmax=r_sol, drm=drm,
                      oversample=oversample)
    return x, dict(iters=k, res_hist=hist)
