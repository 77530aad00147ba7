"""Dense gradients of ``loss(theta, b) = ||x - x_t||^2`` with ``A(theta) x = b``
on tiny grids (plain linear algebra on the dense operator; no TT solver).

With ``A(theta) = sum_k theta_k (I x .. x L x .. x I)`` (L in position k):

* ``lambda = A^{-T} 2 (x - x_t)`` (adjoint solve),
* ``d loss / d b = lambda``,
* ``d loss / d theta_k = - lambda^T (I x .. x L x .. x I) x``,
* ``d loss / d C_k[a, i, c] = sum_{alpha, beta} lambda[alpha, i, beta]
  P_{<k}[alpha, a] Q_{>k}[beta, c]`` where ``P_{<k}`` and ``Q_{>k}`` are the
  left and right interface matrices of b's TT (Section 2.2).
"""
from __future__ import annotations

import numpy as np

from . import tt as ttm
from . import closed_forms as cf


def loss_and_grads(theta, L, b_cores, xt_cores):
    """Loss and gradients w.r.t. ``theta`` and b's cores (dense)."""
    d = len(b_cores)
    ns = [c.shape[1] for c in b_cores]
    mats = [t * L for t in theta]
    bfull = ttm.full(b_cores)
    x = cf.kron_sum_solve_dense(mats, bfull)
    xt = ttm.full(xt_cores)
    g = 2.0 * (x - xt)
    lam = cf.kron_sum_solve_dense([M.T for M in mats], g)
    loss = float(np.sum((x - xt) ** 2))
    X = x.reshape(ns)
    dtheta = np.zeros(d)
    for k in range(d):
        LX = np.moveaxis(np.tensordot(L, X, axes=([1], [k])), 0, k).reshape(-1)
        dtheta[k] = -float(lam @ LX)
    dcores = []
    for k in range(d):
        left = np.ones((1, 1))
        for c in b_cores[:k]:
            left = (left @ c.reshape(c.shape[0], -1)).reshape(-1, c.shape[2])
        right = np.ones((1, 1))
        for c in reversed(b_cores[k + 1:]):
            right = (c.reshape(-1, c.shape[2]) @ right.T).reshape(c.shape[0], -1).T
        # left: (n_<k, r_{k-1}); right: (n_>k, r_k)
        Lam = lam.reshape(left.shape[0], ns[k], right.shape[0])
        dcores.append(np.einsum("xiy,xa,yc->aic", Lam, left, right))
    return loss, dtheta, dcores, x, lam


def interfaces(x, y):
    """Left and right interface matrices of TT ``x`` against TT ``y``
    (Section 2.2 inner-product sweep, kept at every bond):
    ``P[0] = 1``, ``P[k+1] = sum_i X_k[:, i, :]^T P[k] Y_k[:, i, :]`` and
    ``Q[d] = 1``, ``Q[k] = sum_i X_k[:, i, :] Q[k+1] Y_k[:, i, :]^T``."""
    d = len(x)
    P = [None] * (d + 1)
    Q = [None] * (d + 1)
    P[0] = np.ones((1, 1))
    for k in range(d):
        P[k + 1] = sum(x[k][:, i, :].T @ P[k] @ y[k][:, i, :] for i in range(x[k].shape[1]))
    Q[d] = np.ones((1, 1))
    for k in range(d - 1, -1, -1):
        Q[k] = sum(x[k][:, i, :] @ Q[k + 1] @ y[k][:, i, :].T for i in range(x[k].shape[1]))
    return P, Q


def dot_grad(x, y):
    """Derivative of ``<x, y>`` with respect to every core of ``y``:
    ``G_k[b, i, c] = sum_{a, a'} P_k[a, b] X_k[a, i, a'] Q_{k+1}[a', c]``."""
    P, Q = interfaces(x, y)
    return [np.einsum("ab,aic,ce->bie", P[k], x[k], Q[k + 1]) for k in range(len(x))]


def local_dots(x, y, mats):
    """``out[k] = <x, (I x .. x mats[k] x .. x I) y>`` through the interfaces:
    ``<G_k, mats[k] x_2 Y_k>``."""
    G = dot_grad(x, y)
    return np.array([np.sum(G[k] * np.einsum("ij,bjc->bic", mats[k], y[k]))
                     for k in range(len(x))])
