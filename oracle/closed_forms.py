"""Closed forms for the model problems (no TT arithmetic involved).

* Eigenpairs of tridiagonal Toeplitz matrices ``tridiag(a_sub, a_diag,
  a_sup)`` with ``a_sub a_sup > 0``: ``lambda_j = a_diag + 2 sign(a_sub)
  sqrt(a_sub a_sup) cos(j pi / (n+1))`` with
  eigenvector entries ``(a_sub / a_sup)^{i/2} sin(i j pi / (n+1))``,
  ``i, j = 1..n``.  For ``L = (n+1)^2 tridiag(-1, 2, -1)`` this is
  ``lambda_j = 4 (n+1)^2 sin^2(j pi / (2(n+1)))`` with the orthonormal sine
  vectors ``sqrt(2/(n+1)) sin(i j pi/(n+1))``.
* For a Kronecker sum ``A = sum_k I x .. x M_k x .. x I`` and a rank-1 tensor
  of eigenvectors ``q = q_{j_1} x .. x q_{j_d}``: ``A q = (sum_k lambda_{j_k}) q``.
* Dense solve of a Kronecker sum by fast diagonalisation:
  ``x = (V_1 x .. x V_d) [((V_1^{-1} x .. x V_d^{-1}) b) / (sum_k lambda_{i_k})]``.
"""
from __future__ import annotations

import numpy as np


def toeplitz_tridiag_eig(n, a_sub, a_diag, a_sup):
    """Eigenvalues and (unnormalised) eigenvectors of ``tridiag(a_sub, a_diag,
    a_sup)`` of order n; eigenvector j is column j-1."""
    if a_sub * a_sup <= 0:
        raise ValueError("only a_sub * a_sup > 0 (real spectrum) is supported")
    j = np.arange(1, n + 1)
    i = np.arange(1, n + 1)
    # with rho = sqrt(a_sub / a_sup): a_sub / rho = a_sup * rho = sign(a_sub) sqrt(a_sub a_sup)
    lam = a_diag + 2.0 * np.sign(a_sub) * np.sqrt(a_sub * a_sup) * np.cos(j * np.pi / (n + 1))
    scale = (a_sub / a_sup) ** (i / 2.0)
    V = scale[:, None] * np.sin(np.outer(i, j) * np.pi / (n + 1))
    return lam, V


def laplacian_eig(n):
    """``lambda_j = 4 (n+1)^2 sin^2(j pi / (2(n+1)))`` and the orthonormal
    sine eigenvectors of ``(n+1)^2 tridiag(-1, 2, -1)``."""
    j = np.arange(1, n + 1)
    lam = 4.0 * (n + 1) ** 2 * np.sin(j * np.pi / (2.0 * (n + 1))) ** 2
    Q = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(j, j) * np.pi / (n + 1))
    return lam, Q


def convdiff_eig(n, c=10.0):
    """Eigenpairs of ``(n+1)^2 tridiag(-1,2,-1) + c (n+1)/2 tridiag(-1,0,1)``
    (sub-diagonal ``-(n+1)^2 - c(n+1)/2``, super-diagonal ``-(n+1)^2 +
    c(n+1)/2``)."""
    h2 = float(n + 1) ** 2
    g = c * (n + 1) / 2.0
    return toeplitz_tridiag_eig(n, -h2 - g, 2.0 * h2, -h2 + g)


def kron_sum_solve_dense(mats, bfull):
    """Dense solution of ``(sum_k I x .. x M_k x .. x I) x = b`` (C order,
    mode 1 slowest) by eigendecomposition of every ``M_k``."""
    d = len(mats)
    ns = [M.shape[0] for M in mats]
    T = np.asarray(bfull, dtype=np.float64).reshape(ns)
    lams, Vs, Vinvs = [], [], []
    for M in mats:
        lam, V = np.linalg.eig(M)
        if np.max(np.abs(lam.imag)) > 1e-9 * np.max(np.abs(lam)):
            raise ValueError("complex spectrum not supported")
        lam, V = lam.real, V.real
        lams.append(lam)
        Vs.append(V)
        Vinvs.append(np.linalg.inv(V))
    for k in range(d):
        T = np.moveaxis(np.tensordot(Vinvs[k], T, axes=([1], [k])), 0, k)
    denom = np.zeros(ns)
    for k in range(d):
        shape = [1] * d
        shape[k] = ns[k]
        denom = denom + lams[k].reshape(shape)
    T = T / denom
    for k in range(d):
        T = np.moveaxis(np.tensordot(Vs[k], T, axes=([1], [k])), 0, k)
    return T.reshape(-1)


def kron_sum_apply_dense(mats, xfull):
    """``(sum_k I x .. x M_k x .. x I) x`` on a dense tensor, mode by mode."""
    ns = [M.shape[0] for M in mats]
    X = np.asarray(xfull, dtype=np.float64).reshape(ns)
    out = np.zeros_like(X)
    for k, M in enumerate(mats):
        out += np.moveaxis(np.tensordot(M, X, axes=([1], [k])), 0, k)
    return out.reshape(-1)
