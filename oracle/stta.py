"""Streaming tensor-train approximation (STTA), Section 3.3: the two-sided
sketch of a TT tensor with two Gaussian TT-DRMs and the recovery of an
approximant from the sketches alone.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Notation (Section 3.3): ``T`` has cores ``C_k [t_{k-1}][n_k][t_k]``; ``X`` is a
Gaussian TT-DRM of ranks ``r_mu`` (the target ranks) whose right interface
matrices ``X_{>mu}`` ((n_{mu+1}..n_d) x r_mu) sketch from the right, and ``Y``
one of ranks ``l_mu > r_mu`` whose left interface matrices ``Y_{<=mu}``
((n_1..n_mu) x l_mu) sketch from the left.  With ``T_{<=mu}`` the unfolding of
rows ``(i_1..i_mu)`` and columns ``(i_{mu+1}..i_d)`` (``i_1`` slowest):

* ``Psi_mu = (Y_{<=mu-1}^T kron I_{n_mu}) T_{<=mu} X_{>mu}``, a
  ``[l_{mu-1}][n_mu][r_mu]`` array, mu = 1..d;
* ``Omega_mu = Y_{<=mu}^T T_{<=mu} X_{>mu}``, ``l_mu x r_mu``, mu = 1..d-1;
* the approximant's cores, right unfolding ``C^_mu = Omega_{mu-1}^+ Psi_mu``
  (``C^_1 = Psi_1``).

Sketches are linear in ``T``: the sketches of ``sum_i a_i T_i`` are the same
combination of the terms' sketches, which is how a sum is approximated
without forming it.

Reading (the paper does not say how the pseudo-inverse is formed): ``Omega^+``
is the least-squares solution with singular values below ``rcond`` times the
largest treated as zero (``rcond = 1e-12``; a caller with single-precision
sketches passes a larger one).
"""
from __future__ import annotations

import numpy as np

from . import rounding as rnd

RCOND = 1e-12


def left_interface(Y, mu):
    """``Y_{<=mu}`` as a dense ``(n_1..n_mu) x l_mu`` matrix (mu = 0: ``[[1]]``)."""
    out = np.ones((1, 1))
    for k in range(mu):
        c = Y[k]
        out = (out @ c.reshape(c.shape[0], -1)).reshape(-1, c.shape[2])
    return out


def right_interface(X, mu):
    """``X_{>mu}`` as a dense ``(n_{mu+1}..n_d) x r_mu`` matrix (mu = d: ``[[1]]``)."""
    d = len(X)
    out = np.ones((1, 1))          # rows (i_{k+1}..i_d), columns r_k
    for k in range(d - 1, mu - 1, -1):
        c = X[k]                   # [r_k][n][r_{k+1}]
        # new[(i_k, rest), a] = sum_b c[a, i_k, b] out[rest, b]
        new = np.einsum("aib,jb->ija", c, out)
        out = new.reshape(-1, c.shape[0])
    return out


def sketch_dense(full, ns, X, Y):
    """``(Psi, Omega)`` from the definitions on the dense tensor ``full``
    (tiny sizes only).  ``Psi[mu-1]`` is ``Psi_mu``, ``Omega[mu-1]`` is
    ``Omega_mu``."""
    d = len(ns)
    T = np.asarray(full, dtype=np.float64).reshape(-1)
    Psi, Omega = [], []
    for mu in range(1, d + 1):
        rows = int(np.prod(ns[:mu]))
        Tmu = T.reshape(rows, -1)
        Xr = right_interface(X, mu)
        Yl = left_interface(Y, mu - 1)
        lhs = np.kron(Yl.T, np.eye(ns[mu - 1]))
        P = lhs @ Tmu @ Xr
        Psi.append(P.reshape(Yl.shape[1], ns[mu - 1], Xr.shape[1]))
        if mu < d:
            Omega.append(left_interface(Y, mu).T @ Tmu @ Xr)
    return Psi, Omega


def left_partial_contractions(cores, Y):
    """``L_mu = Y_{<=mu}^T C_{<=mu}`` (``l_mu x t_mu``) for mu = 0..d-1, by the
    left-to-right sweep ``L_mu = sum_i Y_mu[:, i, :]^T L_{mu-1} C_mu[:, i, :]``."""
    d = len(cores)
    L = [np.ones((1, 1))]
    for mu in range(1, d):
        C, Yc = cores[mu - 1], Y[mu - 1]
        acc = np.zeros((Yc.shape[2], C.shape[2]))
        for i in range(C.shape[1]):
            acc += Yc[:, i, :].T @ L[mu - 1] @ C[:, i, :]
        L.append(acc)
    return L


def sketch(cores, X, Y):
    """``(Psi, Omega)`` of a TT through its partial contractions (Section
    3.3): ``Psi_mu = L_{mu-1} x_1 C_mu x_3 R_mu^T`` and ``Omega_mu = L_mu R_mu``
    with ``R_mu = C_{>mu}^T X_{>mu}`` the right partial contractions."""
    d = len(cores)
    L = left_partial_contractions(cores, Y)
    R = rnd.right_partial_contractions(cores, X)   # R[mu]: t_mu x r_mu
    Psi, Omega = [], []
    for mu in range(1, d + 1):
        C = cores[mu - 1]
        Psi.append(np.einsum("ac,cie,eb->aib", L[mu - 1], C, R[mu]))
        if mu < d:
            Omega.append(L[mu] @ R[mu])
    return Psi, Omega


def sketch_sum(terms, X, Y):
    """Sketches of ``sum_i a_i T_i`` (``terms`` = [(a_i, cores_i)]) as the
    same combination of the terms' sketches."""
    Psi, Omega = None, None
    for a, cores in terms:
        P, O = sketch(cores, X, Y)
        if Psi is None:
            Psi = [a * p for p in P]
            Omega = [a * o for o in O]
        else:
            Psi = [u + a * p for u, p in zip(Psi, P)]
            Omega = [u + a * o for u, o in zip(Omega, O)]
    return Psi, Omega


def recover(Psi, Omega, rcond=RCOND):
    """Cores of the approximant: ``C^_1 = Psi_1`` and
    ``C^_mu = Omega_{mu-1}^+ Psi_mu`` (right unfoldings), the pseudo-inverse
    by least squares with relative cutoff ``rcond``."""
    d = len(Psi)
    cores = [np.array(Psi[0], dtype=np.float64)]
    for mu in range(2, d + 1):
        P = Psi[mu - 1]
        Om = Omega[mu - 2]
        sol = np.linalg.lstsq(Om, P.reshape(P.shape[0], -1), rcond=rcond)[0]
        cores.append(sol.reshape(Om.shape[1], P.shape[1], P.shape[2]))
    return cores
