"""TT rounding in float64: deterministic TT-SVD and randomize-then-orthogonalize.

``tt_svd_round`` follows the TT-SVD rounding recalled in Section 2.2 (QR
orthogonalisation, then truncated SVDs of the interface matrices, accuracy
``||T - T~||_F <= eps ||T||_F`` or ranks capped at ``rmax``).

``rto_round`` is the randomize-then-orthogonalize rounding the paper cites in
Section 3.3 (right partial contractions with a Gaussian TT-DRM, Definition
"Random Gaussian TT-Tensor", then a left-to-right sweep of QR + projection),
applied to an implicit sum ``sum_b a_b X^(b)`` term by term (never forming the
block cores), followed by the TT-SVD truncation sweep that turns the fixed-rank
result into one meeting the tolerance.
"""
from __future__ import annotations

import numpy as np

from . import tt as ttm


def truncation_rank(sigma, delta, rmax=None):
    """Smallest ``r >= 1`` with ``sqrt(sum_{i >= r} sigma_i^2) <= delta``,
    capped at ``rmax`` (ties go to the smaller rank)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    tail = np.sqrt(np.cumsum((sigma ** 2)[::-1]))[::-1]  # tail[i] = ||sigma[i:]||
    r = len(sigma)
    for i in range(1, len(sigma) + 1):
        t = tail[i] if i < len(sigma) else 0.0
        if t <= delta:
            r = i
            break
    if rmax is not None:
        r = min(r, int(rmax))
    return max(1, r)


def tt_svd_round(cores, eps=0.0, rmax=None):
    """TT-SVD rounding: right-to-left QR orthogonalisation, then left-to-right
    truncated SVDs with the per-bond threshold ``delta = eps ||T|| /
    sqrt(d - 1)``.  Returns left-orthogonal cores 1..d-1."""
    d = len(cores)
    X = ttm.right_orthogonalize(cores)
    if d == 1:
        return X
    nrm = np.linalg.norm(X[0])
    delta = eps * nrm / np.sqrt(d - 1)
    for k in range(d - 1):
        r0, n, r1 = X[k].shape
        U, s, Vt = np.linalg.svd(X[k].reshape(r0 * n, r1), full_matrices=False)
        r = truncation_rank(s, delta, rmax)
        X[k] = U[:, :r].reshape(r0, n, r)
        X[k + 1] = np.einsum("ab,bic->aic", s[:r, None] * Vt[:r], X[k + 1])
    return X


def rto_ranks(term_ranks, ns, rmax, oversample):
    """Sketch ranks of the randomized rounding: ``l_0 = l_d = 1`` and, left to
    right, ``l_mu = min(rmax + p, t_mu, l_{mu-1} n_mu, prod_{k > mu} n_k)``
    where ``t_mu`` is the representation rank of the sum (sum of the terms'
    ranks).  The caps keep every QR input at full column rank by shape."""
    d = len(ns)
    t = [sum(r[mu] for r in term_ranks) for mu in range(d + 1)]
    ells = [1]
    for mu in range(1, d):
        right = int(np.prod(ns[mu:], dtype=np.float64)) if d - mu < 40 else 1 << 60
        cap = rmax + oversample if rmax is not None else t[mu]
        ells.append(int(min(cap, t[mu], ells[-1] * ns[mu - 1], right)))
    ells.append(1)
    return ells


def right_partial_contractions(X, drm):
    """``W_mu = X_{>mu}^T R_{>mu}`` for mu = d-1..1 (Section 3.3): with
    ``W_d = 1``, ``W_{mu-1} = sum_i X_mu[:, i, :] W_mu R_mu[:, i, :]^T``.
    Returns the list indexed by mu (``W[mu]`` has shape ``t_mu x l_mu``)."""
    d = len(X)
    W = [None] * (d + 1)
    W[d] = np.ones((1, 1))
    for mu in range(d, 1, -1):
        C, R = X[mu - 1], drm[mu - 1]
        acc = np.zeros((C.shape[0], R.shape[0]))
        for i in range(C.shape[1]):
            acc += C[:, i, :] @ W[mu] @ R[:, i, :].T
        W[mu - 1] = acc
    return W


def truncate_simultaneous(cores, eps=0.0, rmax=None):
    """Truncation of a left-orthogonal TT (cores 1..d-1 left-orthogonal) with
    all bonds decided from the same tensor: the right Gram matrices
    ``G_mu = C_{>mu}^T C_{>mu}`` (one right-to-left sweep) have the squared
    bond singular values as eigenvalues; bond mu keeps the eigenvectors
    ``W_mu`` of the largest ones (smallest rank with tail <= eps ||T|| /
    (d - 1), capped at rmax) and core mu becomes ``W_{mu-1}^T C_mu W_mu``.
    Telescoping over the bonds bounds the error by the sum of the dropped
    tails, hence by ``eps ||T||``."""
    d = len(cores)
    G = [None] * (d + 1)
    G[d] = np.ones((1, 1))
    for mu in range(d, 1, -1):
        C = cores[mu - 1]
        acc = np.zeros((C.shape[0], C.shape[0]))
        for i in range(C.shape[1]):
            acc += C[:, i, :] @ G[mu] @ C[:, i, :].T
        G[mu - 1] = acc
    nrm = np.sqrt(max(np.trace(G[1]), 0.0))
    delta = eps * nrm / max(d - 1, 1)
    W = [np.ones((1, 1))] + [None] * (d - 1) + [np.ones((1, 1))]
    for mu in range(1, d):
        lam, V = np.linalg.eigh(G[mu])
        order = np.argsort(lam)[::-1]
        sig = np.sqrt(np.maximum(lam[order], 0.0))
        r = truncation_rank(sig, delta, rmax)
        W[mu] = V[:, order[:r]]
    return [np.einsum("ap,aib,bq->piq", W[k], cores[k], W[k + 1]) for k in range(d)]


def rto_round(terms, drm, eps=0.0, rmax=None, oversample=10, truncation="sequential"):
    """Randomize-then-orthogonalize rounding of ``sum_b a_b X^(b)``.

    ``terms`` is a list of ``(a_b, cores_b)``; ``drm`` is a Gaussian TT-DRM
    whose ranks are at least the sketch ranks of :func:`rto_ranks` (its
    leading sub-blocks are used; a sub-block of a Gaussian core is again a
    Gaussian core and the DRM's scale does not change the computed range).

    1. Right sweep: partial contractions ``W^(b)_mu`` of every term with the DRM.
    2. Left sweep: ``Z^(b)_1 = a_b X^(b)_1``; at bond mu, ``Y = sum_b
       unfold(Z^(b)_mu) W^(b)_mu``, Householder ``Y = Q R``, core mu <- Q,
       ``M^(b) = Q^T unfold(Z^(b)_mu)``, ``Z^(b)_{mu+1} = M^(b) x_1
       X^(b)_{mu+1}``; the last core is ``sum_b Z^(b)_d``.
    3. Right-to-left truncated SVDs with ``delta = eps ||T|| / sqrt(d-1)``
       and ranks capped at ``rmax`` (this sweep leaves cores 2..d
       right-orthogonal, so ``||T||`` equals ``||core_1||``); or, with
       ``truncation="simultaneous"``, :func:`truncate_simultaneous`.
    """
    d = len(terms[0][1])
    ns = [c.shape[1] for c in terms[0][1]]
    ells = rto_ranks([ttm.ranks(X) for _, X in terms], ns, rmax, oversample)
    R = [drm[k][:ells[k], :, :ells[k + 1]] for k in range(d)]
    if d == 1:
        return [sum(a * X[0] for a, X in terms)]
    Ws = [right_partial_contractions(X, R) for _, X in terms]
    Z = [a * X[0] for a, X in terms]
    out = []
    for mu in range(1, d):
        rows = Z[0].shape[0] * Z[0].shape[1]
        Y = sum(Zb.reshape(rows, Zb.shape[2]) @ W[mu] for Zb, W in zip(Z, Ws))
        Q, _ = np.linalg.qr(Y)
        out.append(Q.reshape(Z[0].shape[0], Z[0].shape[1], Q.shape[1]))
        Mb = [Q.T @ Zb.reshape(rows, Zb.shape[2]) for Zb in Z]
        Z = [np.einsum("qp,pic->qic", M, X[mu]) for M, (_, X) in zip(Mb, terms)]
    out.append(sum(Z))
    if truncation == "simultaneous":
        trunc = eps > 0.0 or any(c.shape[2] > (rmax if rmax is not None else 1 << 60)
                                 for c in out[:-1])
        return truncate_simultaneous(out, eps, rmax) if trunc else out
    # 3. truncation sweep
    nrm = np.linalg.norm(out[-1])
    delta = eps * nrm / np.sqrt(d - 1)
    for mu in range(d - 1, 0, -1):
        r0, n, r1 = out[mu].shape
        U, s, Vt = np.linalg.svd(out[mu].reshape(r0, n * r1), full_matrices=False)
        r = truncation_rank(s, delta, rmax)
        out[mu] = Vt[:r].reshape(r, n, r1)
        out[mu - 1] = np.einsum("aib,bc->aic", out[mu - 1], U[:, :r] * s[:r])
    return out
