"""Krylov solvers in float64: sketched least squares, TT-sGMRES, TT-GMRES.

``tt_sgmres`` is the enhanced TT-sGMRES of Algorithm 4 with incomplete
orthogonalisation against the last ``l`` basis vectors (default 1), carried
out explicitly in TT format (the Remark after Section 3.6 recommends keeping
the last vectors for small l), with
randomize-then-orthogonalize rounding for the Gram-Schmidt step and for the
final solution ``x = sum_i y_i v_i`` (Section 3.5), the operator applied
without truncation (Section 3.2), and ``y_k = (S A V_k)^+ S r_0``
(eq. ``pseudo_inv``).

``solve`` wraps it in the restart loop of Section 3.4 (restart from the true
residual ``r_m = b - A x_m``), stopping on the true relative residual.

``tt_gmres`` is the full-orthogonalisation TT-GMRES of Algorithm 2 with TT-SVD
rounding, used as a deterministic reference solver on small problems.
"""
from __future__ import annotations

import numpy as np

from . import tt as ttm
from . import rounding as rnd


def sketched_lstsq(W, c):
    """``y = argmin ||W y - c||_2`` (eq. ``pseudo_inv``: ``y = W^+ c``) by
    LAPACK's SVD-based least squares, and the residual ``||W y - c||``."""
    W = np.asarray(W, dtype=np.float64)
    y = np.linalg.lstsq(W, c, rcond=None)[0]
    return y, float(np.linalg.norm(W @ y - c))


def true_residual_norm(op, x, b):
    """``||b - A x||`` in exact TT arithmetic: the explicit sum ``b - A x``
    is left-orthogonalised by QR and the norm read off the last core (a QR
    sweep keeps the cancellation error at the level of ``eps ||b||``)."""
    r = ttm.add([(1.0, b), (-1.0, ttm.matvec(op, x))])
    r = ttm.left_orthogonalize(r)
    return float(np.linalg.norm(r[-1]))


def tt_sgmres(op, b, S, drm, maxit, tol, round_tol, rmax, oversample=10,
              r_sol=None, final_tol=None, ell=1):
    """Algorithm 4, zero initial guess, RTO rounding.

    Parameters
    ----------
    op, b : TT operator and right-hand side.
    S : Khatri-Rao factors, list of ``[s, n_k]`` arrays.
    drm : Gaussian TT-DRM used by every randomized rounding (leading
        sub-blocks; see :func:`oracle.rounding.rto_round`).
    maxit : Krylov dimension cap.
    tol : sketched stopping tolerance, ``||W y - S r0|| <= tol ||S r0||``.
    round_tol : relative tolerance of the Gram-Schmidt rounding (``eta tol``).
    rmax : rank cap of the basis vectors.
    r_sol, final_tol : rank cap and tolerance of the final rounding.
    ell : incomplete orthogonalisation: ``h_{i,k} = w^T v_i`` for the last
        ``ell`` basis vectors and ``v~ = Round(w - sum_i h_{i,k} v_i)``
        (Section 3.4).

    Returns ``(x, info)`` with the sketched residual history, basis ranks, the
    number of iterations, the basis ``V`` and the coefficients ``H``
    (``H[i][k] = h_{i,k}``, with ``h_{k+1,k}`` the norm of the rounded vector).
    """
    r_sol = rmax if r_sol is None else r_sol
    final_tol = round_tol if final_tol is None else final_tol
    beta = ttm.norm(b)
    v = ttm.scale(b, 1.0 / beta)
    Sr0 = ttm.sketch_kr_fast(b, S)
    betaS = float(np.linalg.norm(Sr0))
    V = [v]
    Wcols = []
    hist, rank_hist = [], []
    H = np.zeros((maxit + 1, maxit))
    y = None
    k = 0
    for k in range(1, maxit + 1):
        w = ttm.matvec(op, V[-1])                       # untruncated A v_k
        Wcols.append(ttm.sketch_kr_fast(w, S))          # W_k = [W_{k-1}, S w]
        first = max(0, len(V) - ell)
        terms = [(1.0, w)]
        for i in range(first, len(V)):                  # h_{i,k} = w^T v_i
            H[i, k - 1] = ttm.dot(w, V[i])
            terms.append((-H[i, k - 1], V[i]))
        vt = rnd.rto_round(terms, drm, eps=round_tol, rmax=rmax, oversample=oversample)
        hn = ttm.norm(vt)                                # h_{k+1,k}
        H[k, k - 1] = hn
        y, res = sketched_lstsq(np.stack(Wcols, axis=1), Sr0)
        hist.append(res / betaS)
        rank_hist.append(max(ttm.ranks(vt)))
        if res <= tol * betaS or hn == 0.0:
            break
        V.append(ttm.scale(vt, 1.0 / hn))
    terms = [(float(y[i]), V[i]) for i in range(len(y))]
    x = rnd.rto_round(terms, drm, eps=final_tol, rmax=r_sol, oversample=oversample)
    return x, dict(iters=k, res_hist=hist, rank_hist=rank_hist, V=V, H=H[:k + 1, :k])


def solve(op, b, S, drm, maxit, tol, round_tol, rmax, oversample=10, r_sol=None,
          final_tol=None, stop_safety=0.1, max_restarts=5, res_tol=None, ell=1):
    """Restarted TT-sGMRES (Section 3.4): run :func:`tt_sgmres` on the current
    residual, update ``x <- Round(x + e)``, recompute the true residual
    ``r = b - A x`` exactly and stop when ``||r|| / ||b|| <= tol``.

    The sketched stopping tolerance of each cycle is ``stop_safety * tol *
    ||b|| / ||r||`` (relative to the cycle's right-hand side); the residual
    handed to the next cycle is rounded at ``res_tol`` relative accuracy.
    """
    r_sol = rmax if r_sol is None else r_sol
    final_tol = 0.01 * tol if final_tol is None else final_tol
    res_tol = 0.01 if res_tol is None else res_tol
    bnorm = ttm.norm(b)
    x = None
    rhs = b
    rel = 1.0
    total = 0
    cycles = []
    for cyc in range(max_restarts + 1):
        inner_tol = min(0.5, stop_safety * tol / rel)
        e, info = tt_sgmres(op, rhs, S, drm, maxit, inner_tol, round_tol, rmax,
                            oversample=oversample, r_sol=r_sol, final_tol=final_tol, ell=ell)
        info = {k: v for k, v in info.items() if k not in ("V", "H")}
        total += info["iters"]
        if x is None:
            x = e
        else:
            x = rnd.rto_round([(1.0, x), (1.0, e)], drm, eps=final_tol, rmax=r_sol,
                              oversample=oversample)
        rel = true_residual_norm(op, x, b) / bnorm
        cycles.append(dict(info, true_res=rel))
        if rel <= tol:
            break
        r = ttm.add([(1.0, b), (-1.0, ttm.matvec(op, x))])
        rhs = rnd.tt_svd_round(r, eps=res_tol)
    return x, dict(iters=total, true_res=rel, cycles=cycles)


def tt_gmres(op, b, maxit, tol, round_tol):
    """Algorithm 2 (full orthogonalisation, modified Gram-Schmidt with a
    TT-SVD rounding after each update, Hessenberg least squares), zero initial
    guess.  The Hessenberg residual is the stopping test; the final solution
    adds the basis vectors one at a time with a rounding after each addition.
    ``round_tol`` replaces the iteration-dependent threshold of the paper
    (a fixed tight value makes this a reference solver)."""
    beta = ttm.norm(b)
    V = [ttm.scale(b, 1.0 / beta)]
    H = np.zeros((maxit + 1, maxit))
    y = np.zeros(0)
    k = 0
    for k in range(1, maxit + 1):
        w = rnd.tt_svd_round(ttm.matvec(op, V[-1]), eps=round_tol)
        for i in range(k):
            H[i, k - 1] = ttm.dot(w, V[i])
            w = rnd.tt_svd_round(ttm.add([(1.0, w), (-H[i, k - 1], V[i])]), eps=round_tol)
        H[k, k - 1] = ttm.norm(w)
        rhs = np.zeros(k + 1)
        rhs[0] = beta
        y, *_ = np.linalg.lstsq(H[:k + 1, :k], rhs, rcond=None)
        res = np.linalg.norm(H[:k + 1, :k] @ y - rhs)
        if res <= tol * beta or H[k, k - 1] == 0.0:
            break
        V.append(ttm.scale(w, 1.0 / H[k, k - 1]))
    x = ttm.scale(V[0], y[0])
    for i in range(1, len(y)):
        x = rnd.tt_svd_round(ttm.add([(1.0, x), (y[i], V[i])]), eps=round_tol)
    return x, dict(iters=k)
