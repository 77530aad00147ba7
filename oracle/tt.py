"""TT containers and exact TT arithmetic in float64 (Section 2.2 of the paper).

A TT vector is a Python list of cores ``C_k`` with shape ``[r_{k-1}, n_k, r_k]``
and ``r_0 = r_d = 1`` (eq. ``tt-format``).  A TT operator is a list of cores
``D_k`` with shape ``[R_{k-1}, n_out, n_in, R_k]`` (eq. ``operator
tt-format``).  Full tensors use C order (``i_1`` slowest).
"""
from __future__ import annotations

import numpy as np


def check_tt(cores):
    """Validate a TT: 3-D cores, matching bond ranks, ``r_0 = r_d = 1``."""
    if len(cores) == 0:
        raise ValueError("empty TT")
    if cores[0].shape[0] != 1 or cores[-1].shape[2] != 1:
        raise ValueError("boundary ranks must be 1")
    for a, b in zip(cores[:-1], cores[1:]):
        if a.shape[2] != b.shape[0]:
            raise ValueError("bond rank mismatch")
    return cores


def ranks(cores):
    """Rank tuple ``(r_0, r_1, ..., r_d)``."""
    return [c.shape[0] for c in cores] + [cores[-1].shape[2]]


def full(cores) -> np.ndarray:
    """Dense vector of a TT, entry ``T[i_1..i_d] = C_1[0,i_1,:] C_2[:,i_2,:] ..
    C_d[:,i_d,0]`` (eq. ``tt-format``), in C order.  The product is formed
    core by core: the running matrix has rows ``(i_1..i_k)`` and columns
    ``r_k``."""
    check_tt(cores)
    X = cores[0].reshape(cores[0].shape[1], cores[0].shape[2])
    for c in cores[1:]:
        r0, n, r1 = c.shape
        X = (X @ c.reshape(r0, n * r1)).reshape(-1, r1)
    return X.reshape(-1)


def op_full(op) -> np.ndarray:
    """Dense matrix of a TT operator: ``A[(i_1..i_d),(j_1..j_d)] = D_1[0,i_1,j_1,:]
    .. D_d[:,i_d,j_d,0]`` (eq. ``operator tt-format``)."""
    R0, n, m, R1 = op[0].shape
    # running tensor indexed [I, J, R] with I, J the merged row/column indices
    X = op[0].reshape(n, m, R1)
    for c in op[1:]:
        Ra, n2, m2, Rb = c.shape
        X = np.einsum("IJa,aijb->IiJjb", X, c)
        I, J = X.shape[0] * n2, X.shape[2] * m2
        X = X.reshape(I, J, Rb)
    return X[:, :, 0]


def matvec(op, cores):
    """Cores of ``y = A v`` (Section 2.2, matvec formula):
    ``G_k[(a, l), i, (a', l')] = sum_j D_k[a, i, j, a'] C_k[l, j, l']``.

    The merged rank index is ``a * r + l`` (operator rank slowest), so the
    output ranks are ``R_k r_k`` exactly.
    """
    out = []
    for D, C in zip(op, cores):
        Ra, n, m, Rb = D.shape
        ra, m2, rb = C.shape
        if m != m2:
            raise ValueError("operator column size does not match the vector mode size")
        G = np.einsum("aijb,ljm->alibm", D, C)
        out.append(G.reshape(Ra * ra, n, Rb * rb))
    return out


def transpose_op(op):
    """Cores of ``A^T``: ``D[a, i, j, a'] -> D[a, j, i, a']``."""
    return [np.ascontiguousarray(D.transpose(0, 2, 1, 3)) for D in op]


def dot(x, y) -> float:
    """``<x, y>`` by the left-to-right Gram sweep ``Z_k = sum_i X_k[:, i, :]^T
    Z_{k-1} Y_k[:, i, :]`` with ``Z_0 = 1``; the result is ``Z_d``."""
    if len(x) != len(y):
        raise ValueError("different number of modes")
    Z = np.ones((1, 1))
    for X, Y in zip(x, y):
        if X.shape[1] != Y.shape[1]:
            raise ValueError("mode size mismatch")
        Zn = np.zeros((X.shape[2], Y.shape[2]))
        for i in range(X.shape[1]):
            Zn += X[:, i, :].T @ Z @ Y[:, i, :]
        Z = Zn
    return float(Z[0, 0])


def norm(x) -> float:
    """``||x||_F`` from the Gram sweep."""
    return float(np.sqrt(max(dot(x, x), 0.0)))


def scale(x, a):
    """``a * x`` (the scalar is applied to the first core)."""
    out = [c.copy() for c in x]
    out[0] = out[0] * a
    return out


def add(terms):
    """Explicit TT of ``sum_b a_b X^(b)``: first cores concatenated along the
    right rank, middle cores block-diagonal, last cores stacked along the
    left rank; ``a_b`` multiplies the first core of term b."""
    d = len(terms[0][1])
    out = []
    for k in range(d):
        blocks = [X[k] * (a if k == 0 else 1.0) for a, X in terms]
        n = blocks[0].shape[1]
        if d == 1:
            out.append(sum(blocks))
        elif k == 0:
            out.append(np.concatenate(blocks, axis=2))
        elif k == d - 1:
            out.append(np.concatenate(blocks, axis=0))
        else:
            r0 = sum(b.shape[0] for b in blocks)
            r1 = sum(b.shape[2] for b in blocks)
            C = np.zeros((r0, n, r1))
            p = q = 0
            for b in blocks:
                C[p:p + b.shape[0], :, q:q + b.shape[2]] = b
                p += b.shape[0]
                q += b.shape[2]
            out.append(C)
    return out


def sketch_kr(cores, S):
    """Khatri-Rao sketch ``S_odot x`` (Section 3.1): row j equals
    ``prod_k (sum_i S_k[j, i] C_k[:, i, :])``, evaluated left to right for all
    rows (a 1 x r_k row vector per sketch row)."""
    s = S[0].shape[0]
    out = np.zeros(s)
    for j in range(s):
        z = np.ones((1, 1))
        for Sk, C in zip(S, cores):
            z = z @ np.einsum("i,aib->ab", Sk[j], C)
        out[j] = z[0, 0]
    return out


def sketch_kr_fast(cores, S):
    """Same product as :func:`sketch_kr`, all rows at once: ``Z_k[j, :] =
    Z_{k-1}[j, :] (sum_i S_k[j, i] C_k[:, i, :])`` (used at larger sizes)."""
    s = S[0].shape[0]
    Z = np.ones((s, 1))
    for Sk, C in zip(S, cores):
        M = np.einsum("ji,aib->jab", Sk, C)
        Z = np.einsum("ja,jab->jb", Z, M)
    return Z[:, 0]


def sketch_dense(xfull, S):
    """Explicit Khatri-Rao sketch of a dense vector: row j of ``S_odot`` is
    ``S_1[j, :] kron ... kron S_d[j, :]`` (Section 3.1)."""
    s = S[0].shape[0]
    out = np.zeros(s)
    for j in range(s):
        row = np.ones(1)
        for Sk in S:
            row = np.kron(row, Sk[j])
        out[j] = row @ xfull
    return out


def sketch_tt_rows(cores, Y):
    """Sketch whose row j is a TT tensor of its own (rank R > 1 generalises the
    Khatri-Rao rows, which are rank 1): ``(S x)_j = <Y_j, x>`` by the Gram sweep
    ``Z_k = sum_i Y_k[j, :, i, :]^T Z_{k-1} C_k[:, i, :]``.  ``Y[k]`` has shape
    ``[s][R_{k-1}][n_k][R_k]`` (R_0 = R_d = 1).  Not in the paper: reading
    beyond the Khatri-Rao sketch, for a sketch that still embeds at large d."""
    s = Y[0].shape[0]
    out = np.zeros(s)
    for j in range(s):
        Z = np.ones((1, 1))
        for Yk, C in zip(Y, cores):
            Z = sum(Yk[j, :, i, :].T @ Z @ C[:, i, :] for i in range(C.shape[1]))
        out[j] = Z[0, 0]
    return out


def sketch_tt_rows_dense(xfull, Y):
    """Row j of the TT-row sketch formed explicitly as the full tensor of the
    TT ``Y_j`` and applied to the dense vector."""
    s = Y[0].shape[0]
    return np.array([full([Yk[j] for Yk in Y]) @ xfull for j in range(s)])


def left_orthogonalize(cores):
    """QR sweep left to right; returns cores 1..d-1 left-orthogonal and the
    represented tensor unchanged."""
    out = [c.copy() for c in cores]
    for k in range(len(out) - 1):
        r0, n, r1 = out[k].shape
        Q, R = np.linalg.qr(out[k].reshape(r0 * n, r1))
        out[k] = Q.reshape(r0, n, Q.shape[1])
        out[k + 1] = np.einsum("ab,bic->aic", R, out[k + 1])
    return out


def right_orthogonalize(cores):
    """QR sweep right to left; cores 2..d right-orthogonal."""
    out = [c.copy() for c in cores]
    for k in range(len(out) - 1, 0, -1):
        r0, n, r1 = out[k].shape
        Q, R = np.linalg.qr(out[k].reshape(r0, n * r1).T)
        out[k] = Q.T.reshape(Q.shape[1], n, r1)
        out[k - 1] = np.einsum("aib,cb->aic", out[k - 1], R)
    return out


def entry(cores, idx) -> float:
    """One entry ``T[i_1..i_d]`` as the product of core slices."""
    z = np.ones((1, 1))
    for C, i in zip(cores, idx):
        z = z @ C[:, i, :]
    return float(z[0, 0])
