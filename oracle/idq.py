"""Oracle: interpolative decomposition by truncated column-pivoted QR (Sec. 3).

Test infrastructure only (see oracle/analysis.py).

Row ID of M (m x n): a column-pivoted Householder QR of M^T (Businger-Golub:
pivot = largest remaining column 2-norm, lowest index on ties) truncated at
rank k, the smallest k with |R_{k+1,k+1}| <= tol * |R_11| (relative reading of
"ID with a tolerance"), capped at max_rank (0 = no cap).  With M^T P = Q R,
the row ID is  M ~= P [I; (R11^-1 R12)^T] M(I,:) = U M(I,:)  where I are the
first k pivots.  Transposes are plain (not conjugate) transposes.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

FLOPS = [0]


def row_id(M: np.ndarray, tol: float, max_rank: int = 0):
    """Returns (U, sk): U is m x k with U[sk] = I_k and M ~= U @ M[sk]."""
    M = np.asarray(M, dtype=np.complex128)
    m, n = M.shape
    A = M.T.copy()                    # n x m ; columns of A are rows of M
    perm = np.arange(m)
    kmax = min(m, n)
    if max_rank > 0:
        kmax = min(kmax, max_rank)
    rank = 0
    ref = 0.0
    for k in range(kmax):
        norms = np.linalg.norm(A[k:, k:], axis=0)
        j = k + int(np.argmax(norms))
        nu = float(norms[j - k])
        if k == 0:
            ref = nu
            if ref == 0.0:
                break
        if nu <= tol * ref:
            break
        if j != k:
            A[:, [k, j]] = A[:, [j, k]]
            perm[[k, j]] = perm[[j, k]]
        x = A[k:, k].copy()
        nx = np.linalg.norm(x)
        phase = x[0] / abs(x[0]) if x[0] != 0 else 1.0
        alpha = -phase * nx
        v = x.copy()
        v[0] -= alpha
        nv = np.linalg.norm(v)
        if nv > 0:
            v /= nv
            A[k:, k:] -= 2.0 * np.outer(v, v.conj() @ A[k:, k:])
        A[k + 1:, k] = 0.0
        FLOPS[0] += 8 * 2 * (n - k) * (m - k)
        rank = k + 1
    r = rank
    U = np.zeros((m, r), dtype=np.complex128)
    if r:
        R11 = np.triu(A[:r, :r])
        R12 = A[:r, r:]
        T = sla.solve_triangular(R11, R12) if R12.shape[1] else np.zeros((r, 0), np.complex128)
        U[perm[:r]] = np.eye(r)
        U[perm[r:]] = T.T
    return U, perm[:r].copy()


def col_id(M: np.ndarray, tol: float, max_rank: int = 0):
    """Column ID M ~= M[:, sk] @ V.T (row ID of M^T)."""
    V, sk = row_id(np.asarray(M).T, tol, max_rank)
    return V, sk
