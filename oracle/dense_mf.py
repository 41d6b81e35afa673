"""Oracle: exact (uncompressed) multifrontal factorization and solve, complex128.

Test infrastructure only (see oracle/analysis.py).  Follows Alg. 1 and the
four steps of Sec. 2 literally, one front at a time in topological order:
  1. F_tau = [A(Is,Is) A(Is,Iu); A(Iu,Is) 0]  (+)  C_nu1  (+)  C_nu2   (extend-add)
  2. P L U = F11 with partial pivoting inside F11 only (Sec. 2: the pivot
     search ignores F12 and F21); pivot = largest modulus, lowest row on ties
  3. F12 <- L^-1 P^T F12,  F21 <- F21 U^-1
  4. C_tau = F22 - F21 F12
Solve (Alg. 1 last line): forward z_s = L^-1 P^T b_s, b_u -= F21 z_s;
backward x_s = U^-1 (z_s - F12 x_u).
"""
from __future__ import annotations

import numpy as np


def permuted_matrix(prob, an):
    """A in the new numbering, as scipy CSR (rows/cols permuted by P A P^T)."""
    A = prob.to_scipy()
    Ap = A[an.perm][:, an.perm].tocsr()
    Ap.sort_indices()
    return Ap


def front_index(f):
    """Global new indices of the front's rows/columns: I^s then I^u."""
    return np.concatenate([np.arange(f.sep_begin, f.sep_end), f.upd])


def relative_map(child, parent):
    """Position in the parent front of every index of the child's update set."""
    gidx = front_index(parent)
    pos = {int(g): i for i, g in enumerate(gidx)}
    return np.array([pos[int(g)] for g in child.upd], dtype=np.int64)


def assemble_sparse(Ap, f):
    """[A(Is,Is) A(Is,Iu); A(Iu,Is) 0] as a dense n x n block (step 1 of Sec. 2)."""
    gidx = front_index(f)
    n = len(gidx)
    F = np.zeros((n, n), dtype=np.complex128)
    sub = Ap[gidx][:, gidx].toarray()
    s = f.s
    F[:s, :] = sub[:s, :]
    F[s:, :s] = sub[s:, :s]
    return F


def lu_partial_pivot(M):
    """In-place LU with partial pivoting by largest modulus (ties: lowest row).

    Returns (LU, piv) where piv[k] is the row swapped with row k at step k
    (LAPACK convention), L unit-lower and U upper packed in LU.
    """
    A = np.array(M, dtype=np.complex128, copy=True)
    s = A.shape[0]
    piv = np.zeros(s, dtype=np.int64)
    for k in range(s):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        piv[k] = p
        if p != k:
            A[[k, p], :] = A[[p, k], :]
        if A[k, k] == 0:
            raise ZeroDivisionError("zero pivot")
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    return A, piv


def apply_row_swaps(B, piv):
    B = B.copy()
    for k, p in enumerate(piv):
        if p != k:
            B[[k, p], :] = B[[p, k], :]
    return B


def lower_solve_unit(LU, B):
    """L^-1 B with L the unit lower triangle of LU (forward substitution)."""
    X = np.array(B, dtype=np.complex128, copy=True)
    s = LU.shape[0]
    for k in range(s):
        X[k + 1:] -= np.outer(LU[k + 1:, k], X[k])
    return X


def upper_solve(LU, B):
    """U^-1 B with U the upper triangle of LU (back substitution)."""
    X = np.array(B, dtype=np.complex128, copy=True)
    s = LU.shape[0]
    for k in range(s - 1, -1, -1):
        X[k] /= LU[k, k]
        X[:k] -= np.outer(LU[:k, k], X[k])
    return X


def right_upper_solve(LU, B):
    """B U^-1 (solve X U = B column by column)."""
    return upper_solve_T(LU, B.T).T


def upper_solve_T(LU, B):
    """U^-T B: forward substitution with U^T (lower)."""
    X = np.array(B, dtype=np.complex128, copy=True)
    s = LU.shape[0]
    for k in range(s):
        X[k] /= LU[k, k]
        X[k + 1:] -= np.outer(LU[k, k + 1:], X[k])
    return X


class DenseFrontFactor:
    def __init__(self, s, LU, piv, F12, F21):
        self.s, self.LU, self.piv, self.F12, self.F21 = s, LU, piv, F12, F21


def factor_front_dense(F, s):
    """Steps 2-4 of Sec. 2 on an assembled front; returns (factor, C)."""
    LU, piv = lu_partial_pivot(F[:s, :s])
    F12 = lower_solve_unit(LU, apply_row_swaps(F[:s, s:], piv))
    F21 = right_upper_solve(LU, F[s:, :s])
    C = F[s:, s:] - F21 @ F12
    return DenseFrontFactor(s, LU, piv, F12, F21), C


def multifrontal_factor(prob, an):
    """Exact multifrontal factorization (Alg. 1).  Returns the list of front factors."""
    Ap = permuted_matrix(prob, an)
    factors = [None] * len(an.fronts)
    cb = {}
    flops = 0
    for f in an.fronts:                       # post-order = topological order
        F = assemble_sparse(Ap, f)
        for c in f.children:
            rel = relative_map(an.fronts[c], f)
            F[np.ix_(rel, rel)] += cb.pop(c)  # extend-add, child block released
        fac, C = factor_front_dense(F, f.s)
        s, u = f.s, f.u
        flops += 8 * (s ** 3 / 3 + s * s * u + s * u * u)
        factors[f.id] = fac
        if f.parent >= 0:
            cb[f.id] = C
    return factors, flops


def multifrontal_solve(an, factors, b):
    """Forward/backward substitution through the tree (new numbering in/out)."""
    x = np.array(b, dtype=np.complex128, copy=True)
    if x.ndim == 1:
        x = x[:, None]
    for f in an.fronts:                        # forward, leaves -> root
        fac = factors[f.id]
        sl = slice(f.sep_begin, f.sep_end)
        z = lower_solve_unit(fac.LU, apply_row_swaps(x[sl], fac.piv))
        x[sl] = z
        if f.u:
            x[f.upd] -= fac.F21 @ z
    for f in reversed(an.fronts):              # backward, root -> leaves
        fac = factors[f.id]
        sl = slice(f.sep_begin, f.sep_end)
        rhs = x[sl]
        if f.u:
            rhs = rhs - fac.F12 @ x[f.upd]
        x[sl] = upper_solve(fac.LU, rhs)
    return x


def solve(prob, an, factors, b):
    """x = A^-1 b in the original numbering."""
    b = np.asarray(b)
    bp = b[an.perm]
    xp = multifrontal_solve(an, factors, bp)
    x = np.empty_like(xp)
    x[an.perm] = xp
    return x.reshape(b.shape) if b.ndim == 1 else x
