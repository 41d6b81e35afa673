"""Oracle: right-preconditioned restarted GMRES(m) with modified Gram-Schmidt, FP64.

Test infrastructure only (see oracle/analysis.py).

Sec. 6 runs GMRES(30) with modified Gram-Schmidt and a zero initial guess,
preconditioned by the approximate multifrontal factorization.  Reading: right
preconditioning, A M^-1 y = b, x = M^-1 y, and the stopping test is on the
true residual ||b - A x|| / ||b|| <= rtol, recomputed by an explicit sparse
product at every restart and at exit.  Each right-hand side is independent.
Iterative refinement (used for the exact solver in Sec. 6) is refine().
"""
from __future__ import annotations

import numpy as np


def gmres_one(A, b, Minv, rtol=1e-8, restart=30, max_iters=300):
    n = len(b)
    nb = np.linalg.norm(b)
    x = np.zeros(n, np.complex128)
    if nb == 0:
        return x, 0, 0.0
    its = 0
    r = b.copy()
    res = 1.0
    while its < max_iters:
        beta = np.linalg.norm(r)
        if beta / nb <= rtol:
            break
        V = np.zeros((n, restart + 1), np.complex128)
        H = np.zeros((restart + 1, restart), np.complex128)
        cs = np.zeros(restart, np.complex128)
        sn = np.zeros(restart, np.complex128)
        g = np.zeros(restart + 1, np.complex128)
        g[0] = beta
        V[:, 0] = r / beta
        j_used = 0
        for j in range(restart):
            w = A @ Minv(V[:, j])
            for i in range(j + 1):                      # modified Gram-Schmidt
                H[i, j] = np.vdot(V[:, i], w)
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[:, j + 1] = w / H[j + 1, j]
            # complex Givens rotations G_i = [[conj(c), conj(s)], [-s, c]], c = a / d, s = b / d,
            # d = sqrt(|a|^2 + |b|^2): G_i (a, b) = (d, 0), so R = G H is upper triangular
            for i in range(j):                          # previous rotations
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, bb = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            cs[j] = a / den if den else 1.0
            sn[j] = bb / den if den else 0.0
            H[j, j] = den if den else a
            H[j + 1, j] = 0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            its += 1
            j_used = j + 1
            if abs(g[j + 1]) / nb <= rtol or its >= max_iters:
                break
        y = np.linalg.solve(np.triu(H[:j_used, :j_used]), g[:j_used])
        x = x + Minv(V[:, :j_used] @ y)
        r = b - A @ x
        res = np.linalg.norm(r) / nb
        if res <= rtol:
            break
    return x, its, np.linalg.norm(b - A @ x) / nb


def gmres(A, B, Minv, rtol=1e-8, restart=30, max_iters=300):
    B = np.asarray(B, np.complex128)
    if B.ndim == 1:
        B = B[:, None]
    X = np.zeros_like(B)
    its, res = [], []
    for c in range(B.shape[1]):
        x, it, rr = gmres_one(A, B[:, c], Minv, rtol, restart, max_iters)
        X[:, c] = x
        its.append(it)
        res.append(rr)
    return X, its, res


def refine(A, B, Minv, rtol=1e-8, max_iters=50):
    """Iterative refinement x <- x + M^-1 (b - A x) until the true residual meets rtol."""
    B = np.asarray(B, np.complex128)
    if B.ndim == 1:
        B = B[:, None]
    X = Minv(B)
    nb = np.linalg.norm(B, axis=0)
    its = 0
    while its < max_iters:
        R = B - A @ X
        if np.all(np.linalg.norm(R, axis=0) <= rtol * nb):
            break
        X = X + Minv(R)
        its += 1
    return X, its, np.linalg.norm(B - A @ X, axis=0) / nb
