"""Oracle: hierarchically off-diagonal butterfly (HOD-BF) matrices (Sec. 4), complex128.

Test infrastructure only (see oracle/analysis.py).

HOD-BF (Sec. 4, Fig. 4): a cluster tree T_H of uniform depth L_H over [0, n);
dense leaf blocks D_tau; for every node tau at level l >= 1 the off-diagonal
block K(tau, sibling(tau)) is a butterfly with L_H - l levels over the two
subtrees (leaf siblings: 0 levels, i.e. low rank).

  hodbf_entry_eval  Sec. 4.1 (Alg. 2 on every off-diagonal block)
  extract_hodbf     Sec. 4.1 (dense leaves + Alg. 3 per off-diagonal block)
  hodbf_invert      Alg. 4 (recursive; B_tau_i <- D_tau_i^-1 B_tau_i by
                    randomized products; BF_SMW for [I B1; B2 I]^-1)
  bf_smw            Alg. 4, BF_SMW: (I + K)^-1 = I + K' for a butterfly K,
                    split into four (L-2)-level children, recursion, and
                    reconstruction by randomized products; L = 0 is the
                    low-rank Sherman-Morrison-Woodbury formula and L = 1 the
                    same formula with the rank <= 2r factors of the level.

The inverse is kept in the product form that Alg. 4 produces:
  D^-1 = M_root diag(M_level1) ... diag(M_level(L_H-1)) diag(D_leaf^-1),
with M_tau = I + K'_tau and K'_tau a butterfly over subtree(tau).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .butterfly import (Butterfly, Operator, Proxies, bf_entry_eval, bf_random_matvec,
                        bf_split, subtree, extend_tree)
from .idq import FLOPS


class HODBF:
    def __init__(self, n, tree):
        self.n = n
        self.tree = tree
        self.LH = len(tree) - 1
        self.D = {}
        self.off = {}          # (l, i) -> Butterfly for K(node(l,i), node(l,i^1))

    def rng(self, l, i):
        return self.tree[l][i]

    def apply(self, x, transpose=False):
        x = np.asarray(x, np.complex128)
        vec = x.ndim == 1
        if vec:
            x = x[:, None]
        y = np.zeros_like(x)
        for i, (a, b) in enumerate(self.tree[self.LH]):
            D = self.D[i]
            y[a:b] += (D.T if transpose else D) @ x[a:b]
            FLOPS[0] += 8 * D.size * x.shape[1]
        for (l, i), bf in self.off.items():
            a, b = self.rng(l, i)
            c, d = self.rng(l, i ^ 1)
            if transpose:      # (K(tau, sib))^T maps x(tau) -> y(sib)
                y[c:d] += bf.applyT(x[a:b])
            else:
                y[a:b] += bf.apply(x[c:d])
        return y[:, 0] if vec else y

    def applyT(self, x):
        return self.apply(x, transpose=True)

    def dense(self):
        return self.apply(np.eye(self.n, dtype=np.complex128))

    def storage(self):
        return sum(D.size for D in self.D.values()) + sum(bf.storage() for bf in self.off.values())

    def max_rank(self):
        return max([bf.max_rank() for bf in self.off.values()] + [0])

    def extract(self, lst):
        out = []
        for X, Y in lst:
            X = np.asarray(X, np.int64); Y = np.asarray(Y, np.int64)
            blk = np.zeros((len(X), len(Y)), np.complex128)
            if len(X) and len(Y):
                for i, (a, b) in enumerate(self.tree[self.LH]):
                    px = np.nonzero((X >= a) & (X < b))[0]
                    py = np.nonzero((Y >= a) & (Y < b))[0]
                    if len(px) and len(py):
                        blk[np.ix_(px, py)] += self.D[i][np.ix_(X[px] - a, Y[py] - a)]
                for (l, i), bf in self.off.items():
                    a, b = self.rng(l, i)
                    c, d = self.rng(l, i ^ 1)
                    px = np.nonzero((X >= a) & (X < b))[0]
                    py = np.nonzero((Y >= c) & (Y < d))[0]
                    if len(px) and len(py):
                        blk[np.ix_(px, py)] += bf.extract([(X[px] - a, Y[py] - c)])[0]
            out.append(blk)
        return out


def block_proxies(nn_global, rows_off, cols_off, nrows, ncols, alpha, knn, nn_col_global=None):
    """Proxies for the block [rows_off, +nrows) x [cols_off, +ncols) of an
    index space in which nn_global[x] lists neighbours of x (same space)."""
    nn_col_global = nn_col_global if nn_col_global is not None else nn_global
    nn_r = [[c - cols_off for c in nn_global[rows_off + x] if cols_off <= c < cols_off + ncols] for x in range(nrows)]
    nn_c = [[r - rows_off for r in nn_col_global[cols_off + y] if rows_off <= r < rows_off + nrows] for y in range(ncols)]
    return Proxies(nn_r, nn_c, alpha, knn)


def hodbf_entry_eval(extract, n, tree, nn, alpha, knn, tol, max_rank=0):
    """Sec. 4.1: dense leaves by extraction, Alg. 2 on every off-diagonal block.

    extract(lst) returns K(X, Y) for index arrays in [0, n); nn[x] lists
    graph neighbours of x in [0, n)."""
    H = HODBF(n, tree)
    LH = H.LH
    leaves = tree[LH]
    blocks = extract([(np.arange(a, b), np.arange(a, b)) for a, b in leaves])
    for i, Bk in enumerate(blocks):
        H.D[i] = Bk
    for l in range(1, LH + 1):
        for i in range(1 << l):
            a, b = tree[l][i]
            c, d = tree[l][i ^ 1]
            Lb = LH - l
            rt = subtree(tree, l, i, Lb)
            ct = subtree(tree, l, i ^ 1, Lb)
            ext = (lambda a, c: (lambda lst: extract([(X + a, Y + c) for X, Y in lst])))(a, c)
            prox = block_proxies(nn, a, c, b - a, d - c, alpha, knn)
            H.off[(l, i)] = bf_entry_eval(ext, b - a, d - c, rt, ct, Lb, prox, tol, max_rank)
    return H


# ---------------------------------------------------------------------------
# BF_SMW (Alg. 4)
# ---------------------------------------------------------------------------
def _smw_L0(bf):
    """(I + U B V^T)^-1 = I - U B (I + V^T U B)^-1 V^T  (Woodbury)."""
    out = Butterfly(bf.m, bf.n, bf.rtree, bf.ctree, 0)
    U, V, B = bf.U[(0, 0, 0)], bf.V[(0, 0, 0)], bf.B[(0, 0)]
    c = B.shape[1]
    G = np.eye(c) + V.T @ U @ B
    FLOPS[0] += 8 * (V.size * U.shape[1] + c * c * B.shape[0] + c ** 3)
    out.U[(0, 0, 0)] = U
    out.Osk[(0, 0, 0)] = bf.Osk[(0, 0, 0)]
    out.V[(0, 0, 0)] = V
    out.Ssk[(0, 0, 0)] = bf.Ssk[(0, 0, 0)]
    out.B[(0, 0)] = -np.linalg.solve(G.T, B.T).T if c else B.copy()
    return out


def _smw_L1(bf):
    """L = 1: K = Ubar Mbar with Ubar = diag(U_0, U_1) (level 1) and
    Mbar = [R_0 B_0 V_0^T, R_1 B_1 V_1^T]; (I + Ubar Mbar)^-1 = I - Ubar (I + Mbar Ubar)^-1 Mbar,
    kept in the same 1-level form by replacing R_j with -(I + Mbar Ubar)^-1 R_j."""
    out = Butterfly(bf.m, bf.n, bf.rtree, bf.ctree, 1)
    for key in bf.U:
        out.U[key] = bf.U[key]
        out.Osk[key] = bf.Osk[key]
    for key in bf.V:
        out.V[key] = bf.V[key]
        out.Ssk[key] = bf.Ssk[key]
    for key in bf.B:
        out.B[key] = bf.B[key]
    r0 = bf.rank_r(1, 0, 0)
    r1 = bf.rank_r(1, 1, 0)
    U0, U1 = bf.U[(1, 0, 0)], bf.U[(1, 1, 0)]
    a0, b0 = bf.rtree[1][0]
    a1, b1 = bf.rtree[1][1]
    MU = np.zeros((r0 + r1, r0 + r1), np.complex128)
    for j in range(2):
        ca, cb = bf.ctree[1][j]
        # V_j^T Ubar(S_j, :)
        Ub = np.zeros((cb - ca, r0 + r1), np.complex128)
        lo, hi = max(ca, a0), min(cb, b0)
        if lo < hi:
            Ub[lo - ca:hi - ca, :r0] = U0[lo - a0:hi - a0]
        lo, hi = max(ca, a1), min(cb, b1)
        if lo < hi:
            Ub[lo - ca:hi - ca, r0:] = U1[lo - a1:hi - a1]
        MU += bf.U[(0, 0, j)] @ bf.B[(0, j)] @ (bf.V[(0, 0, j)].T @ Ub)
    G = np.eye(r0 + r1) + MU
    FLOPS[0] += 8 * (r0 + r1) ** 3
    for j in range(2):
        out.U[(0, 0, j)] = -np.linalg.solve(G, bf.U[(0, 0, j)])
    return out


def bf_smw(bf: Butterfly, tol, max_rank, key):
    """BF_SMW of Alg. 4 for A = I + K, K = bf (square, rows and columns on the same tree)."""
    L = bf.L
    if L == 0:
        return _smw_L0(bf)
    if L == 1:
        return _smw_L1(bf)
    kids = bf_split(bf)
    K11, K12, K21, K22 = kids[(0, 0)], kids[(0, 1)], kids[(1, 0)], kids[(1, 1)]
    K22i = bf_smw(K22, tol, max_rank, key * 4 + 1)
    return _smw_assemble(bf.m, bf.rtree, bf.ctree, L, K11, K12, K21, K22i, tol, max_rank, key)


def _smw_assemble(n, rtree, ctree, L, K11, K12, K21, K22i, tol, max_rank, key):
    """Given the quadrants of K (K11 and K22 may be None for zero) and
    (I + K22)^-1 = I + K22i, build (I + K)^-1 - I as an L-level butterfly."""
    n1 = rtree[1][0][1]
    inv22 = (lambda x: x + K22i.apply(x)) if K22i is not None else (lambda x: x)
    inv22T = (lambda x: x + K22i.applyT(x)) if K22i is not None else (lambda x: x)
    # A11 <- K11 - K12 (I + K22i) K21   (randomized products, L-2 levels)
    def s_apply(x):
        y = -K12.apply(inv22(K21.apply(x)))
        return y + K11.apply(x) if K11 is not None else y
    def s_applyT(x):
        y = -K21.applyT(inv22T(K12.applyT(x)))
        return y + K11.applyT(x) if K11 is not None else y
    rt1 = subtree(rtree, 1, 0, L - 2)
    ct1 = subtree(ctree, 1, 0, L - 2)
    S = bf_random_matvec(Operator(n1, n1, s_apply, s_applyT), rt1, ct1, L - 2, tol, max_rank, key * 4 + 2)
    K11i = bf_smw(S, tol, max_rank, key * 4 + 3)
    inv11 = lambda x: x + K11i.apply(x)
    inv11T = lambda x: x + K11i.applyT(x)

    # A^-1 = [I 0; -A22^-1 A21 I] diag(A11^-1, A22^-1) [I -A12 A22^-1; 0 I]
    def f_apply(x):
        x1, x2 = x[:n1], x[n1:]
        t1 = x1 - K12.apply(inv22(x2))
        u1 = inv11(t1)
        u2 = inv22(x2)
        y2 = u2 - inv22(K21.apply(u1))
        return np.vstack([u1, y2]) - x
    def f_applyT(x):
        # transpose of the product, factors reversed
        x1, x2 = x[:n1], x[n1:]
        v1 = x1 - K21.applyT(inv22T(x2))
        w1 = inv11T(v1)
        w2 = inv22T(x2)
        z2 = w2 - inv22T(K12.applyT(w1))
        return np.vstack([w1, z2]) - x
    return bf_random_matvec(Operator(n, n, f_apply, f_applyT), rtree, ctree, L, tol, max_rank, key * 4)


class HODBFInverse:
    """D^-1 in the product form of Alg. 4 (see module docstring)."""

    def __init__(self, n, tree):
        self.n, self.tree, self.LH = n, tree, len(tree) - 1
        self.leaf = {}     # i -> (lu, piv) of D_leaf (FP64 pivoting LU)
        self.M = {}        # (l, i) -> Butterfly K' with M = I + K', l = 0 .. LH-1

    def apply_sub(self, x, l0, i0, transpose=False):
        """Inverse of the diagonal block of node (l0, i0), applied to x (rows of that node)."""
        a0, b0 = self.tree[l0][i0]
        y = np.array(x, np.complex128, copy=True)
        nsub = 1 << (self.LH - l0)
        leaves = range(i0 * nsub, (i0 + 1) * nsub)
        order = list(range(self.LH - 1, l0 - 1, -1))
        def leaf_solve(y):
            for i in leaves:
                a, b = self.tree[self.LH][i]
                if b > a:
                    y[a - a0:b - a0] = sla.lu_solve(self.leaf[i], y[a - a0:b - a0], trans=1 if transpose else 0)
                    FLOPS[0] += 8 * (b - a) ** 2 * y.shape[1]
            return y
        def level(y, l):
            span = 1 << (l - l0)
            for i in range(i0 * span, (i0 + 1) * span):
                a, b = self.tree[l][i]
                K = self.M[(l, i)]
                seg = y[a - a0:b - a0]
                y[a - a0:b - a0] = seg + (K.applyT(seg) if transpose else K.apply(seg))
            return y
        if not transpose:
            y = leaf_solve(y)
            for l in order:
                y = level(y, l)
        else:
            for l in reversed(order):
                y = level(y, l)
            y = leaf_solve(y)
        return y

    def apply(self, x):
        x = np.asarray(x, np.complex128)
        vec = x.ndim == 1
        if vec:
            x = x[:, None]
        y = self.apply_sub(x, 0, 0)
        return y[:, 0] if vec else y

    def applyT(self, x):
        x = np.asarray(x, np.complex128)
        vec = x.ndim == 1
        if vec:
            x = x[:, None]
        y = self.apply_sub(x, 0, 0, transpose=True)
        return y[:, 0] if vec else y

    def storage(self):
        return sum(lu[0].size for lu in self.leaf.values()) + sum(K.storage() for K in self.M.values())


def hodbf_invert(H: HODBF, tol, max_rank=0, key=7):
    """Alg. 4 (HODBF_invert), bottom-up over the levels of T_H."""
    inv = HODBFInverse(H.n, H.tree)
    LH = H.LH
    for i, D in H.D.items():
        inv.leaf[i] = sla.lu_factor(D)
        FLOPS[0] += 8 * D.shape[0] ** 3 / 3
    for l in range(LH - 1, -1, -1):
        for i in range(1 << l):
            t1, t2 = 2 * i, 2 * i + 1
            a, b = H.tree[l][i]
            a1, b1 = H.tree[l + 1][t1]
            a2, b2 = H.tree[l + 1][t2]
            n1, n2 = b1 - a1, b2 - a2
            Lq = LH - l - 1
            Bs = []
            for (tt, ts, na, nb) in ((t1, t2, n1, n2), (t2, t1, n2, n1)):
                Boff = H.off[(l + 1, tt)]
                op = Operator(na, nb,
                              (lambda Bo, tt: lambda x: inv.apply_sub(Bo.apply(x), l + 1, tt))(Boff, tt),
                              (lambda Bo, tt: lambda x: Bo.applyT(inv.apply_sub(x, l + 1, tt, transpose=True)))(Boff, tt))
                rt = subtree(H.tree, l + 1, tt, Lq)
                ct = subtree(H.tree, l + 1, ts, Lq)
                Bs.append(bf_random_matvec(op, rt, ct, Lq, tol, max_rank, key=(key * 131 + l * 17 + tt) & 0xFFFFF))
            B1, B2 = Bs
            # BF_SMW([I B1; B2 I]) as a (Lq + 2)-level butterfly over subtree(tau),
            # extended one level below the leaves of T_H.
            L = Lq + 2
            tr = extend_tree(subtree(H.tree, l, i, LH - l), L)
            inv.M[(l, i)] = _smw_assemble(b - a, tr, tr, L, None, B1, B2, None, tol, max_rank,
                                          key=(key * 977 + l * 31 + i) & 0xFFFFF)
    return inv
