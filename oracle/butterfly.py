"""Oracle: butterfly matrices (Sec. 3), complex128.

Test infrastructure only (see oracle/analysis.py).

Representation (Sec. 3.1, Eq. (3.1)-(3.3), hybrid form of Fig. 2 with the
centre at l_c = floor(L/2)):
  Trees: rtree[l], ctree[l] are lists of (a, b) index ranges of the nodes at
  level l (2^l of them), levels 0..L, over [0, m) and [0, n).
  Pairs at level l: (i, j) with tau = node i of rtree level l and nu = node j
  of ctree level L - l.
  Left half, l = L .. l_c:  U[(l,i,j)] is the interpolation matrix U_{tau,nu}
    (l = L, shape |O_tau| x r) or the transfer matrix R_{tau,nu} (l < L, shape
    (r_{2i,j//2} + r_{2i+1,j//2}) x r) from a row ID; Osk[(l,i,j)] holds the
    skeleton rows (local row indices in [0, m)).
  Right half, l = 0 .. l_c:  V[(l,i,j)] is V_{tau,nu} (l = 0, |S_nu| x c) or
    the transfer W_{tau,nu} (l > 0, (c_{i//2,2j} + c_{i//2,2j+1}) x c) from a
    column ID, K(O_tau, Y) ~= K(O_tau, Ybar) V^T; Ssk[(l,i,j)] the skeleton
    columns.
  Centre: B[(i,j)] = K(Obar_{tau,nu}, Sbar_{tau,nu}) at level l_c.

Algorithms: apply / transpose apply (O(n log n), Sec. 3.1), extraction of a
list of sub-blocks (Alg. 3), construction from entry evaluation (Alg. 2),
construction from matrix-vector products (Sec. 3.2; the paper defers the
algorithm to its reference [liu2020butterfly] -- the reading implemented here
is an ID-based sketching variant of Alg. 2, see bf_random_matvec), and the
split of an L-level butterfly into its four (L-2)-level children (Alg. 4,
BF_SMW).
"""
from __future__ import annotations

import numpy as np

from workloads import counter_normal_complex
from .idq import row_id, FLOPS


def subtree(tree, l0, i0, depth):
    """Levels 0..depth of the subtree rooted at node i0 of level l0 (ranges shifted to start at 0)."""
    a0 = tree[l0][i0][0]
    out = []
    for d in range(depth + 1):
        lv = tree[l0 + d][i0 * (1 << d):(i0 + 1) * (1 << d)]
        out.append([(a - a0, b - a0) for a, b in lv])
    return out


def extend_tree(tree, depth):
    """Levels 0..depth; levels beyond the given ones bisect every range (first ceil half)."""
    out = [list(lv) for lv in tree[:depth + 1]]
    while len(out) < depth + 1:
        new = []
        for a, b in out[-1]:
            m = a + (b - a + 1) // 2
            new += [(a, m), (m, b)]
        out.append(new)
    return out


def _cat(*arrs):
    arrs = [np.asarray(a, dtype=np.int64) for a in arrs]
    return np.concatenate(arrs) if arrs else np.zeros(0, np.int64)


class Butterfly:
    def __init__(self, m, n, rtree, ctree, L):
        self.m, self.n, self.L = m, n, L
        self.lc = L // 2
        self.rtree = [list(x) for x in rtree[:L + 1]]
        self.ctree = [list(x) for x in ctree[:L + 1]]
        assert len(self.rtree) == L + 1 and len(self.ctree) == L + 1
        self.U, self.Osk, self.V, self.Ssk, self.B = {}, {}, {}, {}, {}

    def pairs(self, l):
        for i in range(1 << l):
            for j in range(1 << (self.L - l)):
                yield i, j

    def rank_r(self, l, i, j):
        return len(self.Osk[(l, i, j)])

    def rank_c(self, l, i, j):
        return len(self.Ssk[(l, i, j)])

    def max_rank(self):
        rs = [len(v) for v in self.Osk.values()] + [len(v) for v in self.Ssk.values()]
        return max(rs) if rs else 0

    def storage(self):
        """Number of stored complex entries."""
        return sum(x.size for d in (self.U, self.V, self.B) for x in d.values())

    # ---------------- products ----------------
    def right_transform(self, x):
        """x (n x k) -> dict of V_{tau,nu}^T x(S_nu) for all pairs at level l_c."""
        L, lc = self.L, self.lc
        xs = {}
        for j, (a, b) in enumerate(self.ctree[L]):
            V = self.V[(0, 0, j)]
            xs[(0, j)] = V.T @ x[a:b]
            FLOPS[0] += 8 * V.size * x.shape[1]
        for l in range(1, lc + 1):
            new = {}
            for i, j in self.pairs(l):
                W = self.V[(l, i, j)]
                new[(i, j)] = W.T @ np.vstack([xs[(i // 2, 2 * j)], xs[(i // 2, 2 * j + 1)]])
                FLOPS[0] += 8 * W.size * x.shape[1]
            xs = new
        return xs

    def apply(self, x):
        """y = K x (Eq. (3.3) read right to left)."""
        x = np.asarray(x, dtype=np.complex128)
        vec = x.ndim == 1
        if vec:
            x = x[:, None]
        L, lc = self.L, self.lc
        k = x.shape[1]
        xs = self.right_transform(x)
        ys = {}
        for i, j in self.pairs(lc):
            ys[(i, j)] = self.B[(i, j)] @ xs[(i, j)]
            FLOPS[0] += 8 * self.B[(i, j)].size * k
        for l in range(lc, L):
            new = {(i, j): np.zeros((self.rank_r(l + 1, i, j), k), np.complex128) for i, j in self.pairs(l + 1)}
            for i, j in self.pairs(l):
                R = self.U[(l, i, j)]
                z = R @ ys[(i, j)]
                FLOPS[0] += 8 * R.size * k
                r1 = self.rank_r(l + 1, 2 * i, j // 2)
                new[(2 * i, j // 2)] += z[:r1]
                new[(2 * i + 1, j // 2)] += z[r1:]
            ys = new
        y = np.zeros((self.m, k), np.complex128)
        for i, (a, b) in enumerate(self.rtree[L]):
            U = self.U[(L, i, 0)]
            y[a:b] = U @ ys[(i, 0)]
            FLOPS[0] += 8 * U.size * k
        return y[:, 0] if vec else y

    def applyT(self, x):
        """y = K^T x (plain transpose)."""
        x = np.asarray(x, dtype=np.complex128)
        vec = x.ndim == 1
        if vec:
            x = x[:, None]
        L, lc = self.L, self.lc
        k = x.shape[1]
        xs = {}
        for i, (a, b) in enumerate(self.rtree[L]):
            U = self.U[(L, i, 0)]
            xs[(i, 0)] = U.T @ x[a:b]
            FLOPS[0] += 8 * U.size * k
        for l in range(L - 1, lc - 1, -1):
            new = {}
            for i, j in self.pairs(l):
                R = self.U[(l, i, j)]
                new[(i, j)] = R.T @ np.vstack([xs[(2 * i, j // 2)], xs[(2 * i + 1, j // 2)]])
                FLOPS[0] += 8 * R.size * k
            xs = new
        ys = {}
        for i, j in self.pairs(lc):
            ys[(i, j)] = self.B[(i, j)].T @ xs[(i, j)]
            FLOPS[0] += 8 * self.B[(i, j)].size * k
        for l in range(lc, 0, -1):
            new = {(i, j): np.zeros((self.rank_c(l - 1, i, j), k), np.complex128) for i, j in self.pairs(l - 1)}
            for i, j in self.pairs(l):
                W = self.V[(l, i, j)]
                z = W @ ys[(i, j)]
                FLOPS[0] += 8 * W.size * k
                c1 = self.rank_c(l - 1, i // 2, 2 * j)
                new[(i // 2, 2 * j)] += z[:c1]
                new[(i // 2, 2 * j + 1)] += z[c1:]
            ys = new
        y = np.zeros((self.n, k), np.complex128)
        for j, (a, b) in enumerate(self.ctree[L]):
            V = self.V[(0, 0, j)]
            y[a:b] = V @ ys[(0, j)]
            FLOPS[0] += 8 * V.size * k
        return y[:, 0] if vec else y

    def dense(self):
        return self.apply(np.eye(self.n, dtype=np.complex128))

    # ---------------- extraction (Alg. 3) ----------------
    def extract(self, lst):
        """K(X, Y) for every (X, Y) in lst; X, Y are arrays of local indices."""
        return [self._extract_one(np.asarray(X, np.int64), np.asarray(Y, np.int64)) for X, Y in lst]

    def _extract_one(self, X, Y):
        L, lc = self.L, self.lc
        out = np.zeros((len(X), len(Y)), np.complex128)
        if len(X) == 0 or len(Y) == 0:
            return out
        # rows of X inside each row node, per level (positions into X)
        def rows_in(tree, l, idx):
            res = []
            for a, b in tree[l]:
                res.append(np.nonzero((idx >= a) & (idx < b))[0])
            return res
        Xin = [rows_in(self.rtree, l, X) for l in range(L + 1)]
        Yin = [rows_in(self.ctree, l, Y) for l in range(L + 1)]
        # E^l_{tau,nu} for pairs with X cap O_tau and Y cap S_nu non-empty (l = L .. l_c)
        E = {}
        for i in range(1 << L):
            px = Xin[L][i]
            if len(px) and len(Yin[0][0]):
                a = self.rtree[L][i][0]
                E[(i, 0)] = (px, self.U[(L, i, 0)][X[px] - a])
        for l in range(L - 1, lc - 1, -1):
            new = {}
            for i, j in self.pairs(l):
                px, py = Xin[l][i], Yin[L - l][j]
                if not len(px) or not len(py):
                    continue
                R = self.U[(l, i, j)]
                r1 = self.rank_r(l + 1, 2 * i, j // 2)
                parts, pos = [], []
                e1 = E.get((2 * i, j // 2))
                e2 = E.get((2 * i + 1, j // 2))
                if e1 is not None:
                    parts.append(e1[1] @ R[:r1]); pos.append(e1[0])
                if e2 is not None:
                    parts.append(e2[1] @ R[r1:]); pos.append(e2[0])
                new[(i, j)] = (np.concatenate(pos), np.vstack(parts))
            E = new
        F = {}
        for j in range(1 << L):
            py = Yin[L][j]
            if len(py) and len(Xin[0][0]):
                a = self.ctree[L][j][0]
                F[(0, j)] = (py, self.V[(0, 0, j)][Y[py] - a].T)
        for l in range(1, lc + 1):
            new = {}
            for i, j in self.pairs(l):
                px, py = Xin[l][i], Yin[L - l][j]
                if not len(px) or not len(py):
                    continue
                W = self.V[(l, i, j)]
                c1 = self.rank_c(l - 1, i // 2, 2 * j)
                parts, pos = [], []
                f1 = F.get((i // 2, 2 * j))
                f2 = F.get((i // 2, 2 * j + 1))
                if f1 is not None:
                    parts.append(W[:c1].T @ f1[1]); pos.append(f1[0])
                if f2 is not None:
                    parts.append(W[c1:].T @ f2[1]); pos.append(f2[0])
                new[(i, j)] = (np.concatenate(pos), np.hstack(parts))
            F = new
        for (i, j), (px, Eb) in E.items():
            if (i, j) in F:
                py, Fb = F[(i, j)]
                out[np.ix_(px, py)] = Eb @ self.B[(i, j)] @ Fb
                FLOPS[0] += 8 * (Eb.size * Fb.shape[0] + Eb.shape[0] * Fb.size)
        return out


# ---------------------------------------------------------------------------
# Proxy selection (Sec. 3.1: alpha uniform samples + knn nearest neighbours)
# ---------------------------------------------------------------------------
def uniform_sample(a, b, cnt):
    """cnt indices of [a, b) drawn uniformly without replacement, reproducibly.

    Index c gets the 64-bit hash h(c) = splitmix64(salt ^ (c * 0x9E3779B97F4A7C15))
    with salt = (a << 32) | b; the cnt indices of smallest hash (ties by index)
    are returned in increasing order.  A stride pattern aliases with the
    lattice structure of the point sets, a hash ranking does not.
    """
    from workloads import splitmix64
    c = np.arange(a, b, dtype=np.uint64)
    salt = np.uint64(((a & 0xFFFFFFFF) << 32) | (b & 0xFFFFFFFF))
    with np.errstate(over="ignore"):
        h = splitmix64(salt ^ (c * np.uint64(0x9E3779B97F4A7C15)))
    order = np.lexsort((c, h))
    return np.sort(c[order[:cnt]].astype(np.int64))


class Proxies:
    """nn_r[x]: local column indices near local row x (distance order);
    nn_c[y]: local row indices near local column y."""

    def __init__(self, nn_r, nn_c, alpha, knn):
        self.nn_r, self.nn_c, self.alpha, self.knn = nn_r, nn_c, alpha, knn

    def _pick(self, nn, X, a, b):
        size = b - a
        if (self.alpha + self.knn) * len(X) >= size:
            return np.arange(a, b, dtype=np.int64)
        cnt = self.alpha * len(X)
        uni = uniform_sample(a, b, cnt)
        near = [c for x in X for c in nn[int(x)][:self.knn] if a <= c < b]
        return np.unique(np.concatenate([uni, np.asarray(near, np.int64)]))

    def cols(self, X, a, b):
        return self._pick(self.nn_r, X, a, b)

    def rows(self, Y, a, b):
        return self._pick(self.nn_c, Y, a, b)


def bf_entry_eval(extract, m, n, rtree, ctree, L, proxies: Proxies, tol, max_rank=0):
    """Alg. 2: butterfly construction from entry extraction (L + 2 extract calls)."""
    bf = Butterfly(m, n, rtree, ctree, L)
    lc = bf.lc
    for l in range(L, lc - 1, -1):                       # left to middle
        lst, keys = [], []
        for i, j in bf.pairs(l):
            if l == L:
                a, b = bf.rtree[L][i]
                X = np.arange(a, b, dtype=np.int64)
            else:
                X = _cat(bf.Osk[(l + 1, 2 * i, j // 2)], bf.Osk[(l + 1, 2 * i + 1, j // 2)])
            ca, cb = bf.ctree[L - l][j]
            lst.append((X, proxies.cols(X, ca, cb)))
            keys.append((i, j))
        blocks = extract(lst)
        for (i, j), (X, _), K in zip(keys, lst, blocks):
            U, sk = row_id(K, tol, max_rank)
            bf.U[(l, i, j)] = U
            bf.Osk[(l, i, j)] = X[sk]
    for l in range(0, lc + 1):                           # right to middle
        lst, keys = [], []
        for i, j in bf.pairs(l):
            if l == 0:
                a, b = bf.ctree[L][j]
                Y = np.arange(a, b, dtype=np.int64)
            else:
                Y = _cat(bf.Ssk[(l - 1, i // 2, 2 * j)], bf.Ssk[(l - 1, i // 2, 2 * j + 1)])
            ra, rb = bf.rtree[l][i]
            lst.append((proxies.rows(Y, ra, rb), Y))
            keys.append((i, j))
        blocks = extract(lst)
        for (i, j), (_, Y), K in zip(keys, lst, blocks):
            V, sk = row_id(K.T, tol, max_rank)           # column ID
            bf.V[(l, i, j)] = V
            bf.Ssk[(l, i, j)] = Y[sk]
    keys = list(bf.pairs(lc))                            # centre
    blocks = extract([(bf.Osk[(lc, i, j)], bf.Ssk[(lc, i, j)]) for i, j in keys])
    for (i, j), K in zip(keys, blocks):
        bf.B[(i, j)] = K
    return bf


# ---------------------------------------------------------------------------
# Randomized construction from products (Sec. 3.2)
# ---------------------------------------------------------------------------
class Operator:
    """A black-box m x n operator with apply(X) = K X and applyT(X) = K^T X."""

    def __init__(self, m, n, apply, applyT):
        self.m, self.n, self.apply, self.applyT = m, n, apply, applyT


def _sketch(size_rows, groups, q, key, level, side):
    """Block-sparse random matrix: group g supported on rows [a,b) with q columns.

    Groups no wider than q get the identity on their rows (exact sampling).
    Returns (Omega, colranges)."""
    cols = []
    total = 0
    for a, b in groups:
        w = (b - a) if (b - a) <= q else q
        cols.append((total, total + w))
        total += w
    Om = np.zeros((size_rows, total), np.complex128)
    for g, ((a, b), (c0, c1)) in enumerate(zip(groups, cols)):
        if c1 - c0 == b - a:
            Om[a:b, c0:c1] = np.eye(b - a)
        else:
            stream = (key * 1000003 + level * 7919 + side * 104729 + g) & 0xFFFFFF
            rows = np.arange(a, b, dtype=np.int64)
            for c in range(c1 - c0):
                Om[a:b, c0 + c] = counter_normal_complex(stream, rows, c)
    return Om, cols


def bf_random_matvec(op: Operator, rtree, ctree, L, tol, max_rank=0, key=1, p=8, q_start=64):
    """Butterfly construction from products with K and K^T (Sec. 3.2).

    Reading (the paper defers the algorithm to [liu2020butterfly]): Alg. 2 with
    random mixtures in place of proxy rows/columns.
      left half, l = L..l_c: Y = K Omega with Omega block-sparse, one group of q
        Gaussian columns per nu at level L-l of T_S supported on S_nu; row ID of
        Y(X, cols(nu)) with X = O_tau (l = L) or the children's skeletons.
      right half, l = 0..l_c: Z = K^T Psi, groups per tau at level l of T_O;
        row ID of Z(Y, cols(tau)) gives the column ID of K(O_tau, Y).
      centre: B_{tau,nu} solves B (V_{tau,nu}^T Omega_nu) = Y(Obar_{tau,nu}, cols(nu))
        in the least-squares sense, on the level-l_c sketches.
    q = max_rank + p columns per group (q_start + p without a cap); without a
    cap a level is redone with doubled q when an ID uses more than q - p columns.
    """
    m, n = op.m, op.n
    bf = Butterfly(m, n, rtree, ctree, L)
    lc = bf.lc
    q0 = (max_rank if max_rank > 0 else q_start) + p
    centre = None
    for l in range(L, lc - 1, -1):
        groups = bf.ctree[L - l]
        q = q0
        while True:
            Om, cols = _sketch(n, groups, q, key, l, 0)
            Y = op.apply(Om)
            res, grow = {}, False
            for i, j in bf.pairs(l):
                if l == L:
                    a, b = bf.rtree[L][i]
                    X = np.arange(a, b, dtype=np.int64)
                else:
                    X = _cat(bf.Osk[(l + 1, 2 * i, j // 2)], bf.Osk[(l + 1, 2 * i + 1, j // 2)])
                c0, c1 = cols[j]
                U, sk = row_id(Y[X, c0:c1], tol, max_rank)
                res[(i, j)] = (U, X[sk])
                ga, gb = groups[j]
                if max_rank <= 0 and (c1 - c0) < (gb - ga) and len(sk) > (c1 - c0) - p:
                    grow = True
            if grow:
                q *= 2
                continue
            break
        for (i, j), (U, sk) in res.items():
            bf.U[(l, i, j)] = U
            bf.Osk[(l, i, j)] = sk
        if l == lc:
            centre = (Om, Y, cols)
    for l in range(0, lc + 1):
        groups = bf.rtree[l]
        q = q0
        while True:
            Ps, cols = _sketch(m, groups, q, key, l, 1)
            Z = op.applyT(Ps)
            res, grow = {}, False
            for i, j in bf.pairs(l):
                if l == 0:
                    a, b = bf.ctree[L][j]
                    Yc = np.arange(a, b, dtype=np.int64)
                else:
                    Yc = _cat(bf.Ssk[(l - 1, i // 2, 2 * j)], bf.Ssk[(l - 1, i // 2, 2 * j + 1)])
                c0, c1 = cols[i]
                V, sk = row_id(Z[Yc, c0:c1], tol, max_rank)
                res[(i, j)] = (V, Yc[sk])
                ga, gb = groups[i]
                if max_rank <= 0 and (c1 - c0) < (gb - ga) and len(sk) > (c1 - c0) - p:
                    grow = True
            if grow:
                q *= 2
                continue
            break
        for (i, j), (V, sk) in res.items():
            bf.V[(l, i, j)] = V
            bf.Ssk[(l, i, j)] = sk
    Om, Y, cols = centre
    T = bf.right_transform(Om)
    for i, j in bf.pairs(lc):
        c0, c1 = cols[j]
        Tij = T[(i, j)][:, c0:c1]                 # c x q
        Yr = Y[bf.Osk[(lc, i, j)], c0:c1]          # r x q
        r, c = Yr.shape[0], Tij.shape[0]
        if r == 0 or c == 0:
            bf.B[(i, j)] = np.zeros((r, c), np.complex128)
        else:
            sol, *_ = np.linalg.lstsq(Tij.T, Yr.T, rcond=None)
            bf.B[(i, j)] = sol.T
            FLOPS[0] += 8 * c * c * (c1 - c0) + 8 * r * c * (c1 - c0)
    return bf


# ---------------------------------------------------------------------------
# Split of an L-level butterfly into four (L-2)-level children (Alg. 4, BF_SMW)
# ---------------------------------------------------------------------------
def bf_split(bf: Butterfly):
    """Children K(O_a, S_b), a, b in {0, 1} (level-1 nodes), each with L-2 levels.

    The child's factors are the parent's factors of levels 1..L-1 restricted to
    the quadrant; the child's outermost U (V) is the product of the parent's
    level-L U (level-0 V) with the level-(L-1) R (level-1 W).
    """
    L, lc = bf.L, bf.lc
    assert L >= 2
    Lp = L - 2
    kids = {}
    for a in range(2):
        for b in range(2):
            ra0 = bf.rtree[1][a][0]
            cb0 = bf.ctree[1][b][0]
            rt = subtree(bf.rtree, 1, a, Lp)
            ct = subtree(bf.ctree, 1, b, Lp)
            ch = Butterfly(rt[0][0][1], ct[0][0][1], rt, ct, Lp)
            for lp in range(ch.lc, Lp + 1):             # left half
                l = lp + 1
                for ip, jp in ch.pairs(lp):
                    i = a * (1 << lp) + ip
                    j = b * (1 << (Lp - lp)) + jp
                    R = bf.U[(l, i, j)]
                    if l == L - 1:
                        r1 = bf.rank_r(L, 2 * i, 0)
                        U1, U2 = bf.U[(L, 2 * i, 0)], bf.U[(L, 2 * i + 1, 0)]
                        R = np.vstack([U1 @ R[:r1], U2 @ R[r1:]])
                    ch.U[(lp, ip, jp)] = R
                    ch.Osk[(lp, ip, jp)] = bf.Osk[(l, i, j)] - ra0
            for lp in range(0, ch.lc + 1):               # right half
                l = lp + 1
                for ip, jp in ch.pairs(lp):
                    i = a * (1 << lp) + ip
                    j = b * (1 << (Lp - lp)) + jp
                    W = bf.V[(l, i, j)]
                    if l == 1:
                        c1 = bf.rank_c(0, 0, 2 * j)
                        V1, V2 = bf.V[(0, 0, 2 * j)], bf.V[(0, 0, 2 * j + 1)]
                        W = np.vstack([V1 @ W[:c1], V2 @ W[c1:]])
                    ch.V[(lp, ip, jp)] = W
                    ch.Ssk[(lp, ip, jp)] = bf.Ssk[(l, i, j)] - cb0
            for ip, jp in ch.pairs(ch.lc):
                i = a * (1 << ch.lc) + ip
                j = b * (1 << (Lp - ch.lc)) + jp
                ch.B[(ip, jp)] = bf.B[(i, j)]
            kids[(a, b)] = ch
    return kids
