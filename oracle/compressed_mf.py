"""Oracle: rank-structured multifrontal factorization with HOD-BF fronts (Alg. 5).

Test infrastructure only (see oracle/analysis.py).

For every front in topological order (Alg. 5):
  * separator smaller than nmin_sep: dense front, Alg. 1 (dense_mf.py);
  * otherwise (Sec. 5, steps after Eq. (5.1); the large-front branch of Alg. 5):
      F11   <- HODBF_entry_eval(A(Is,Is) (+) C_nu1 (+) C_nu2)
      F11^-1<- HODBF_invert(F11)                                   (Alg. 4)
      F12   <- BF_entry_eval(A(Is,Iu) (+) C_nu1 (+) C_nu2)          (Alg. 2)
      F21   <- BF_entry_eval(A(Iu,Is) (+) C_nu1 (+) C_nu2)
      S     <- BF_random_matvec(F21 F11^-1 F12)                    (Sec. 3.2)
      C_tau <- HODBF_entry_eval(C_nu1 (+) C_nu2 - S)
    Entries are extracted by splitting each requested block into an A-list
    and one list per child contribution block (Sec. 5, step 1), dense
    children by gathering, compressed children by extract_HODBF.
  * F12 uses T_H as T_O and the F22 tree as T_S (F21 the reverse); the deeper
    tree is truncated so both have the same number of levels (Sec. 5).
Solve (Sec. 5 last paragraph; block-LU reading): forward w = F11^-1 b_s,
b_u -= F21 w; backward x_s = w - F11^-1 (F12 x_u).
Preconditioned GMRES(30) is in gmres.py.
"""
from __future__ import annotations

import numpy as np

from . import dense_mf as dm
from .analysis import front_neighbours
from .butterfly import Operator, Proxies, bf_entry_eval, bf_random_matvec
from .hodbf import hodbf_entry_eval, hodbf_invert, HODBF
from .idq import FLOPS


class CompressedFront:
    def __init__(self, s, u, F11, F11inv, F12, F21, C):
        self.s, self.u = s, u
        self.F11, self.F11inv, self.F12, self.F21 = F11, F11inv, F12, F21
        self.C = C


class DenseCB:
    """A dense contribution block with index positions in the parent front."""

    def __init__(self, C):
        self.C = C

    def extract(self, lst):
        return [self.C[np.ix_(X, Y)] for X, Y in lst]

    def dense(self):
        return self.C


class FrontExtractor:
    """extract(lst) over front-local indices of F_tau = A-part (+) children (- S)."""

    def __init__(self, Ap, f, kids, with_A=True, S=None):
        self.f = f
        self.gidx = dm.front_index(f)
        self.s = f.s
        self.Ap = Ap if with_A else None
        self.kids = []
        n = len(self.gidx)
        for child, cb in kids:
            rel = dm.relative_map(child, f)
            inv = np.full(n, -1, np.int64)
            inv[rel] = np.arange(len(rel))
            self.kids.append((inv, cb))
        self.S = S

    def __call__(self, lst):
        out = []
        for X, Y in lst:
            X = np.asarray(X, np.int64); Y = np.asarray(Y, np.int64)
            blk = np.zeros((len(X), len(Y)), np.complex128)
            if len(X) and len(Y):
                if self.Ap is not None:
                    sub = self.Ap[self.gidx[X]][:, self.gidx[Y]].toarray()
                    mask = (X[:, None] < self.s) | (Y[None, :] < self.s)
                    blk += np.where(mask, sub, 0)
                for inv, cb in self.kids:
                    cx, cy = inv[X], inv[Y]
                    px = np.nonzero(cx >= 0)[0]
                    py = np.nonzero(cy >= 0)[0]
                    if len(px) and len(py):
                        blk[np.ix_(px, py)] += cb.extract([(cx[px], cy[py])])[0]
                if self.S is not None:
                    blk -= self.S.extract([(X - self.s, Y - self.s)])[0]
            out.append(blk)
        return out


def _nn_local(nn, base_glob, loc_of):
    """Map a dict of global neighbour lists to local index lists."""
    return nn


def compressed_factor(prob, an, tol, alpha=2, knn=8, max_rank=0, key=11):
    Ap = dm.permuted_matrix(prob, an)
    factors = [None] * len(an.fronts)
    cbs = {}
    stats = dict(compressed=0, dense=0, max_rank=0, flops_dense=0.0)
    FLOPS[0] = 0
    for f in an.fronts:
        kids = [(an.fronts[c], cbs.pop(c)) for c in f.children]
        s, u = f.s, f.u
        if not f.compressed:
            F = dm.assemble_sparse(Ap, f)
            for child, cb in kids:
                rel = dm.relative_map(child, f)
                F[np.ix_(rel, rel)] += cb.dense()
            fac, C = dm.factor_front_dense(F, s)
            factors[f.id] = fac
            stats["dense"] += 1
            stats["flops_dense"] += 8 * (s ** 3 / 3 + s * s * u + s * u * u)
            if f.parent >= 0:
                cbs[f.id] = DenseCB(C)
            continue
        stats["compressed"] += 1
        nn = front_neighbours(an, f, knn)
        ext = FrontExtractor(Ap, f, kids)
        # front-local neighbour lists: I^s -> [0,s), I^u -> s + position
        loc = {int(g): i for i, g in enumerate(dm.front_index(f))}
        def local(d):
            return {loc[g]: [loc[h] for h in lst] for g, lst in d.items()}
        nn11 = local(nn["nn11"]); nn22 = local(nn["nn22"])
        nn12 = local(nn["nn12"]); nn21 = local(nn["nn21"])
        n11 = [nn11.get(x, []) for x in range(s)]
        F11 = hodbf_entry_eval(lambda lst: ext(lst), s, f.th_tree, n11, alpha, knn, tol, max_rank)
        F11inv = hodbf_invert(F11, tol, max_rank, key=(key * 7 + f.id) & 0xFFFFF)
        F12 = F21 = C = None
        if u:
            LH = len(f.th_tree) - 1
            L22 = len(f.f22_tree) - 1
            L = min(LH, L22)
            t22 = f.f22_tree
            # F12: rows I^s (tree T_H), columns I^u (F22 tree)
            nr = [[c - s for c in nn12.get(x, [])] for x in range(s)]
            nc = [[r for r in nn21.get(s + y, [])] for y in range(u)]
            ext12 = lambda lst: ext([(X, Y + s) for X, Y in lst])
            F12 = bf_entry_eval(ext12, s, u, f.th_tree, t22, L, Proxies(nr, nc, alpha, knn), tol, max_rank)
            ext21 = lambda lst: ext([(X + s, Y) for X, Y in lst])
            F21 = bf_entry_eval(ext21, u, s, t22, f.th_tree, L, Proxies(nc, nr, alpha, knn), tol, max_rank)
            op = Operator(u, u,
                          lambda x: F21.apply(F11inv.apply(F12.apply(x))),
                          lambda x: F12.applyT(F11inv.applyT(F21.applyT(x))))
            S = bf_random_matvec(op, t22, t22, L22, tol, max_rank, key=(key * 13 + f.id) & 0xFFFFF)
            n22 = [[c - s for c in nn22.get(s + x, [])] for x in range(u)]
            extC = FrontExtractor(Ap, f, kids, with_A=False, S=S)
            Cext = lambda lst: extC([(X + s, Y + s) for X, Y in lst])
            C = hodbf_entry_eval(Cext, u, t22, n22, alpha, knn, tol, max_rank)
            stats["max_rank"] = max(stats["max_rank"], F12.max_rank(), F21.max_rank(), S.max_rank(), C.max_rank())
            if f.parent >= 0:
                cbs[f.id] = C
        stats["max_rank"] = max(stats["max_rank"], F11.max_rank())
        factors[f.id] = CompressedFront(s, u, F11, F11inv, F12, F21, C)
    stats["flops"] = FLOPS[0] + stats["flops_dense"]
    return factors, stats


def compressed_solve_permuted(an, factors, b):
    """Preconditioner application M^-1 b (new numbering)."""
    x = np.array(b, dtype=np.complex128, copy=True)
    if x.ndim == 1:
        x = x[:, None]
    for f in an.fronts:
        fac = factors[f.id]
        sl = slice(f.sep_begin, f.sep_end)
        if isinstance(fac, CompressedFront):
            w = fac.F11inv.apply(x[sl])
            x[sl] = w
            if f.u:
                x[f.upd] -= fac.F21.apply(w)
        else:
            z = dm.lower_solve_unit(fac.LU, dm.apply_row_swaps(x[sl], fac.piv))
            x[sl] = z
            if f.u:
                x[f.upd] -= fac.F21 @ z
    for f in reversed(an.fronts):
        fac = factors[f.id]
        sl = slice(f.sep_begin, f.sep_end)
        if isinstance(fac, CompressedFront):
            if f.u:
                x[sl] = x[sl] - fac.F11inv.apply(fac.F12.apply(x[f.upd]))
        else:
            rhs = x[sl]
            if f.u:
                rhs = rhs - fac.F12 @ x[f.upd]
            x[sl] = dm.upper_solve(fac.LU, rhs)
    return x


def preconditioner(an, factors):
    """v (original numbering) -> M^-1 v (original numbering)."""
    def apply(v):
        v = np.asarray(v)
        vv = v[:, None] if v.ndim == 1 else v
        xp = compressed_solve_permuted(an, factors, vv[an.perm])
        x = np.empty_like(xp)
        x[an.perm] = xp
        return x[:, 0] if v.ndim == 1 else x
    return apply
