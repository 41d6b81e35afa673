"""Pins of the oracle's numerical kernels against mathematics it does not share:
dense LU (scipy/LAPACK), SVD bounds, exact low rank, dense expansions, the
Woodbury identity, closed forms of the Green's function."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as w
from oracle.analysis import analyze, cluster_tree_geometric
from oracle import dense_mf as dm
from oracle.idq import row_id, col_id
from oracle.butterfly import (Butterfly, Operator, Proxies, bf_entry_eval, bf_random_matvec,
                              bf_split, extend_tree)
from oracle.hodbf import hodbf_entry_eval, hodbf_invert, bf_smw


# ---------------- exact multifrontal (Alg. 1) ----------------
@pytest.mark.parametrize("gen", [lambda: w.helmholtz7(4, 8), lambda: w.helmholtz7(6, 8),
                                 lambda: w.helmholtz7(8, 8), lambda: w.yee_maxwell(4, 10)])
def test_exact_multifrontal_equals_dense_lu(gen):
    p = gen()
    an = analyze(p, 16, 10 ** 9)
    fac, _ = dm.multifrontal_factor(p, an)
    b = w.rhs_gaussian(p, 2, 3)
    x = dm.solve(p, an, fac, b)
    xr = sla.lu_solve(sla.lu_factor(p.to_scipy().toarray()), b)
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-12


def test_exact_multifrontal_16cube_residual_and_flops():
    p = w.helmholtz7(16, 8)
    an = analyze(p, 64, 10 ** 9)
    fac, flops = dm.multifrontal_factor(p, an)
    b = w.rhs_point_plus_gaussian(p)
    x = dm.solve(p, an, fac, b)
    assert np.linalg.norm(p.to_scipy() @ x - b) / np.linalg.norm(b) < 1e-12
    assert abs(flops - 7.33e8) / 7.33e8 < 0.01


def test_partial_pivot_rule():
    M = np.array([[1, 2], [3j, 1], [-3, 0]], complex)[:2, :2]
    LU, piv = dm.lu_partial_pivot(M)
    assert list(piv) == [1, 1]                 # |3i| > |1|
    M2 = np.array([[2, 1], [-2, 5]], complex)  # tie -> lowest row
    _, piv2 = dm.lu_partial_pivot(M2)
    assert piv2[0] == 0


# ---------------- ID (Sec. 3) ----------------
def test_row_id_exact_rank_and_identity_rows():
    rng = np.random.default_rng(0)
    A = (rng.standard_normal((60, 9)) + 1j * rng.standard_normal((60, 9))) @ \
        (rng.standard_normal((9, 45)) + 1j * rng.standard_normal((9, 45)))
    U, sk = row_id(A, 1e-12)
    assert len(sk) == 9
    assert np.array_equal(U[sk], np.eye(9))
    assert np.linalg.norm(A - U @ A[sk]) / np.linalg.norm(A) < 1e-12
    V, sc = col_id(A, 1e-12)
    assert len(sc) == 9 and np.linalg.norm(A - A[:, sc] @ V.T) / np.linalg.norm(A) < 1e-12


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-6])
def test_row_id_error_vs_svd_bound(tol):
    rng = np.random.default_rng(1)
    Q1, _ = np.linalg.qr(rng.standard_normal((70, 70)) + 1j * rng.standard_normal((70, 70)))
    Q2, _ = np.linalg.qr(rng.standard_normal((50, 50)) + 1j * rng.standard_normal((50, 50)))
    s = 10.0 ** (-np.arange(50) / 5)
    M = (Q1[:, :50] * s) @ Q2
    U, sk = row_id(M, tol)
    k = len(sk)
    err = np.linalg.norm(M - U @ M[sk], 2)
    assert err <= 10 * tol * s[0]
    assert s[k] <= tol * s[0] * 10          # rank not larger than needed by more than the QR gap
    assert s[k - 1] >= tol * s[0] / 10       # and not too small


# ---------------- butterfly (Sec. 3) ----------------
def _green_block(m, sep):
    P, Q, k = w.green_planes(m, 1.0, math.pi / 4)
    Q = Q.copy(); Q[:, 2] = sep
    order, tree = cluster_tree_geometric(P.astype(np.int64), 16)
    P, Q = P[order], Q[order]
    K = w.green_entries(P, Q, k, np.arange(m * m), np.arange(m * m))
    d2 = ((P[:, None, :2] - Q[None, :, :2]) ** 2).sum(-1)
    nn = [list(np.lexsort((np.arange(m * m), d2[i]))[:8]) for i in range(m * m)]
    return K, tree, nn


@pytest.fixture(scope="module")
def green16():
    return _green_block(16, 3.0)


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-6])
def test_bf_entry_eval_green_function(green16, tol):
    K, tree, nn = green16
    L = len(tree) - 1
    ext = lambda lst: [K[np.ix_(X, Y)] for X, Y in lst]
    bf = bf_entry_eval(ext, K.shape[0], K.shape[1], tree, tree, L, Proxies(nn, nn, 2, 8), tol)
    err = np.linalg.norm(bf.dense() - K) / np.linalg.norm(K)
    assert err <= 10 * tol


def test_bf_extract_and_transpose_match_dense(green16):
    K, tree, nn = green16
    L = len(tree) - 1
    ext = lambda lst: [K[np.ix_(X, Y)] for X, Y in lst]
    bf = bf_entry_eval(ext, K.shape[0], K.shape[1], tree, tree, L, Proxies(nn, nn, 2, 8), 1e-4)
    D = bf.dense()
    rng = np.random.default_rng(4)
    lst = [(rng.choice(256, 20, replace=False), rng.choice(256, 31, replace=False)),
           (np.arange(3), np.arange(200, 256)), (np.array([7]), np.array([9]))]
    for (X, Y), E in zip(lst, bf.extract(lst)):
        assert np.abs(E - D[np.ix_(X, Y)]).max() <= 1e-13 * np.abs(D).max()
    x = rng.standard_normal((256, 3)) + 0j
    assert np.abs(bf.applyT(x) - D.T @ x).max() <= 1e-13 * np.abs(D.T @ x).max()


def test_bf_random_matvec_reconstructs(green16):
    K, tree, _ = green16
    L = len(tree) - 1
    op = Operator(256, 256, lambda X: K @ X, lambda X: K.T @ X)
    for tol in (1e-4, 1e-6):
        bf = bf_random_matvec(op, tree, tree, L, tol, key=3)
        assert np.linalg.norm(bf.dense() - K) / np.linalg.norm(K) <= 10 * tol


def test_bf_level0_is_a_low_rank_id():
    rng = np.random.default_rng(5)
    A = (rng.standard_normal((40, 6)) + 0j) @ (rng.standard_normal((6, 30)) + 0j)
    ext = lambda lst: [A[np.ix_(X, Y)] for X, Y in lst]
    nn = [[] for _ in range(40)]
    bf = bf_entry_eval(ext, 40, 30, [[(0, 40)]], [[(0, 30)]], 0, Proxies(nn, nn, 100, 0), 1e-12)
    assert bf.B[(0, 0)].shape == (6, 6)
    assert np.linalg.norm(bf.dense() - A) / np.linalg.norm(A) < 1e-12


def test_bf_split_children_equal_quadrants(green16):
    K, tree, nn = green16
    L = len(tree) - 1
    ext = lambda lst: [K[np.ix_(X, Y)] for X, Y in lst]
    bf = bf_entry_eval(ext, 256, 256, tree, tree, L, Proxies(nn, nn, 2, 8), 1e-4)
    D = bf.dense()
    for (a, b), ch in bf_split(bf).items():
        ra, cb = bf.rtree[1][a], bf.ctree[1][b]
        assert ch.L == L - 2
        assert np.abs(ch.dense() - D[ra[0]:ra[1], cb[0]:cb[1]]).max() <= 1e-13 * np.abs(D).max()


def test_bf_storage_n_log_n():
    # Sec. 3.1: the butterfly stores O(n log n) entries at bounded rank.  With a
    # fixed number of wavelengths across the planes the rank stays bounded and the
    # stored entries stay within (L + 2) * n * r_max while the dense block grows as n^2.
    ratios = []
    for m in (16, 24, 32):
        P, Q, k = w.green_planes(m, 1.0, math.pi / 4 * 16 / m)
        Q = Q.copy(); Q[:, 2] = 3.0 * m / 16
        order, tree = cluster_tree_geometric(P.astype(np.int64), 16)
        P, Q = P[order], Q[order]
        K = w.green_entries(P, Q, k, np.arange(m * m), np.arange(m * m))
        d2 = ((P[:, None, :2] - Q[None, :, :2]) ** 2).sum(-1)
        nn = [list(np.lexsort((np.arange(m * m), d2[i]))[:8]) for i in range(m * m)]
        L = len(tree) - 1
        ext = lambda lst, K=K: [K[np.ix_(X, Y)] for X, Y in lst]
        bf = bf_entry_eval(ext, m * m, m * m, tree, tree, L, Proxies(nn, nn, 2, 8), 1e-3)
        n = m * m
        r = bf.max_rank()
        assert bf.storage() <= (L + 2) * n * r * max(1.0, 2.0 * r / 16)
        assert np.linalg.norm(bf.dense() - K) / np.linalg.norm(K) <= 1e-2
        ratios.append(bf.storage() / n ** 2)
    assert ratios[0] > ratios[1] > ratios[2]


# ---------------- SMW / HOD-BF (Sec. 4, Alg. 4) ----------------
def test_smw_level0_is_woodbury():
    rng = np.random.default_rng(6)
    n, r = 40, 5
    A = 0.1 * (rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r))) @ \
        (rng.standard_normal((r, n)) + 1j * rng.standard_normal((r, n)))
    ext = lambda lst: [A[np.ix_(X, Y)] for X, Y in lst]
    nn = [[] for _ in range(n)]
    bf = bf_entry_eval(ext, n, n, [[(0, n)]], [[(0, n)]], 0, Proxies(nn, nn, 100, 0), 1e-13)
    inv = bf_smw(bf, 1e-12, 0, 1)
    ref = np.linalg.inv(np.eye(n) + A) - np.eye(n)
    assert np.abs(inv.dense() - ref).max() < 1e-11


def _front_matrix(n=12, nmin=100, leaf=16):
    """Dense root-separator Schur complement of a small Helmholtz problem (a real F11)."""
    p = w.helmholtz7(n, 8)
    an = analyze(p, 32, nmin, leaf)
    Ap = dm.permuted_matrix(p, an)
    root = an.fronts[-1]
    fac_cb = {}
    for f in an.fronts:
        F = dm.assemble_sparse(Ap, f)
        for c in f.children:
            rel = dm.relative_map(an.fronts[c], f)
            F[np.ix_(rel, rel)] += fac_cb.pop(c)
        if f is root:
            return F, root, an
        _, C = dm.factor_front_dense(F, f.s)
        fac_cb[f.id] = C


def test_hodbf_construct_and_invert():
    F, root, an = _front_matrix()
    s = root.s
    from oracle.analysis import front_neighbours
    nn = front_neighbours(an, root, 8)["nn11"]
    nnl = [[g - root.sep_begin for g in nn[root.sep_begin + x]] for x in range(s)]
    ext = lambda lst: [F[np.ix_(X, Y)] for X, Y in lst]
    for tol in (1e-4, 1e-7):
        H = hodbf_entry_eval(ext, s, root.th_tree, nnl, 2, 8, tol)
        assert np.linalg.norm(H.dense() - F) / np.linalg.norm(F) <= 10 * tol
        inv = hodbf_invert(H, tol, 0, key=3)
        x = np.random.default_rng(2).standard_normal((s, 4)) + 0j
        # ||x - A (A^-1 x)|| relative, against the compressed A; and against dense inverse
        y = inv.apply(x)
        cond = np.linalg.cond(F)
        assert np.linalg.norm(H.apply(y) - x) / np.linalg.norm(x) <= 10 * tol * cond
        assert np.linalg.norm(y - np.linalg.solve(F, x)) / np.linalg.norm(np.linalg.solve(F, x)) <= 10 * tol * cond
        xt = inv.applyT(x)
        assert np.linalg.norm(H.applyT(xt) - x) / np.linalg.norm(x) <= 10 * tol * cond


def test_oracle_per_front_compression_error_16cube():
    # Sec. 6.1 / Alg. 5: every compressed front of the 16^3 workload (tol 1e-6) against the same
    # blocks of the exact elimination in the same ordering (dense assembly, Alg. 1)
    from oracle import compressed_mf as cm
    p = w.helmholtz7(16, 8)
    an = analyze(p, 64, 128, 64)
    fac, st = cm.compressed_factor(p, an, 1e-6)
    Ap = dm.permuted_matrix(p, an)
    cbs, seen = {}, 0
    for f in an.fronts:
        F = dm.assemble_sparse(Ap, f)
        for c in f.children:
            rel = dm.relative_map(an.fronts[c], f)
            F[np.ix_(rel, rel)] += cbs.pop(c)
        s = f.s
        C = F[s:, s:] - F[s:, :s] @ np.linalg.solve(F[:s, :s], F[:s, s:]) if f.u else None
        if f.compressed:
            seen += 1
            fc = fac[f.id]
            rel_err = lambda A, B: np.linalg.norm(A - B) / np.linalg.norm(B)
            assert rel_err(fc.F11.dense(), F[:s, :s]) <= 1e-5
            if f.u:
                assert rel_err(fc.F12.dense(), F[:s, s:]) <= 1e-5
                assert rel_err(fc.F21.dense(), F[s:, :s]) <= 1e-5
                assert rel_err(fc.C.dense(), C) <= 1e-5
        if f.parent >= 0:
            cbs[f.id] = C
    assert seen == 2
