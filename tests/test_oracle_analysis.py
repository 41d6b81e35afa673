"""Pins of the oracle's symbolic analysis (Sec. 2, Sec. 5.1, Sec. 5.2)."""
import os

import numpy as np
import pytest

import workloads as w
from oracle.analysis import analyze, bfs_nearest, cluster_tree_geometric, cluster_tree_balanced, \
    front_neighbours, levels_of_fronts

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid2d(n):
    """n x n x 1 node lattice with the 5-point pattern (for Fig. 5)."""
    import scipy.sparse as sp
    idx = np.arange(n * n)
    i, j = idx % n, idx // n
    rows, cols = [idx], [idx]
    for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        ok = (i + di >= 0) & (i + di < n) & (j + dj >= 0) & (j + dj < n)
        rows.append(idx[ok]); cols.append(idx[ok] + di + n * dj)
    r = np.concatenate(rows); c = np.concatenate(cols)
    A = sp.csr_matrix((np.ones(len(r), complex), (r, c)), shape=(n * n, n * n))
    A.sort_indices()
    coords = np.stack([i, j, np.zeros_like(i)], 1).astype(np.int32)
    return w.SparseProblem("grid2d", n * n, A.indptr.astype(np.int64), A.indices.astype(np.int32),
                           A.data, coords, w.LATTICE_NODE)


def test_nested_dissection_matches_fig5_example():
    p = _grid2d(11)
    an = analyze(p, leaf_size=8, nmin_sep=10 ** 9)
    spec = {}
    for line in open(os.path.join(GOLDEN, "nd_11x11_fig5.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, xl, xh, yl, yh = line.split()
        spec[name] = (int(xl), int(xh), int(yl), int(yh))
    def box(f):
        c = p.coords[an.perm[f.sep_begin:f.sep_end]]
        return (c[:, 0].min(), c[:, 0].max(), c[:, 1].min(), c[:, 1].max()), len(c)
    root = an.fronts[-1]
    assert box(root) == (spec["S0"], 11)
    kids = [an.fronts[c] for c in root.children]
    assert [box(k)[0] for k in kids] == [spec["S1_0"], spec["S1_1"]]
    g = [box(an.fronts[c])[0] for k in kids for c in k.children]
    assert g == [spec["S2_00"], spec["S2_01"], spec["S2_10"], spec["S2_11"]]


@pytest.mark.parametrize("gen", [lambda: w.helmholtz7(12, 8), lambda: w.yee_maxwell(6, 10)])
def test_structure_invariants(gen):
    p = gen()
    an = analyze(p, leaf_size=16, nmin_sep=40, hodbf_leaf=8)
    N = p.n
    assert np.array_equal(np.sort(an.perm), np.arange(N))
    assert sum(f.s for f in an.fronts) == N
    A = p.to_scipy()[an.perm][:, an.perm].tocoo()
    owner = np.empty(N, np.int64)
    for f in an.fronts:
        owner[f.sep_begin:f.sep_end] = f.id
    anc = {}
    for f in an.fronts:
        a, q = set(), f.id
        while q >= 0:
            a.add(q); q = an.fronts[q].parent
        anc[f.id] = a
    # no entry of A couples two fronts neither of which is an ancestor of the other
    for r, c in zip(A.row, A.col):
        fr, fc = owner[r], owner[c]
        assert fr in anc[fc] or fc in anc[fr]
    for f in an.fronts:
        ok = set(range(f.sep_begin, f.sep_end)) | set(f.upd.tolist())
        for c in f.children:
            assert set(an.fronts[c].upd.tolist()) <= ok
        if f.compressed:
            assert len(f.th_tree[-1]) == 2 ** (len(f.th_tree) - 1)
            assert max(b - a for a, b in f.th_tree[-1]) <= 8


def test_symbolic_equals_bruteforce_elimination():
    """Fill pattern of L+U from a dense symbolic elimination == the fronts' structure."""
    for p in (w.helmholtz7(6, 8), w.yee_maxwell(4, 10)):
        an = analyze(p, leaf_size=10, nmin_sep=10 ** 9)
        N = p.n
        P = (p.to_scipy()[an.perm][:, an.perm].toarray() != 0)
        S = P.copy()
        for k in range(N):                      # symbolic Gaussian elimination
            rows = np.nonzero(S[k + 1:, k])[0] + k + 1
            cols = np.nonzero(S[k, k + 1:])[0] + k + 1
            S[np.ix_(rows, cols)] = True
        for f in an.fronts:
            idx = list(range(f.sep_begin, f.sep_end))
            below = set()
            for k in idx:
                below |= set((np.nonzero(S[k + 1:, k])[0] + k + 1).tolist())
            assert below - set(idx) == set(f.upd.tolist())


def test_16cube_front_shapes_by_hand():
    # planar nested dissection of the 16^3 grid (reading A11): the root separator is the plane
    # x = 8 (16 x 16 = 256 unknowns, no update set); its children split x in [0, 8) and [9, 16),
    # whose separators are planes of 16 x 8 = 128 and 16 x 7 = 112 unknowns, each updating the
    # whole root plane (256)
    an = analyze(w.helmholtz7(16, 8), 64, 128, 64)
    assert len(an.fronts) == 101 and len(levels_of_fronts(an)) == 7
    assert an.fronts[-1].s == 256 and an.fronts[-1].u == 0
    assert sorted((an.fronts[c].s, an.fronts[c].u) for c in an.fronts[-1].children) == [(112, 256), (128, 256)]
    assert sum(f.compressed for f in an.fronts) == 2


def test_cluster_trees():
    order, lv = cluster_tree_geometric(np.array([[x, y, 0] for y in range(8) for x in range(16)]), 16)
    assert len(lv) == 4 and all(b - a == 16 for a, b in lv[-1])
    # first cut is at x = 8 (largest extent), every leaf is a 4 x 4 square
    assert sorted(order[:64] % 16)[-1] == 7
    bl = cluster_tree_balanced(10, 3)
    assert bl[1] == [(0, 5), (5, 10)] and bl[2] == [(0, 3), (3, 5), (5, 8), (8, 10)]


def test_bfs_nearest_order_and_cut():
    # path 0-1-2-3-4 plus a star at 2: 2-5, 2-6
    adj = {0: [1], 1: [0, 2], 2: [1, 3, 5, 6], 3: [2, 4], 4: [3], 5: [2], 6: [2]}
    rp = [0]; ci = []
    for v in range(7):
        ci += adj[v]; rp.append(len(ci))
    rp, ci = np.array(rp), np.array(ci)
    allowed = np.ones(7, bool)
    tgt = np.ones(7, bool)
    assert bfs_nearest(rp, ci, 0, allowed, tgt, 3) == [1, 2, 3]
    assert bfs_nearest(rp, ci, 1, allowed, tgt, 4) == [0, 2, 3, 5]     # distance 2 cut by vertex order
    tgt2 = np.zeros(7, bool); tgt2[[4, 6]] = True
    assert bfs_nearest(rp, ci, 0, allowed, tgt2, 8) == [6, 4]         # 6 at distance 3, 4 at distance 4
    allowed[2] = False
    assert bfs_nearest(rp, ci, 0, allowed, tgt, 8) == [1]


def test_neighbour_lists_respect_targets():
    p = w.helmholtz7(12, 8)
    an = analyze(p, 32, 60, 16)
    f = [f for f in an.fronts if f.compressed and f.u][0]
    nn = front_neighbours(an, f, 4)
    s_set = set(range(f.sep_begin, f.sep_end)); u_set = set(f.upd.tolist())
    assert all(set(v) <= u_set and len(v) == 4 for v in nn["nn12"].values())
    assert all(set(v) <= s_set and len(v) == 4 for v in nn["nn21"].values())
    assert all(set(v) <= s_set for v in nn["nn11"].values())


# ---------------- graph nested dissection (general CSR input, no coordinates) ----------------
def _pattern_problem(n, edges, name="graph"):
    """A SparseProblem from an undirected edge list (unit off-diagonal, diagonal n), no coordinates."""
    import scipy.sparse as sp
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    r = np.concatenate([e[:, 0], e[:, 1], np.arange(n)])
    c = np.concatenate([e[:, 1], e[:, 0], np.arange(n)])
    v = np.concatenate([-np.ones(2 * len(e)), np.full(n, float(n))]).astype(complex)
    A = sp.csr_matrix((v, (r, c)), shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    return w.SparseProblem(name, n, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data,
                           np.zeros((n, 3), np.int32), w.LATTICE_NODE)


def random_graph(seed=4, n1=700, n2=120):
    """Two components: a random geometric graph in the unit square and a smaller one far away."""
    rng = np.random.default_rng(seed)
    pts = np.concatenate([rng.random((n1, 2)), 10.0 + rng.random((n2, 2))])
    d = np.sqrt(((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1))
    i, j = np.nonzero(np.triu(d < 0.075, 1))
    return _pattern_problem(n1 + n2, np.stack([i, j], 1), "rgg")


def test_graph_nd_path_by_hand():
    # path 0-1-...-9, leaf 3: the search from 0 ends at 9; from 9 the levels are 9, 8, ..., 0 and the
    # fifth level (vertex 5) is where half of the ten vertices are passed -> root separator {5};
    # [6..9]: levels from 9 are 9, 8, 7, 6 -> separator {8}, children [9] and [6, 7];
    # [0..4]: from 4 the levels are 4, 3, 2, 1, 0 -> separator {2}, children [3, 4] and [0, 1]
    p = _pattern_problem(10, [(k, k + 1) for k in range(9)])
    an = analyze(p, leaf_size=3, nmin_sep=10 ** 9, graph=True)
    assert an.perm.tolist() == [9, 6, 7, 8, 3, 4, 0, 1, 2, 5]
    assert [f.s for f in an.fronts] == [1, 2, 1, 2, 2, 1, 1]
    assert an.fronts[-1].children == [2, 5]


@pytest.mark.parametrize("gen", [lambda: w.helmholtz7(12, 8), lambda: w.yee_maxwell(6, 10), random_graph])
def test_graph_nd_structure_invariants(gen):
    p = gen()
    an = analyze(p, leaf_size=16, nmin_sep=40, hodbf_leaf=8, graph=True)
    N = p.n
    assert np.array_equal(np.sort(an.perm), np.arange(N))
    assert sum(f.s for f in an.fronts) == N
    A = p.to_scipy()[an.perm][:, an.perm].tocoo()
    owner = np.empty(N, np.int64)
    for f in an.fronts:
        owner[f.sep_begin:f.sep_end] = f.id
    anc = {}
    for f in an.fronts:
        a, q = set(), f.id
        while q >= 0:
            a.add(q); q = an.fronts[q].parent
        anc[f.id] = a
    for r, c in zip(A.row, A.col):        # separators separate: no entry couples unrelated fronts
        fr, fc = owner[r], owner[c]
        assert fr in anc[fc] or fc in anc[fr]
    for f in an.fronts:
        ok = set(range(f.sep_begin, f.sep_end)) | set(f.upd.tolist())
        for c in f.children:
            assert set(an.fronts[c].upd.tolist()) <= ok
        if f.compressed:
            assert max(b - a for a, b in f.th_tree[-1]) <= 8
    assert sum(f.compressed for f in an.fronts) >= 1


def test_graph_nd_symbolic_equals_bruteforce_elimination():
    for p in (w.helmholtz7(6, 8), w.yee_maxwell(4, 10), random_graph(5, 150, 30)):
        an = analyze(p, leaf_size=10, nmin_sep=10 ** 9, graph=True)
        N = p.n
        P = (p.to_scipy()[an.perm][:, an.perm].toarray() != 0)
        S = P.copy()
        for k in range(N):
            rows = np.nonzero(S[k + 1:, k])[0] + k + 1
            cols = np.nonzero(S[k, k + 1:])[0] + k + 1
            S[np.ix_(rows, cols)] = True
        for f in an.fronts:
            idx = list(range(f.sep_begin, f.sep_end))
            below = set()
            for k in idx:
                below |= set((np.nonzero(S[k + 1:, k])[0] + k + 1).tolist())
            assert below - set(idx) == set(f.upd.tolist())


def test_graph_separator_bisection_gives_compact_clusters():
    # Sec. 5.1: the HOD-BF hierarchy of a separator comes from recursive bisection of its graph, so
    # that the clusters are compact pieces of the separator surface (the off-diagonal ranks depend
    # on it).  The root separator of the level-structure ordering of a 24^3 grid is a diagonal
    # plane; every cluster of its tree keeps diameter / sqrt(size) below 3, as a disc-like piece of
    # a plane does, while the same tree over index order (strips) passes 4 at its leaves
    p = w.helmholtz7(24, 8)
    an = analyze(p, 64, 200, 32, graph=True)
    f = an.fronts[-1]
    assert f.compressed and len(f.th_tree) >= 5
    X = p.coords[an.perm].astype(float)

    def worst(S, lvl):
        return max(np.sqrt(((S[a:b, None] - S[None, a:b]) ** 2).sum(-1)).max() / np.sqrt(b - a)
                   for a, b in f.th_tree[lvl])
    S = X[f.sep_begin:f.sep_end]
    assert all(worst(S, lvl) < 3.0 for lvl in range(1, len(f.th_tree)))
    assert worst(X[np.sort(an.perm[f.sep_begin:f.sep_end])], len(f.th_tree) - 1) > 4.0
    # the separator is a level set of the 7-point graph: no edge joins two of its vertices
    A = p.to_scipy()[an.perm][:, an.perm].tocsr()[f.sep_begin:f.sep_end, f.sep_begin:f.sep_end]
    assert A.nnz == f.s


# ---------------- hybrid ordering: planar while compressed, graph nested dissection below ----------------
@pytest.mark.parametrize("gen", [lambda: w.helmholtz7(14, 8), lambda: w.yee_maxwell(6, 10)])
def test_hybrid_structure_invariants_and_symbolic(gen):
    p = gen()
    an = analyze(p, leaf_size=16, nmin_sep=40, hodbf_leaf=8, ordering="hybrid")
    N = p.n
    assert np.array_equal(np.sort(an.perm), np.arange(N))
    P = (p.to_scipy()[an.perm][:, an.perm].toarray() != 0)
    S = P.copy()
    for k in range(N):                      # brute-force symbolic elimination
        rows = np.nonzero(S[k + 1:, k])[0] + k + 1
        cols = np.nonzero(S[k, k + 1:])[0] + k + 1
        S[np.ix_(rows, cols)] = True
    # a part beyond a level-structure separator can fall apart into pieces that stay one subtree
    # (a front has at most two children), so an update set may also hold indices of the other
    # pieces' neighbours with no fill (structural zeros): it must contain the fill and lie in the
    # ancestors' separators
    owner = np.empty(N, np.int64)
    for f in an.fronts:
        owner[f.sep_begin:f.sep_end] = f.id
    extra = total = 0
    for f in an.fronts:
        idx = list(range(f.sep_begin, f.sep_end))
        below = set()
        for k in idx:
            below |= set((np.nonzero(S[k + 1:, k])[0] + k + 1).tolist())
        upd = set(f.upd.tolist())
        assert below - set(idx) <= upd
        anc, q = set(), f.parent
        while q >= 0:
            anc.add(q)
            q = an.fronts[q].parent
        assert all(int(owner[x]) in anc for x in upd)
        extra += len(upd - below)
        total += len(upd)
    assert extra <= 0.02 * total


def test_hybrid_keeps_the_compressed_fronts_of_the_planar_ordering():
    # the rule only reorders boxes whose planar separator would stay dense, so every compressed
    # front (its separator in HOD-BF order, its cluster trees and its update set, in original
    # numbering) is the planar ordering's, while the dense fronts hold less fill
    p = w.helmholtz7(24, 8)
    a0 = analyze(p, 32, 200, 32)
    a1 = analyze(p, 32, 200, 32, ordering="hybrid")

    def compressed(an):
        out = []
        for f in an.fronts:
            if f.compressed:
                out.append((an.perm[f.sep_begin:f.sep_end].tolist(), sorted(an.perm[f.upd].tolist()),
                            f.th_tree, f.f22_tree))
        return out
    c0, c1 = compressed(a0), compressed(a1)
    assert len(c0) >= 3 and len(c0) == len(c1)
    for x, y in zip(c0, c1):
        assert x[0] == y[0] and x[1] == y[1] and x[2] == y[2] and x[3] == y[3]

    def dense_fill(an):
        return sum(f.s * f.s + 2 * f.s * len(f.upd) for f in an.fronts if not f.compressed)
    assert dense_fill(a1) < 0.95 * dense_fill(a0)


# ---------------- parallel separators at the top levels (the remedy of the remark in Sec. 5.3) ----------------
@pytest.mark.parametrize("gen,args", [(lambda: w.helmholtz7(24, 8), (32, 150, 32)), (lambda: w.yee_maxwell(10, 10), (32, 100, 32))])
def test_parallel_levels_cut_along_the_root_axis(gen, args):
    p = gen()
    P = 3
    an = analyze(p, *args, parallel_levels=P)
    a0 = analyze(p, *args)
    assert np.array_equal(np.sort(an.perm), np.arange(p.n))
    # depth of every front below the root
    depth = {}
    for f in reversed(an.fronts):
        depth[f.id] = 0 if f.parent < 0 else depth[f.parent] + 1

    def axis(f):
        c = p.coords[an.perm[f.sep_begin:f.sep_end]]
        return int(np.argmin(c.max(0) - c.min(0)))   # the separator plane's constant coordinate
    root = an.fronts[-1]
    for f in an.fronts:
        if 0 < depth[f.id] < P and f.s > an.leaf_size:
            assert axis(f) == axis(root)
    # the default rule alternates: some separator of depth 1 or 2 crosses the root separator
    d0 = {}
    for f in reversed(a0.fronts):
        d0[f.id] = 0 if f.parent < 0 else d0[f.parent] + 1
    c = [int(np.argmin(np.ptp(p.coords[a0.perm[f.sep_begin:f.sep_end]], axis=0)))
         for f in a0.fronts if d0[f.id] in (1, 2) and f.s > a0.leaf_size]
    assert any(x != axis(a0.fronts[-1]) for x in c)
