"""Oracle: symbolic analysis of the multifrontal method (test infrastructure only).

This file is part of the CPU oracle.  It is test infrastructure: only the
tests, the smoke check and the benchmark's CPU-baseline leg may use it.  It
shares no code with the GPU path (whose host analysis is written separately
in C++ from the same rules) and must agree with it bit for bit.

Rules implemented (Sec. 2; Sec. 5.1; Sec. 5.2; the ordering and symbolic steps of Alg. 1 and Alg. 5):
  * nested dissection by planar separators on lattice boxes (the Helmholtz runs
    of Sec. 6 use planar separators), or, for a general CSR input without
    coordinates, by graph level structures (breadth-first search from a
    pseudo-peripheral vertex; the separator is the level where half of the
    reached vertices are passed; compressed separators ordered by a
    breadth-first search of their own subgraph, balanced cluster tree),
  * post-order assembly tree, I^s (a separator) and I^u (update set) per front,
    with  I^u_nu  contained in  I^s_tau U I^u_tau  (Sec. 2),
  * rank-reducing separator reordering P-hat by recursive geometric bisection
    of compressed separators (Sec. 5.1) -> HOD-BF cluster tree T_H,
  * F22 cluster tree: sorted I^u split into balanced halves (Sec. 5.1),
  * graph nearest neighbours by breadth-first search (Sec. 5.2).

Readings where the paper is silent (planar separators instead of METIS, tie
breaks, uniform-depth cluster trees) are the builder's and documented.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

LATTICE_NODE = 0
LATTICE_EDGE = 1


@dataclass
class Front:
    id: int
    parent: int
    children: list
    sep_begin: int               # I^s = [sep_begin, sep_end) in the new numbering
    sep_end: int
    sub_begin: int               # first new index in this front's subtree
    upd: np.ndarray              # I^u, sorted new indices (int64)
    level: int = 0               # depth in the assembly tree (root = 0)
    compressed: bool = False
    th_tree: list = field(default_factory=list)    # T_H levels: lists of (a, b) ranges over [0, s)
    f22_tree: list = field(default_factory=list)   # F22 levels: lists of (a, b) ranges over [0, u)

    @property
    def s(self):
        return self.sep_end - self.sep_begin

    @property
    def u(self):
        return len(self.upd)


@dataclass
class Analysis:
    n: int
    perm: np.ndarray             # perm[new] = old
    iperm: np.ndarray            # iperm[old] = new
    fronts: list                 # in post-order (children before parents)
    rowptr: np.ndarray           # permuted pattern (new numbering), CSR
    colind: np.ndarray
    leaf_size: int
    nmin_sep: int
    hodbf_leaf: int


def _lex_order(coords: np.ndarray, ids: np.ndarray) -> np.ndarray:
    """ids sorted by (z, y, x) of their coordinates (x fastest)."""
    c = coords[ids]
    key = np.lexsort((c[:, 0], c[:, 1], c[:, 2]))
    return ids[key]


def _initial_box(coords: np.ndarray, lattice: int):
    mn = coords.min(axis=0).astype(np.int64)
    mx = coords.max(axis=0).astype(np.int64)
    if lattice == LATTICE_NODE:
        return mn, mx + 1
    lo = 2 * ((mn - 1) // 2) + 1
    hi = 2 * (mx // 2 + 1)
    return lo, hi


def _split(lo, hi, lattice, axis=None):
    """Separator axis and plane coordinate for a box [lo, hi) (half-open per axis).  axis: cut along
    this axis instead when the box extends 3 or more units along it (parallel separators)."""
    if lattice == LATTICE_NODE:
        ext = hi - lo
    else:
        ext = (hi - lo + 1) // 2          # number of lattice cells
    a = int(np.argmax(ext))               # first axis of largest extent: x, then y, then z
    if axis is not None and ext[axis] >= 3:
        a = int(axis)
    if lattice == LATTICE_NODE:
        mid = int(lo[a] + ext[a] // 2)
    else:
        mid = int((lo[a] - 1) + 2 * (ext[a] // 2))
    return a, mid


def cluster_tree_geometric(coords: np.ndarray, leaf: int):
    """Recursive geometric bisection of a point set (Sec. 5.1), uniform depth.

    Returns (order, levels): order is a permutation of range(len(coords));
    levels[l] is the list of (a, b) ranges of the clusters at level l over the
    reordered points.  Every cluster of a level is split while any cluster of
    that level holds more than `leaf` points.  A cluster is cut at
    lo + ext//2 along the first axis of largest bounding-box extent.
    """
    npts = len(coords)
    base = _lex_order(coords, np.arange(npts))
    clusters = [base]
    levels_lists = [clusters]
    while max(len(c) for c in clusters) > leaf:
        new = []
        for c in clusters:
            if len(c) == 0:
                new += [c, c]
                continue
            cc = coords[c]
            lo = cc.min(axis=0)
            ext = cc.max(axis=0) - lo + 1
            a = int(np.argmax(ext))
            cut = lo[a] + ext[a] // 2
            new.append(c[cc[:, a] < cut])
            new.append(c[cc[:, a] >= cut])
        clusters = new
        levels_lists.append(clusters)
    order = np.concatenate(clusters) if clusters else np.zeros(0, np.int64)
    # express every level as ranges of the final order
    levels = []
    for lv in levels_lists:
        ranges, p = [], 0
        for c in lv:
            ranges.append((p, p + len(c)))
            p += len(c)
        levels.append(ranges)
    # The final order must refine every level: true because each split keeps
    # the relative order of its parent and children are concatenated in order.
    return order.astype(np.int64), levels


def cluster_tree_balanced(npts: int, leaf: int):
    """Balanced index bisection: first ceil(len/2) / rest, uniform depth."""
    levels = [[(0, npts)]]
    while max(b - a for a, b in levels[-1]) > leaf:
        new = []
        for a, b in levels[-1]:
            m = a + (b - a + 1) // 2
            new += [(a, m), (m, b)]
        levels.append(new)
    return levels


def _separator_bisection(sep, adj, th):
    """Order a graph separator by recursive bisection along its HOD-BF tree th (Sec. 5.1).

    In the algebraic setting the paper takes the HOD-BF hierarchy of F11 from a recursive
    bisection of the graph of A(I^s, I^s).  A level-structure separator of a 7-point stencil has
    no edges inside it (its vertices all lie at one distance from p), so the graph bisected here
    is the two-hop graph of the separator: u ~ v when A(u, v) != 0 or u and v share a neighbour
    in A.  Bisection of a node's vertex set (sorted): breadth-first search from its smallest
    vertex (neighbours in increasing index), p = the smallest vertex of the last level, search
    again from p; the sequence is the levels from p, each sorted, then the vertices not reached
    (sorted).  The node's first child takes the first (child size) vertices of the sequence, the
    second child the rest; leaves are sorted.  Returns the separator in HOD-BF order."""
    S = set(sep)
    adj2 = {}
    for v in sep:
        nb = set()
        for x in adj[v]:
            if x in S:
                nb.add(x)
            for y in adj[x]:
                if y in S and y != v:
                    nb.add(y)
        adj2[v] = sorted(nb)

    def levels_from(start, inside, seen):
        lv = [[start]]
        seen.add(start)
        while True:
            nxt = []
            for v in lv[-1]:
                for x in adj2[v]:
                    if x in inside and x not in seen:
                        seen.add(x)
                        nxt.append(x)
            if not nxt:
                return lv
            lv.append(nxt)

    def split(vs, h):
        if not vs:
            return [], []
        inside = set(vs)
        p = min(levels_from(vs[0], inside, set())[-1])
        reached = set()
        seq = [v for level in levels_from(p, inside, reached) for v in sorted(level)]
        seq += [v for v in vs if v not in reached]
        return sorted(seq[:h]), sorted(seq[h:])

    def order(vs, lvl, k):
        if lvl == len(th) - 1:
            return vs
        a, m = th[lvl + 1][2 * k]
        left, right = split(vs, m - a)
        return order(left, lvl + 1, 2 * k) + order(right, lvl + 1, 2 * k + 1)

    return order(sorted(sep), 0, 0)


def _graph_nd(N, rp, ci, leaf_size, nmin_sep, hodbf_leaf, fronts_sep, perm_parts):
    """Graph nested dissection of a CSR pattern (no coordinates); returns the recursion nd(ids),
    which orders the vertex set ids (sorted) and returns the front id of its subtree root.

    The fill-reducing ordering of a general sparse matrix comes from nested dissection of its
    graph (Sec. 2; the Maxwell experiment of Sec. 6.2 is ordered this way).  The graph is the
    (structurally symmetric) pattern of A without self loops.  The bisection rule here is a level-structure one
    (METIS's multilevel partitioner, which the paper names, is a library this project does not
    reproduce); the rule is deterministic, so the GPU analysis can be compared with it exactly.
    A set of more than leaf_size vertices: breadth-first search inside the set from its smallest
    vertex, neighbours visited in increasing index; p = the smallest vertex of the last level;
    search again from p.  The separator is level m, the first level at which levels 0..m hold at
    least half of the vertices reached from p, kept in 1 .. (number of levels - 2); levels below m
    form the first child, levels above m and the vertices not reached from p (other components)
    the second.  With fewer than three levels the set is a front of its own.  A separator at or
    above nmin_sep is ordered by _separator_bisection along its balanced HOD-BF tree."""
    adj = [sorted(set(int(c) for c in ci[rp[i]:rp[i + 1]]) - {i}) for i in range(N)]

    def bfs(start, inside, seen):
        levels = [[start]]
        seen.add(start)
        while True:
            nxt = []
            for v in levels[-1]:
                for w in adj[v]:
                    if w in inside and w not in seen:
                        seen.add(w)
                        nxt.append(w)
            if not nxt:
                return levels
            levels.append(nxt)

    def new_front(sep, kids, compressed, th):
        sep = np.asarray(sep, dtype=np.int64)
        fronts_sep.append((sep, kids, compressed, th))
        perm_parts.append(sep)
        return len(fronts_sep) - 1

    def nd(ids):                     # ids: sorted list of vertices
        if len(ids) <= leaf_size:
            return new_front(ids, [], False, None)
        inside = set(ids)
        lv0 = bfs(ids[0], inside, set())
        p = min(lv0[-1])
        reached = set()
        lv = bfs(p, inside, reached)
        nl = len(lv)
        if nl < 3:
            return new_front(ids, [], False, None)
        total = sum(len(l) for l in lv)
        acc, m = 0, 0
        while m < nl:
            acc += len(lv[m])
            if 2 * acc >= total:
                break
            m += 1
        m = max(1, min(m, nl - 2))
        left = sorted(v for i in range(m) for v in lv[i])
        right = sorted([v for i in range(m + 1, nl) for v in lv[i]] + [v for v in ids if v not in reached])
        sep = sorted(lv[m])
        kids = []
        if left:
            kids.append(nd(left))
        if right:
            kids.append(nd(right))
        if len(sep) >= nmin_sep:
            th = cluster_tree_balanced(len(sep), hodbf_leaf)
            return new_front(_separator_bisection(sep, adj, th), kids, True, th)
        return new_front(sep, kids, False, None)

    return nd


def analyze(prob, leaf_size=64, nmin_sep=1024, hodbf_leaf=64, graph=False, ordering="auto",
            parallel_levels=0) -> Analysis:
    """Nested dissection + assembly tree + symbolic factorization (the ordering and symbolic steps of Alg. 1 and Alg. 5).
    ordering: "auto" (planar separators), "graph" (graph nested dissection of the pattern, the
    coordinates ignored; also graph=True) or "hybrid" (planar separators while they are compressed,
    |sep| >= nmin_sep; a box whose planar separator would be smaller, a dense front, is ordered by
    graph nested dissection of its vertices).  Nested dissection is the paper's fill-reducing
    ordering (Sec. 2); the choice of separators below the compressed levels is free.
    parallel_levels: the planar rule cuts the boxes of the top parallel_levels levels along the
    root's axis, so that those separators are parallel planes rather than crossing ones (the
    remedy the remark of Sec. 5.3 gives for the ranks of F12 / F21 between crossing separators)."""
    if graph:
        ordering = "graph"
    if ordering not in ("auto", "hybrid", "graph"):
        raise ValueError(f"unknown ordering {ordering}")
    lattice = prob.lattice
    N = prob.n
    rp, ci = prob.rowptr, prob.colind
    gnd = None

    fronts_sep = []     # list of (old ids of separator in front order, children front ids, compressed)
    perm_parts = []

    root_axis = [0]

    def nd(ids, lo, hi, depth=0):
        """Returns the front id of the subtree root."""
        if len(ids) <= leaf_size:
            sep = _lex_order(coords, ids)
            fid = len(fronts_sep)
            fronts_sep.append((sep, [], False, None))
            perm_parts.append(sep)
            return fid
        a, mid = _split(lo, hi, lattice, root_axis[0] if 0 < depth < parallel_levels else None)
        if depth == 0:
            root_axis[0] = a
        ca = coords[ids, a]
        if ordering == "hybrid" and int(np.count_nonzero(ca == mid)) < nmin_sep:
            return gnd(sorted(int(v) for v in ids))   # the box's planar separator would stay dense
        left = ids[ca < mid]
        right = ids[ca > mid]
        sep = ids[ca == mid]
        kids = []
        if len(left):
            hi2 = hi.copy(); hi2[a] = mid
            kids.append(nd(left, lo.copy(), hi2, depth + 1))
        if len(right):
            lo2 = lo.copy(); lo2[a] = mid + 1
            kids.append(nd(right, lo2, hi.copy(), depth + 1))
        if len(sep) == 0:
            raise ValueError("empty separator: the lattice rule does not apply to this input")
        compressed = len(sep) >= nmin_sep
        if compressed:
            order, th = cluster_tree_geometric(coords[_lex_order(coords, sep)], hodbf_leaf)
            sep = _lex_order(coords, sep)[order]
        else:
            sep = _lex_order(coords, sep)
            th = None
        fid = len(fronts_sep)
        fronts_sep.append((sep, kids, compressed, th))
        perm_parts.append(sep)
        return fid

    if ordering != "auto":
        gnd = _graph_nd(N, rp, ci, leaf_size, nmin_sep, hodbf_leaf, fronts_sep, perm_parts)
    if ordering == "graph":
        gnd(list(range(N)))
    else:
        coords = prob.coords.astype(np.int64)
        lo, hi = _initial_box(coords, lattice)
        nd(np.arange(N, dtype=np.int64), lo, hi)

    perm = np.concatenate(perm_parts).astype(np.int64)
    assert len(perm) == N
    iperm = np.empty(N, dtype=np.int64)
    iperm[perm] = np.arange(N)

    # permuted pattern
    A = prob.to_scipy()
    Ap = A[perm][:, perm].tocsr()
    Ap.sort_indices()
    prp, pci = Ap.indptr.astype(np.int64), Ap.indices.astype(np.int64)

    fronts = []
    pos = 0
    for fid, (sep, kids, compressed, th) in enumerate(fronts_sep):
        f = Front(fid, -1, list(kids), pos, pos + len(sep), pos, np.zeros(0, np.int64),
                  compressed=compressed, th_tree=th or [])
        pos += len(sep)
        fronts.append(f)
    for f in fronts:
        for c in f.children:
            fronts[c].parent = f.id
    for f in fronts:       # subtree start = min over children subtree starts
        if f.children:
            f.sub_begin = min(fronts[c].sub_begin for c in f.children)
    # symbolic: I^u = (adj(I^s) U children I^u) \ subtree
    for f in fronts:
        cand = [pci[prp[f.sep_begin]:prp[f.sep_end]]]
        for c in f.children:
            cand.append(fronts[c].upd)
        u = np.unique(np.concatenate(cand)) if cand else np.zeros(0, np.int64)
        f.upd = u[u >= f.sep_end].astype(np.int64)
        f.f22_tree = cluster_tree_balanced(len(f.upd), hodbf_leaf) if f.compressed else []
    # depth
    for f in reversed(fronts):
        f.level = 0 if f.parent < 0 else fronts[f.parent].level + 1
    return Analysis(N, perm, iperm, fronts, prp, pci, leaf_size, nmin_sep, hodbf_leaf)


# ---------------------------------------------------------------------------
# Graph nearest neighbours (Sec. 5.2)
# ---------------------------------------------------------------------------
def bfs_nearest(rp, ci, start: int, allowed: np.ndarray, target: np.ndarray, knn: int) -> list:
    """First `knn` vertices v with target[v] found by BFS from `start`.

    BFS runs on the subgraph induced by the vertices with allowed[v] (new
    numbering).  Vertices are taken level by level (distance 1, 2, ...), in
    increasing vertex order within a level; the last level is cut by vertex
    order.  The start vertex itself is never returned.
    """
    seen = {start}
    frontier = [start]
    out = []
    while frontier and len(out) < knn:
        nxt = set()
        for v in frontier:
            for w in ci[rp[v]:rp[v + 1]]:
                w = int(w)
                if allowed[w] and w not in seen:
                    nxt.add(w)
        nxt = sorted(nxt)
        seen.update(nxt)
        for w in nxt:
            if target[w]:
                out.append(w)
                if len(out) == knn:
                    break
        frontier = nxt
    return out


def front_neighbours(an: Analysis, f: Front, knn: int, stride: int = 1):
    """Nearest-neighbour lists of a compressed front (Sec. 5.2).

    stride > 1 computes the lists of every stride-th vertex of I^s and of I^u only (a sample
    for checks at full size); the lists themselves do not depend on it.

    Returns dict with
      nn11[x]  x in I^s : first knn vertices of graph A(I^s,I^s) outside x's T_H leaf,
      nn22[x]  x in I^u : first knn vertices of graph A(I^u,I^u) outside x's F22 leaf,
      nn12[x]  x in I^s : first knn vertices in I^u, BFS on A over I^s U I^u,
      nn21[y]  y in I^u : first knn vertices in I^s, same graph.
    Lists hold new (global) indices.
    """
    N = an.n
    rp, ci = an.rowptr, an.colind
    s_idx = np.arange(f.sep_begin, f.sep_end)
    u_idx = f.upd
    in_s = np.zeros(N, bool); in_s[s_idx] = True
    in_u = np.zeros(N, bool); in_u[u_idx] = True
    both = in_s | in_u
    out = {}
    # T_H leaf id per separator vertex
    leaf_of = np.full(N, -1, np.int64)
    for li, (a, b) in enumerate(f.th_tree[-1] if f.th_tree else [(0, f.s)]):
        leaf_of[f.sep_begin + a: f.sep_begin + b] = li
    s_sel, u_sel = s_idx[::stride], u_idx[::stride]
    nn11 = {}
    for x in s_sel:
        tgt = in_s & (leaf_of != leaf_of[x])
        nn11[int(x)] = bfs_nearest(rp, ci, int(x), in_s, tgt, knn)
    out["nn11"] = nn11
    leaf22 = np.full(N, -1, np.int64)
    if len(u_idx):
        for li, (a, b) in enumerate(f.f22_tree[-1] if f.f22_tree else [(0, f.u)]):
            leaf22[u_idx[a:b]] = li
    nn22 = {}
    for x in u_sel:
        tgt = in_u & (leaf22 != leaf22[x])
        nn22[int(x)] = bfs_nearest(rp, ci, int(x), in_u, tgt, knn)
    out["nn22"] = nn22
    out["nn12"] = {int(x): bfs_nearest(rp, ci, int(x), both, in_u, knn) for x in s_sel}
    out["nn21"] = {int(y): bfs_nearest(rp, ci, int(y), both, in_s, knn) for y in u_sel}
    return out


def levels_of_fronts(an: Analysis):
    """Fronts grouped by assembly-tree depth, deepest first."""
    depth = max(f.level for f in an.fronts) + 1
    lv = [[] for _ in range(depth)]
    for f in an.fronts:
        lv[f.level].append(f.id)
    return lv[::-1]
