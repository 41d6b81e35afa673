"""C-ABI tests that need no GPU: the library loads, exports every declared
symbol, validates its arguments, and its host analysis equals the oracle's
bit for bit (nested dissection, tree, update sets, cluster trees, neighbours)."""
import os
import re

import numpy as np
import pytest

import workloads as w
from oracle.analysis import analyze, front_neighbours

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def g():
    from paper_2007_00202_gb300 import build
    build.build()
    import paper_2007_00202_gb300 as pkg
    return pkg


def _declared():
    src = open(os.path.join(ROOT, "include", "mf.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int64_t|int|void|const char\*)\s+(mf_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol(g):
    L = g.lib()
    names = _declared()
    assert "mf_analyze" in names and "mf_factor" in names and "mf_solve" in names
    for n in names:
        assert hasattr(L, n), n
    from paper_2007_00202_gb300.mf import SIGNATURES
    assert set(SIGNATURES) <= set(names)


def test_argument_errors(g):
    from paper_2007_00202_gb300.mf import MfError
    p = w.helmholtz7(4, 8)
    with pytest.raises(MfError) as e:
        g.mf_analyze(p.n, p.rowptr, np.full_like(p.colind, p.n + 5), p.vals, p.coords)
    assert e.value.code == -1
    # an unsymmetric pattern (row 0 loses one off-diagonal entry) is rejected
    rp, ci, v = p.rowptr.copy(), p.colind.copy(), p.vals.copy()
    k = int(np.flatnonzero(ci[rp[0]:rp[1]] != 0)[0])
    keep = np.ones(len(ci), bool)
    keep[k] = False
    rp[1:] -= 1
    with pytest.raises(MfError) as e:
        g.mf_analyze(p.n, rp, ci[keep], v[keep], None)
    assert e.value.code == -1 and "symmetric" in str(e.value)
    h = g.analyze_problem(p)
    with pytest.raises(MfError) as e:
        h.mf_solve(np.ones(p.n, complex))
    assert e.value.code == -2          # solve before factor
    o = g.mf_options_init()
    assert (o.leaf_size, o.nmin_sep, o.gmres_restart, o.rtol) == (64, 1024, 30, 1e-8)


def _compare(g, p, leaf, nmin, hleaf, knn=8, check_nn=True, stride=1, graph=False, ordering="auto", parallel=0):
    an = analyze(p, leaf, nmin, hleaf, graph=graph, ordering=ordering, parallel_levels=parallel)
    code = {"auto": g.MF_ORDER_AUTO, "hybrid": g.MF_ORDER_HYBRID, "graph": g.MF_ORDER_GRAPH}[ordering]
    h = g.analyze_problem(p, graph=graph, leaf_size=leaf, nmin_sep=nmin, hodbf_leaf=hleaf, ordering=code,
                          parallel_levels=parallel)
    e = h.mf_analysis_export()
    assert np.array_equal(e["perm"], an.perm)
    assert len(e["parent"]) == len(an.fronts)
    for i, f in enumerate(an.fronts):
        assert e["parent"][i] == f.parent
        assert tuple(e["sep"][i]) == (f.sep_begin, f.sep_end)
        assert bool(e["compressed"][i]) == f.compressed
        assert np.array_equal(e["upd_idx"][e["upd_ptr"][i]:e["upd_ptr"][i + 1]], f.upd)
        if f.compressed:
            th, f22 = h.mf_front_trees(f.id)
            assert th == [list(map(tuple, l)) for l in f.th_tree]
            assert f22 == [list(map(tuple, l)) for l in f.f22_tree]
            if check_nn:
                nn = h.mf_front_neighbours(f.id, knn, f.s, f.u)
                on = front_neighbours(an, f, knn, stride)
                S = range(f.sep_begin, f.sep_end, stride)
                U = [int(x) for x in f.upd[::stride]]
                assert nn["nn11"][::stride] == [on["nn11"][x] for x in S]
                assert nn["nn12"][::stride] == [on["nn12"][x] for x in S]
                assert nn["nn21"][::stride] == [on["nn21"][x] for x in U]
                assert nn["nn22"][::stride] == [on["nn22"][x] for x in U]
    return an


def test_analysis_bit_exact_helmholtz(g):
    an = _compare(g, w.helmholtz7(16, 8), 64, 128, 64)
    assert sum(f.compressed for f in an.fronts) == 2


def test_analysis_bit_exact_odd_sizes(g):
    _compare(g, w.helmholtz7(13, 8), 20, 40, 16, knn=5)


def test_analysis_bit_exact_yee(g):
    _compare(g, w.yee_maxwell(8, 10), 32, 60, 16)


def test_analysis_bit_exact_64cube_structure(g):
    # full-size configuration of the 64^3 workload: ordering, tree, cluster trees, and the
    # neighbour lists of every compressed front at every 23rd vertex of I^s and of I^u
    p = w.helmholtz7(64, 10)
    an = _compare(g, p, 64, 1024, 64, stride=23)
    assert len(an.fronts) == 4817
    assert sum(f.compressed for f in an.fronts) == 5


def test_hybrid_analysis_bit_exact_64cube(g):
    # the 64^3 workload in the hybrid ordering: graph nested dissection below the compressed
    # levels, the same 5 compressed fronts; tree, update sets and cluster trees in full (the
    # neighbour lists are covered by the planar test above, the compressed fronts being the same)
    p = w.helmholtz7(64, 10)
    an = _compare(g, p, 64, 1024, 64, check_nn=False, ordering="hybrid")
    assert len(an.fronts) == 7847
    assert sum(f.compressed for f in an.fronts) == 5


@pytest.mark.parametrize("which", ["helmholtz13", "yee8", "rgg"])
def test_graph_analysis_bit_exact(g, which):
    # general CSR input (coordinates withheld): the graph nested dissection of the C++ host analysis
    # equals the oracle's bit for bit, including cluster trees and neighbour lists
    from test_oracle_analysis import random_graph
    p = {"helmholtz13": lambda: w.helmholtz7(13, 8), "yee8": lambda: w.yee_maxwell(8, 10),
         "rgg": random_graph}[which]()
    an = _compare(g, p, 24, 40, 16, knn=6, graph=True)
    assert sum(f.compressed for f in an.fronts) >= 1


@pytest.mark.parametrize("which", ["helmholtz13", "helmholtz16", "yee8"])
def test_hybrid_analysis_bit_exact(g, which):
    # planar separators while compressed, graph nested dissection inside boxes whose planar
    # separator would stay dense: the host analysis equals the oracle's bit for bit
    p, args = {"helmholtz13": (w.helmholtz7(13, 8), (24, 40, 16)), "helmholtz16": (w.helmholtz7(16, 8), (32, 100, 16)),
               "yee8": (w.yee_maxwell(8, 10), (24, 40, 16))}[which]
    an = _compare(g, p, *args, knn=6, ordering="hybrid")
    assert sum(f.compressed for f in an.fronts) >= 1


def test_graph_ordering_with_coordinates_bit_exact(g):
    # MF_ORDER_GRAPH ignores the coordinates it is given
    _compare(g, w.helmholtz7(12, 8), 24, 40, 16, knn=6, ordering="graph")
    h = g.analyze_problem(w.helmholtz7(12, 8), graph=True, leaf_size=24, nmin_sep=40, hodbf_leaf=16)
    h2 = g.analyze_problem(w.helmholtz7(12, 8), leaf_size=24, nmin_sep=40, hodbf_leaf=16, ordering=g.MF_ORDER_GRAPH)
    assert np.array_equal(h.mf_analysis_export()["perm"], h2.mf_analysis_export()["perm"])


def test_version_1_options_ignore_the_ordering_field(g):
    # a caller built against the first options layout (ending at coords) gets the planar ordering
    import ctypes as C
    import paper_2007_00202_gb300.mf as mf
    p = w.helmholtz7(12, 8)
    o = mf.mf_options_init(leaf_size=24, nmin_sep=40, hodbf_leaf=16, ordering=mf.MF_ORDER_HYBRID)
    o.version = mf.MF_OPTIONS_V1
    coords = np.ascontiguousarray(p.coords, dtype=np.int32)
    o.coords = coords.ctypes.data_as(C.POINTER(C.c_int32))
    vals = np.ascontiguousarray(p.vals, dtype=np.complex128)
    h = C.c_void_p()
    rc = mf.lib().mf_analyze(p.n, p.rowptr.ctypes.data_as(C.POINTER(C.c_int64)),
                             np.ascontiguousarray(p.colind, dtype=np.int32).ctypes.data_as(C.POINTER(C.c_int32)),
                             C.cast(vals.ctypes.data, C.POINTER(C.c_double)), C.byref(o), None, C.byref(h))
    assert rc == 0
    hv1 = mf.Handle(h, (coords, vals))
    assert np.array_equal(hv1.mf_analysis_export()["perm"], analyze(p, 24, 40, 16).perm)
    with pytest.raises(mf.MfError):   # the hybrid rule reads coordinates
        g.analyze_problem(p, graph=True, ordering=mf.MF_ORDER_HYBRID)
    for bad in ({"ordering": 7}, {"parallel_levels": -1}):
        with pytest.raises(mf.MfError) as e:
            g.analyze_problem(p, **bad)
        assert e.value.code == -1, bad


@pytest.mark.parametrize("which,parallel", [("helmholtz24", 2), ("helmholtz24", 3), ("yee10", 3), ("hybrid20", 3)])
def test_parallel_levels_analysis_bit_exact(g, which, parallel):
    # parallel separators at the top levels (planar rule along the root's axis): bit for bit
    p, args, o = {"helmholtz24": (w.helmholtz7(24, 8), (32, 150, 32), "auto"),
                  "yee10": (w.yee_maxwell(10, 10), (32, 100, 32), "auto"),
                  "hybrid20": (w.helmholtz7(20, 8), (32, 150, 32), "hybrid")}[which]
    an = _compare(g, p, *args, knn=6, ordering=o, parallel=parallel)
    assert sum(f.compressed for f in an.fronts) >= 2

