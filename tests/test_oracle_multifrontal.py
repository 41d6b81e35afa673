"""Pins of the oracle's compressed multifrontal solver (Alg. 5) and GMRES."""
import numpy as np
import pytest

import workloads as w
from oracle.analysis import analyze
from oracle import dense_mf as dm, compressed_mf as cm, gmres as gm


@pytest.fixture(scope="module")
def cfg16():
    p = w.helmholtz7(16, 8)
    b = w.rhs_point_plus_gaussian(p, 42)
    an0 = analyze(p, 64, 10 ** 9, 64)
    fac0, _ = dm.multifrontal_factor(p, an0)
    return p, b, dm.solve(p, an0, fac0, b)


def test_16cube_tol1e6_is_a_direct_solver(cfg16):
    # Sec. 6.2: at eps = 1e-6 the HOD-BF solver serves as a direct solver.
    # Bound used: 100 * tol on both the error and the residual (no refinement).
    p, b, xe = cfg16
    an = analyze(p, 64, 128, 64)
    fac, st = cm.compressed_factor(p, an, 1e-6)
    assert st["compressed"] == 2
    x = cm.preconditioner(an, fac)(b)
    A = p.to_scipy()
    assert np.linalg.norm(x - xe) / np.linalg.norm(xe) <= 1e-4
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= 1e-4
    X, its, res = gm.gmres(A, b, cm.preconditioner(an, fac), rtol=1e-8)
    assert res[0] <= 1e-8 and its[0] <= 3
    assert np.linalg.norm(X[:, 0] - xe[:, 0]) / np.linalg.norm(xe) <= 1e-6


def test_tight_tolerance_reproduces_exact():
    p = w.helmholtz7(10, 8)
    b = w.rhs_gaussian(p, 1, 9)
    an = analyze(p, 16, 40, 16)
    fac, st = cm.compressed_factor(p, an, 1e-12)
    assert st["compressed"] >= 2
    an0 = analyze(p, 16, 10 ** 9, 16)
    xe = dm.solve(p, an0, dm.multifrontal_factor(p, an0)[0], b)
    x = cm.preconditioner(an, fac)(b)
    assert np.linalg.norm(x - xe) / np.linalg.norm(xe) <= 1e-9


def test_gmres_iterations_fall_with_tolerance():
    # Tables 2 and 3: tighter eps -> fewer GMRES iterations
    p = w.helmholtz7(12, 8)
    b = w.rhs_gaussian(p, 1, 5)
    an = analyze(p, 32, 60, 16)
    A = p.to_scipy()
    its = []
    for tol in (1e-2, 1e-4, 1e-6):
        fac, _ = cm.compressed_factor(p, an, tol)
        _, it, res = gm.gmres(A, b, cm.preconditioner(an, fac), rtol=1e-8)
        assert res[0] <= 1e-8
        its.append(it[0])
    assert its[0] > its[1] > its[2]


def test_refinement_with_exact_factor():
    p = w.helmholtz7(8, 8)
    an = analyze(p, 16, 10 ** 9)
    fac, _ = dm.multifrontal_factor(p, an)
    b = w.rhs_gaussian(p, 2, 1)
    X, its, res = gm.refine(p.to_scipy(), b, lambda v: dm.solve(p, an, fac, v))
    assert its <= 1 and max(res) <= 1e-12
