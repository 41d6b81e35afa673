"""GPU parity of the dense multifrontal path (Alg. 1) against the oracle, through the C ABI."""
import numpy as np
import pytest

import workloads as w
from oracle.analysis import analyze
from oracle import dense_mf as dm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2007_00202_gb300 import build
    build.build()
    import paper_2007_00202_gb300 as pkg
    return pkg


def _oracle_exact(p, b, leaf=64):
    an = analyze(p, leaf, 10 ** 9)
    fac, _ = dm.multifrontal_factor(p, an)
    return dm.solve(p, an, fac, b)


@pytest.mark.parametrize("gen,leaf", [(lambda: w.helmholtz7(8, 8), 16), (lambda: w.helmholtz7(16, 8), 64),
                                      (lambda: w.helmholtz7(11, 8), 20), (lambda: w.yee_maxwell(6, 10), 32)])
def test_fp64_exact_factor_matches_oracle(g, gen, leaf):
    p = gen()
    b = w.rhs_gaussian(p, 3, 2)
    h = g.analyze_problem(p, leaf_size=leaf, nmin_sep=10 ** 9, precision=g.MF_PREC_C128, refine=g.MF_REFINE_NONE)
    h.mf_factor(0.0)
    x, info = h.mf_solve(b)
    xo = _oracle_exact(p, b, leaf)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-11
    assert info.max_rel_residual < 1e-11


def test_mixed_precision_gmres_reaches_1e8(g):
    p = w.helmholtz7(16, 8)
    b = w.rhs_point_plus_gaussian(p, 42)
    h = g.analyze_problem(p, nmin_sep=10 ** 9, precision=g.MF_PREC_C64, refine=g.MF_REFINE_GMRES)
    h.mf_factor(0.0)
    x, info = h.mf_solve(b)
    A = p.to_scipy()
    res = np.linalg.norm(A @ x - b) / np.linalg.norm(b)        # independent FP64 residual on the host
    assert res <= 1e-8 and info.converged == 1
    assert info.iters <= 6
    xo = _oracle_exact(p, b)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-6
    # without refinement the complex64 factorization alone is a few 1e-5 accurate
    h2 = g.analyze_problem(p, nmin_sep=10 ** 9, precision=g.MF_PREC_C64, refine=g.MF_REFINE_NONE)
    h2.mf_factor(0.0)
    x2, _ = h2.mf_solve(b)
    assert np.linalg.norm(x2 - xo) / np.linalg.norm(xo) < 1e-2


def test_iterative_refinement_fp64(g):
    p = w.helmholtz7(10, 8)
    b = w.rhs_gaussian(p, 2, 4)
    h = g.analyze_problem(p, leaf_size=20, nmin_sep=10 ** 9, precision=g.MF_PREC_C128, refine=g.MF_REFINE_IR)
    h.mf_factor(0.0)
    x, info = h.mf_solve(b)
    assert info.converged == 1 and info.iters <= 1
    assert np.linalg.norm(p.to_scipy() @ x - b) / np.linalg.norm(b) < 1e-12


def test_solve_device_and_refactor(g):
    import torch
    p = w.helmholtz7(12, 8)
    b = w.rhs_gaussian(p, 4, 5)
    h = g.analyze_problem(p, leaf_size=32, nmin_sep=10 ** 9)
    h.mf_factor(0.0)
    h.mf_factor(0.0)                                  # refactorization reuses the plan
    bd = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()      # column-major N x nrhs == row-major nrhs x N
    xd = torch.empty_like(bd)
    info = h.mf_solve_device(4, bd.data_ptr(), xd.data_ptr())
    torch.cuda.synchronize()
    x = xd.cpu().numpy().T
    assert info.converged == 1
    assert np.linalg.norm(p.to_scipy() @ x - b) / np.linalg.norm(b) <= 1e-8
    xh, _ = h.mf_solve(b)
    assert np.linalg.norm(xh - x) / np.linalg.norm(x) < 1e-9


def test_launch_counter_moves(g):
    p = w.helmholtz7(6, 8)
    h = g.analyze_problem(p, leaf_size=16, nmin_sep=10 ** 9)
    c0 = g.lib().mf_launch_counter()
    h.mf_factor(0.0)
    st = h.mf_stats()
    assert g.lib().mf_launch_counter() - c0 == st["gpu_launches_factor"] > 0
