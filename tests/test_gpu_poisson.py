"""3D Poisson (Sec. 6.3: the same solver with k = 0) on the GPU compressed path: complex64 HOD-BF
fronts at tol 1e-4, FP64 GMRES to 1e-8, compared with the oracle's exact multifrontal solution."""
import numpy as np
import pytest

import workloads as w

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


def test_poisson_32cube_compressed_gmres_to_1e8(g):
    p = w.helmholtz7(32, 10, damping=0.0, k=0.0)
    b = w.rhs_gaussian(p, 4, 13)
    h = g.analyze_problem(p, nmin_sep=256, max_rank=64, precision=g.MF_PREC_C64, refine=g.MF_REFINE_GMRES)
    h.mf_factor(1e-4)
    st = h.mf_stats()
    assert st["ncompressed"] >= 3 and st["max_rank"] <= 64
    x, info = h.mf_solve(b)
    A = p.to_scipy()
    res = np.linalg.norm(A @ x - b, axis=0) / np.linalg.norm(b, axis=0)
    assert info.converged == 1 and res.max() <= 1e-8
    # the oracle's exact multifrontal solution (Alg. 1, FP64) of the same system
    from oracle.analysis import analyze
    from oracle import dense_mf as dm
    an = analyze(p, 64, 10 ** 9)
    xe = dm.solve(p, an, dm.multifrontal_factor(p, an)[0], b)
    assert np.linalg.norm(A @ xe - b) / np.linalg.norm(b) <= 1e-12
    assert np.linalg.norm(x - xe) / np.linalg.norm(xe) <= 1e-6
