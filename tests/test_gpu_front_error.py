"""Per-front compression error of the GPU factorization (Alg. 5) against the oracle.

Every compressed front's operators are read back through mf_front_apply (applied to an
identity block) and compared with the same blocks assembled densely by the oracle's exact
multifrontal elimination in the same ordering (Alg. 1): F11, F12, F21 of the front
F = A-part (+) C_nu1 (+) C_nu2 and its contribution block C = F22 - F21 F11^-1 F12.  The
bound is the relative Frobenius error 10 tol for every front (the ID tolerance of Sec. 6.1
with a factor 10 allowance for the products of several IDs; the children's own compression
errors are inside it, since a compressed front is assembled from compressed children).
"""
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


def _exact_fronts(p, an):
    """Dense F (assembled, before elimination) and exact contribution block of every front."""
    Ap = dm.permuted_matrix(p, an)
    cbs, out = {}, {}
    for f in an.fronts:
        F = dm.assemble_sparse(Ap, f)
        for c in f.children:
            rel = dm.relative_map(an.fronts[c], f)
            F[np.ix_(rel, rel)] += cbs.pop(c)
        s = f.s
        C = F[s:, s:] - F[s:, :s] @ np.linalg.solve(F[:s, :s], F[:s, s:]) if f.u else None
        if f.compressed:
            out[f.id] = (F.copy(), C)
        if f.parent >= 0:
            cbs[f.id] = C
    return out


def _rel(A, B):
    return float(np.linalg.norm(A - B) / np.linalg.norm(B))


@pytest.mark.parametrize("grid,ppw,nmin,tol,prec", [
    (16, 8, 128, 1e-6, "c128"),      # the 16^3 workload: complex128, tol 1e-6
    (20, 10, 128, 1e-4, "c64"),      # complex64 factors at the production tolerance
])
def test_every_compressed_front_within_10_tol(g, grid, ppw, nmin, tol, prec):
    import paper_2007_00202_gb300.mf as mf
    p = w.helmholtz7(grid, ppw)
    precision = g.MF_PREC_C128 if prec == "c128" else g.MF_PREC_C64
    h = g.analyze_problem(p, leaf_size=64, nmin_sep=nmin, hodbf_leaf=64, precision=precision,
                          refine=g.MF_REFINE_NONE)
    h.mf_factor(tol)
    an = analyze(p, 64, nmin, 64)
    ex = h.mf_analysis_export()
    assert np.array_equal(ex["compressed"], np.array([f.compressed for f in an.fronts]))
    ref = _exact_fronts(p, an)
    assert len(ref) >= 2
    worst = {}
    for fid, (F, C) in ref.items():
        f = an.fronts[fid]
        s, u = f.s, f.u
        Is = np.eye(s, dtype=complex)
        errs = {"F11": _rel(h.mf_front_apply(fid, mf.MF_OP_F11, Is, s), F[:s, :s])}
        inv = np.linalg.inv(F[:s, :s])
        errs["F11inv"] = _rel(h.mf_front_apply(fid, mf.MF_OP_F11_INV, Is, s), inv)
        if u:
            Iu = np.eye(u, dtype=complex)
            errs["F12"] = _rel(h.mf_front_apply(fid, mf.MF_OP_F12, Iu, s), F[:s, s:])
            errs["F21"] = _rel(h.mf_front_apply(fid, mf.MF_OP_F21, Is, u), F[s:, :s])
            if f.parent >= 0:
                errs["C"] = _rel(h.mf_front_apply(fid, mf.MF_OP_C, Iu, u), C)
        for k, e in errs.items():
            worst[k] = max(worst.get(k, 0.0), e)
        for k in ("F11", "F12", "F21", "C"):
            if k in errs:
                assert errs[k] <= 10 * tol, (fid, s, u, k, errs)
        # the inverse carries the condition number of F11 (Alg. 4 inverts the compressed F11)
        assert errs["F11inv"] <= 10 * tol * np.linalg.cond(F[:s, :s]), (fid, errs)
    print(grid, prec, tol, {k: f"{v:.1e}" for k, v in worst.items()})


def test_front_apply_rejects_dense_fronts(g):
    import paper_2007_00202_gb300.mf as mf
    p = w.helmholtz7(12, 8)
    h = g.analyze_problem(p, leaf_size=32, nmin_sep=64, hodbf_leaf=32, max_rank=32)
    h.mf_factor(1e-4)
    ex = h.mf_analysis_export()
    dense = int(np.flatnonzero(~ex["compressed"])[0])
    with pytest.raises(mf.MfError):
        h.mf_front_apply(dense, mf.MF_OP_F11, np.eye(4, dtype=complex), 4)
