"""Serving: continuous batching over resident factorizations.  Each result must be
the same alone and in the mix (both at the 1e-8 residual, and close to each other)."""
import threading
import time

import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2007_00202_gb300 import build
    build.build()
    import paper_2007_00202_gb300 as g
    probs = [w.helmholtz7(12, 8), w.helmholtz7(16, 8)]
    streams = [torch.cuda.Stream() for _ in probs]
    hs = []
    for p, s in zip(probs, streams):
        h = g.analyze_problem(p, nmin_sep=128, leaf_size=64, stream=s.cuda_stream)
        h.mf_factor(1e-4)
        hs.append(h)
    return g, probs, hs, streams


def test_results_same_alone_and_in_the_mix(env):
    g, probs, hs, streams = env
    import paper_2007_00202_gb300.mf as mf
    rng = np.random.default_rng(5)
    reqs = []
    for r in range(24):
        pi = int(rng.integers(len(probs)))
        nrhs = int(rng.integers(1, 6))
        reqs.append((pi, w.complex_gaussian(rng, probs[pi].n, nrhs)))
    alone, alone_info = [], []
    for pi, b in reqs:
        x, info = hs[pi].mf_solve(b)
        alone.append(x)
        alone_info.append((int(info.converged), int(info.iters)))
    srv = mf.Server(hs, max_batch_rhs=32, mem_budget_bytes=8 << 30)
    ids = [None] * len(reqs)

    def client(lo, hi):
        for k in range(lo, hi):
            ids[k] = srv.submit(reqs[k][0], reqs[k][1])
            time.sleep(0.001)

    th = [threading.Thread(target=client, args=(a, a + 8)) for a in (0, 8, 16)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    out = [srv.wait(i) for i in ids]
    srv.close()
    batched = 0
    for (pi, b), xa, (conv_a, its_a), (xm, info) in zip(reqs, alone, alone_info, out):
        A = probs[pi].to_scipy()
        for x in (xa, xm):
            assert np.max(np.linalg.norm(A @ x - b, axis=0) / np.linalg.norm(b, axis=0)) <= 1e-8
        assert np.linalg.norm(xm - xa) / np.linalg.norm(xa) <= 1e-6
        # what a request reports is its own: status, converged flag and iterations as when alone
        assert info["status"] == 0 and info["converged"] == conv_a == 1
        assert abs(info["iters"] - its_a) <= 1
        rel = np.max(np.linalg.norm(A @ xm - b, axis=0) / np.linalg.norm(b, axis=0))
        assert info["max_rel_residual"] <= 1e-8 and abs(info["max_rel_residual"] - rel) <= 1e-9
        assert info["t_done"] >= info["t_start"] >= info["t_arrival"]
        batched += info["batch_rhs"] > info["nrhs"]
    assert batched > 0          # some requests shared a batch with others


def test_admission_rejects_oversized_request(env):
    g, probs, hs, streams = env
    import paper_2007_00202_gb300.mf as mf
    srv = mf.Server(hs[:1], max_batch_rhs=8, mem_budget_bytes=1 << 20)
    with pytest.raises(mf.MfError) as e:
        srv.submit(0, np.ones((probs[0].n, 4), complex))
    assert e.value.code == -4
    srv.close()


def test_request_status_does_not_depend_on_its_batch(env):
    # a handle capped at one Krylov iteration: Gaussian right-hand sides stop above rtol, a zero
    # right-hand side is solved exactly (x = 0); batched together, each keeps its own status
    g, probs, hs, streams = env
    import paper_2007_00202_gb300.mf as mf
    p = probs[0]
    h = g.analyze_problem(p, nmin_sep=128, leaf_size=64, max_iters=1, stream=streams[0].cuda_stream)
    h.mf_factor(1e-4)
    rng = np.random.default_rng(9)
    bad = w.complex_gaussian(rng, p.n, 2)
    zero = np.zeros((p.n, 1), complex)
    x, info = h.mf_solve(np.concatenate([bad, zero], axis=1), allow_no_convergence=True)
    cols = h.mf_solve_columns(3)
    assert list(cols["converged"]) == [0, 0, 1] and cols["rel_residual"][2] == 0.0
    assert np.all(cols["iters"][:2] == 1) and cols["iters"][2] == 0
    srv = mf.Server([h], max_batch_rhs=8, mem_budget_bytes=8 << 30)
    ids = [srv.submit(0, bad), srv.submit(0, zero)]
    (xb, ib), (xz, iz) = srv.wait(ids[0]), srv.wait(ids[1])
    srv.close()
    assert ib["status"] == -6 and ib["converged"] == 0
    assert iz["status"] == 0 and iz["converged"] == 1 and np.all(xz == 0)


def test_wide_request_runs_in_slices_like_alone(env):
    # a request wider than the batch limit runs alone, in slices of max_batch_rhs columns; its
    # columns are independent, so its solution, status and per-column results match one solve
    g, probs, hs, streams = env
    import paper_2007_00202_gb300.mf as mf
    p = probs[1]
    rng = np.random.default_rng(17)
    b = w.complex_gaussian(rng, p.n, 11)
    xa, ia = hs[1].mf_solve(b)
    srv = mf.Server(hs, max_batch_rhs=4, mem_budget_bytes=8 << 30)
    x, info = srv.wait(srv.submit(1, b))
    srv.close()
    A = p.to_scipy()
    res = np.linalg.norm(A @ x - b, axis=0) / np.linalg.norm(b, axis=0)
    assert info["status"] == 0 and info["converged"] == 1 and info["batch_rhs"] == 11
    assert res.max() <= 1e-8 and abs(info["max_rel_residual"] - res.max()) <= 1e-9
    assert np.linalg.norm(x - xa) / np.linalg.norm(xa) <= 1e-6

