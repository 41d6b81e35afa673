"""GPU butterfly / HOD-BF construction (Alg. 2 on every off-diagonal block, Sec. 4.1)
and the level-by-level apply, on Green's-function blocks, against the dense FP64 product."""
import math

import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2007_00202_gb300 import build
    build.build()
    return torch


def _dense_green(P, Q, k):
    d = P[:, None, :] - Q[None, :, :]
    r = np.sqrt((d * d).sum(-1))
    return np.exp(1j * k * r) / (4 * math.pi * r)


@pytest.mark.parametrize("tol", [1e-2, 1e-4])
def test_green_hodbf_apply_matches_dense(tk, tol):
    import paper_2007_00202_gb300.mf as mf
    torch = tk
    ms = [16, 20, 33]
    k = math.pi / 4
    S = mf.GreenSet(ms, k, 1.0, tol, leaf=32)
    P, Q = S.points()
    nrhs = 8
    rng = np.random.default_rng(7)
    X = w.complex_gaussian(rng, S.rows, nrhs)
    dX = torch.from_numpy(np.concatenate([X.real.ravel(), X.imag.ravel()]).astype(np.float32)).cuda()
    dY = torch.zeros_like(dX)
    S.apply(nrhs, dX.data_ptr(), dY.data_ptr())
    torch.cuda.synchronize()
    Y1 = dY.cpu().numpy()
    for _ in range(3):                       # captured on the second call, replayed on the third and fourth
        dY.zero_()
        S.apply(nrhs, dX.data_ptr(), dY.data_ptr())
    torch.cuda.synchronize()
    assert np.array_equal(dY.cpu().numpy(), Y1)
    Yg = dY.cpu().numpy().astype(np.float64)
    Yg = (Yg[:S.rows * nrhs] + 1j * Yg[S.rows * nrhs:]).reshape(S.rows, nrhs)
    off = 0
    for m in ms:
        n = m * m
        K = _dense_green(P[off:off + n], Q[off:off + n], k)
        ref = K @ X[off:off + n]
        err = np.linalg.norm(Yg[off:off + n] - ref) / np.linalg.norm(ref)
        assert err <= 10 * tol, (m, err)
        off += n
    assert S.storage < sum(m ** 4 for m in ms)      # compressed
    assert 0 < S.max_rank <= 64
