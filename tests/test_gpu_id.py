"""Batched row interpolative decomposition (Sec. 3) on the GPU against the oracle's ID."""
import numpy as np
import pytest

from oracle.idq import row_id

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2007_00202_gb300 import build
    build.build()
    return torch


def _mats(rng, nmat, m, n, kind):
    out = []
    for q in range(nmat):
        if kind == "lowrank":
            k = 3 + q % 7
            M = (rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))) @ \
                (rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n)))
        else:
            Q1, _ = np.linalg.qr(rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)))
            Q2, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
            r = min(m, n)
            sv = 10.0 ** (-np.arange(r) / (3 + q))
            M = (Q1[:, :r] * sv) @ Q2[:r]
        out.append(M)
    return out


def run_gpu_id(torch, mats, tol, max_rank=0, fn=None):
    import paper_2007_00202_gb300.mf as mf
    nmat = len(mats)
    m, n = mats[0].shape
    kmax = min(m, n) if max_rank <= 0 else min(m, n, max_rank)
    buf = np.concatenate([np.concatenate([M.real.ravel(), M.imag.ravel()]) for M in mats]).astype(np.float32)
    dM = torch.from_numpy(buf).cuda()
    dU = torch.zeros(nmat * 2 * m * kmax, dtype=torch.float32, device="cuda")
    dsk = torch.zeros(nmat * kmax, dtype=torch.int32, device="cuda")
    drk = torch.zeros(nmat, dtype=torch.int32, device="cuda")
    (fn or mf.mf_row_id_c64)(nmat, m, n, dM.data_ptr(), tol, max_rank, dU.data_ptr(), dsk.data_ptr(), drk.data_ptr())
    torch.cuda.synchronize()
    U = dU.cpu().numpy().reshape(nmat, 2, m, kmax)
    sk = dsk.cpu().numpy().reshape(nmat, kmax)
    rk = drk.cpu().numpy()
    res = []
    for q in range(nmat):
        r = int(rk[q])
        res.append(((U[q, 0, :, :r] + 1j * U[q, 1, :, :r]).astype(np.complex128), sk[q, :r].astype(np.int64)))
    return res


# shapes cover the three kernels: rows in registers (m, n <= 128), QR work in shared memory, and
# the thread-block-cluster kernel for work in global memory (incl. fewer rows than cluster CTAs)
@pytest.mark.parametrize("m,n,kind,tol", [(64, 640, "lowrank", 1e-5), (40, 300, "decay", 1e-3),
                                          (128, 1000, "decay", 1e-4), (7, 5, "decay", 1e-2),
                                          (128, 72, "decay", 1e-4), (256, 1024, "decay", 1e-4),
                                          (200, 333, "lowrank", 1e-5), (5, 6000, "lowrank", 1e-5)])
def test_row_id_matches_oracle(tk, m, n, kind, tol):
    rng = np.random.default_rng(m * n)
    mats = _mats(rng, 12, m, n, kind)
    for M, (U, sk) in zip(mats, run_gpu_id(tk, mats, tol)):
        Uo, sko = row_id(M, tol)
        r = len(sk)
        assert abs(r - len(sko)) <= 1                       # rank decision in FP32 vs FP64 near the threshold
        assert np.array_equal(np.abs(U[sk]), np.eye(r))       # identity on the skeleton rows, exactly
        assert len(set(sk.tolist())) == r
        err = np.linalg.norm(M - U @ M[sk], 2) / np.linalg.norm(M, 2)
        erro = np.linalg.norm(M - Uo @ M[sko], 2) / np.linalg.norm(M, 2)
        assert err <= max(10 * tol, 3 * erro) + 1e-5
        if kind == "lowrank":
            assert r == len(sko)


def test_row_id_rank_cap_and_zero_matrix(tk):
    rng = np.random.default_rng(3)
    mats = _mats(rng, 3, 50, 80, "decay")
    out = run_gpu_id(tk, mats, 1e-12, max_rank=8)
    assert all(len(sk) == 8 for _, sk in out)
    z = [np.zeros((10, 20), complex)]
    (U, sk), = run_gpu_id(tk, z, 1e-4)
    assert len(sk) == 0
