"""The allocation-free row ID entry point against the allocating one.

mf_row_id_c64_noalloc serves callers that cannot allocate device memory when
they need the decomposition (applications whose pool allocator owns all of the
GPU's memory, or loops that must not call cudaMalloc / cudaFree because those
can synchronize the device); it keeps its QR work matrix in a fixed array
inside the library.
This file is collected last so that a failure here comes after every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2007_00202_gb300 import build
    build.build()
    return torch


def _batch(rng, nmat, m, n):
    out = []
    for q in range(nmat):
        k = 4 + q
        A = (rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))) @ \
            (rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n)))
        A += 1e-3 * (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n)))
        out.append(A)
    return out


def _run(torch, fn, mats, tol, max_rank=0):
    nmat = len(mats)
    m, n = mats[0].shape
    kmax = min(m, n) if max_rank <= 0 else min(m, n, max_rank)
    buf = np.concatenate([np.concatenate([M.real.ravel(), M.imag.ravel()]) for M in mats]).astype(np.float32)
    dM = torch.from_numpy(buf).cuda()
    dU = torch.full((nmat * 2 * m * kmax,), float("nan"), dtype=torch.float32, device="cuda")
    dsk = torch.full((nmat * kmax,), -1, dtype=torch.int32, device="cuda")
    drk = torch.full((nmat,), -1, dtype=torch.int32, device="cuda")
    fn(nmat, m, n, dM.data_ptr(), tol, max_rank, dU.data_ptr(), dsk.data_ptr(), drk.data_ptr(),
       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    U = dU.cpu().numpy().reshape(nmat, 2, m, kmax)
    sk = dsk.cpu().numpy().reshape(nmat, kmax)
    rk = drk.cpu().numpy()
    return [(U[q, 0, :, :rk[q]] + 1j * U[q, 1, :, :rk[q]], sk[q, :rk[q]].copy()) for q in range(nmat)]


def test_noalloc_row_id_matches_allocating_call_twice_in_a_row(tk):
    import paper_2007_00202_gb300.mf as mf
    rng = np.random.default_rng(2024)
    for call in range(2):                       # the shared scratch keeps the previous call's contents
        m, n = (96, 700) if call == 0 else (64, 300)
        mats = _batch(rng, 10, m, n)
        ref = _run(tk, mf.mf_row_id_c64, mats, 1e-4)
        got = _run(tk, mf.mf_row_id_c64_noalloc, mats, 1e-4)
        for M, (Ur, skr), (Ug, skg) in zip(mats, ref, got):
            assert len(skg) == len(skr) and np.array_equal(skg, skr)
            assert np.abs(Ug - Ur).max() <= 1e-5 * max(1.0, np.abs(Ur).max())
            err = np.linalg.norm(M - Ug @ M[skg], 2) / np.linalg.norm(M, 2)
            assert err <= 1e-3


def test_cluster_row_id_equals_the_single_cta_body(tk):
    # large blocks: the allocating call runs one thread-block cluster per matrix, the
    # allocation-free one a single CTA with the same per-row arithmetic; skeletons agree exactly
    import paper_2007_00202_gb300.mf as mf
    rng = np.random.default_rng(77)
    for m, n in ((256, 1024), (13, 4000)):
        mats = _batch(rng, 3, m, n)
        ref = _run(tk, mf.mf_row_id_c64, mats, 1e-4, max_rank=64)
        got = _run(tk, mf.mf_row_id_c64_noalloc, mats, 1e-4, max_rank=64)
        for (Ur, skr), (Ug, skg) in zip(ref, got):
            assert np.array_equal(skg, skr)
            assert np.array_equal(Ug, Ur)


def test_noalloc_rejects_batches_beyond_the_fixed_scratch(tk):
    import paper_2007_00202_gb300.mf as mf
    with pytest.raises(mf.MfError) as e:
        mf.mf_row_id_c64_noalloc(40, 256, 256, 1, 1e-4, 0, 1, 1, 1, 0)   # 2*256*256*40 floats > 2^21
    assert e.value.code == -1
