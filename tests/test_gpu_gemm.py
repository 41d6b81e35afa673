"""Front-update GEMM kernels (Sec. 2 step 4: C = F22 - F21 F12) against an FP64 product."""
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


def _planar(torch, M, ld):
    rows, cols = M.shape
    buf = torch.zeros(2, rows, ld, dtype=torch.float32, device="cuda")
    buf[0, :, :cols] = torch.from_numpy(M.real.astype(np.float32))
    buf[1, :, :cols] = torch.from_numpy(M.imag.astype(np.float32))
    return buf


@pytest.mark.parametrize("engine", [0, 1, 2])
@pytest.mark.parametrize("m,n,k,beta", [(300, 257, 100, 1.0), (128, 128, 32, 0.0), (1, 5, 3, 1.0),
                                        (520, 390, 961, 1.0)])
def test_gemm_nt_against_fp64(tk, engine, m, n, k, beta):
    import paper_2007_00202_gb300.mf as mf
    torch = tk
    rng = np.random.default_rng(m + n + k)
    A = rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))
    B = rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))
    C0 = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    lda = (k + 3) // 4 * 4
    ldc = n + 3
    dA, dB, dC = _planar(torch, A, lda), _planar(torch, B, lda), _planar(torch, C0, ldc)
    mf.mf_gemm_c64(engine, m, n, k, dA.data_ptr(), lda, m * lda, dB.data_ptr(), lda, n * lda, dC.data_ptr(), ldc,
                   m * ldc, -1.0, beta, 0)
    torch.cuda.synchronize()
    out = dC[0, :, :n].double().cpu().numpy() + 1j * dC[1, :, :n].double().cpu().numpy()
    ref = -(A @ B.T) + beta * C0
    scale = np.sqrt(k) * np.abs(A).max() * np.abs(B).max()
    err = np.abs(out - ref).max() / scale
    # FP32 SIMT: ~1e-6; one TF32 pass (10-bit mantissa inputs, FP32 accumulate): ~1e-3;
    # split TF32 (three passes): FP32-like
    assert err < {0: 2e-5, 1: 4e-3, 2: 2e-5}[engine], err
    # the padding column of C (beyond n) is untouched
    assert float(dC[0, :, n:].abs().max()) == float(_planar(torch, C0, ldc)[0, :, n:].abs().max())


@pytest.mark.parametrize("trans_a", [0, 1])
@pytest.mark.parametrize("m,n,k,beta,ksplit", [(3072, 16, 3072, 0.0, 0), (40, 16, 2000, 1.0, 0), (70, 3, 33, 1.0, 0),
                                               (1, 1, 1, 0.0, 1), (300, 64, 129, 1.0, 2), (129, 33, 500, 1.0, 8),
                                               (64, 17, 100, 0.0, 4), (200, 72, 300, 1.0, 0),
                                               (33, 128, 64, 0.0, 2)])
def test_gemm_nrhs_against_fp64(tk, trans_a, m, n, k, beta, ksplit):
    # the solve's narrow products: C = -op(A) B + beta C, n <= 128 (column tiles), K split over a cluster
    import paper_2007_00202_gb300.mf as mf
    torch = tk
    rng = np.random.default_rng(7 * m + n + k + trans_a)
    A = rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))
    B = rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))
    C0 = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    As = A.T.copy() if trans_a else A            # stored k x m when transposed
    lda = As.shape[1] + 1
    ldb, ldc = n + 2, n + 1
    dA, dB, dC = _planar(torch, As, lda), _planar(torch, B, ldb), _planar(torch, C0, ldc)
    mf.mf_gemm_nrhs_c64(trans_a, m, n, k, dA.data_ptr(), lda, As.shape[0] * lda, dB.data_ptr(), ldb, k * ldb,
                        dC.data_ptr(), ldc, m * ldc, -1.0, beta, ksplit, 0)
    torch.cuda.synchronize()
    out = dC[0, :, :n].double().cpu().numpy() + 1j * dC[1, :, :n].double().cpu().numpy()
    ref = -(A @ B) + beta * C0
    scale = np.sqrt(k) * np.abs(A).max() * np.abs(B).max()
    assert np.abs(out - ref).max() / scale < 2e-5
    assert float(dC[0, :, n:].abs().max()) == float(_planar(torch, C0, ldc)[0, :, n:].abs().max())


@pytest.mark.parametrize("trans_a", [0, 1])
@pytest.mark.parametrize("m,n,k,beta", [(1, 1, 1, 0.0), (5, 64, 7, 1.0), (40, 64, 80, 0.0), (100, 64, 37, 1.0),
                                        (128, 64, 16, 0.0), (129, 64, 33, 1.0), (300, 16, 260, 1.0),
                                        (77, 3, 1000, 0.0), (600, 64, 64, 1.0)])
def test_gemm_nrhs_tensor_core_against_fp64(tk, trans_a, m, n, k, beta):
    # the tcgen05 narrow kernel (ksplit = -1): transposed products with the 64 vectors on the MMA's
    # M dimension, split TF32; ragged m, n, k (partial 128-row tiles, partial 16-wide K chunks)
    import paper_2007_00202_gb300.mf as mf
    torch = tk
    rng = np.random.default_rng(11 * m + n + 3 * k + trans_a)
    A = rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))
    B = rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))
    C0 = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    As = A.T.copy() if trans_a else A
    lda = As.shape[1] + 1
    ldb, ldc = n + 2, n + 1
    dA, dB, dC = _planar(torch, As, lda), _planar(torch, B, ldb), _planar(torch, C0, ldc)
    mf.mf_gemm_nrhs_c64(trans_a, m, n, k, dA.data_ptr(), lda, As.shape[0] * lda, dB.data_ptr(), ldb, k * ldb,
                        dC.data_ptr(), ldc, m * ldc, -1.0, beta, -1, 0)
    torch.cuda.synchronize()
    out = dC[0, :, :n].double().cpu().numpy() + 1j * dC[1, :, :n].double().cpu().numpy()
    ref = -(A @ B) + beta * C0
    scale = np.sqrt(k) * np.abs(A).max() * np.abs(B).max()
    assert np.abs(out - ref).max() / scale < 2e-5
    assert float(dC[0, :, n:].abs().max()) == float(_planar(torch, C0, ldc)[0, :, n:].abs().max())
