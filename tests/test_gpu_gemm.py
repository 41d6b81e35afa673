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
    # relative Frobenius error: SIMT FP32 ~1e-6; split TF32 ~1e-5 (measured 1.4e-5 at k = 961: the
    # tensor core's accumulation, not the split, sets this floor); one TF32 pass ~3e-4
    rel = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert rel < {0: 1e-5, 1: 2e-3, 2: 5e-5}[engine], rel
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
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 5e-5     # split TF32 (one TF32 pass: ~3e-4)
    assert float(dC[0, :, n:].abs().max()) == float(_planar(torch, C0, ldc)[0, :, n:].abs().max())


def test_split_tf32_passes_recover_fp32_accuracy(tk):
    # the split product (hi*hi + hi*lo + lo*hi) must be clearly more accurate than one TF32 pass on the
    # same operands (a split whose lo parts were lost would match the one-pass error, ~3e-4); its own
    # floor, ~1e-5, is the tensor core's accumulation
    import paper_2007_00202_gb300.mf as mf
    torch = tk
    rng = np.random.default_rng(5)
    m, n, k = 512, 384, 2048
    A = rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))
    B = rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))
    dA, dB = _planar(torch, A, k), _planar(torch, B, k)
    ref = A @ B.T
    errs = {}
    for engine in (1, 2):
        dC = torch.zeros(2, m, n, dtype=torch.float32, device="cuda")
        mf.mf_gemm_c64(engine, m, n, k, dA.data_ptr(), k, m * k, dB.data_ptr(), k, n * k, dC.data_ptr(), n, m * n,
                       1.0, 0.0, 0)
        torch.cuda.synchronize()
        out = dC[0].double().cpu().numpy() + 1j * dC[1].double().cpu().numpy()
        errs[engine] = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert errs[2] < 5e-5 and errs[2] < errs[1] / 8, errs
    # the narrow tensor-core kernel on the same A (first 64 columns of B^T as the block of vectors)
    Bn = B[:64].T.copy()
    dBn = _planar(torch, Bn, 64)
    dC = torch.zeros(2, m, 64, dtype=torch.float32, device="cuda")
    mf.mf_gemm_nrhs_c64(0, m, 64, k, dA.data_ptr(), k, m * k, dBn.data_ptr(), 64, k * 64, dC.data_ptr(), 64, m * 64,
                        1.0, 0.0, -1, 0)
    torch.cuda.synchronize()
    out = dC[0].double().cpu().numpy() + 1j * dC[1].double().cpu().numpy()
    refn = A @ Bn
    assert np.linalg.norm(out - refn) / np.linalg.norm(refn) < 5e-5


def test_expired_waits_return_timeout_and_the_context_stays_usable(tk):
    # failure detection without a fault: with a one-poll limit the bounded mbarrier waits of the
    # tensor-core kernels expire while their MMAs are still running; the kernel records the
    # expiry, drains its committed MMAs, frees its tensor memory and the call returns
    # MF_ERR_TIMEOUT.  The kernels are deterministic, so every attempt either times out or returns
    # exactly the bits of a run with the default limit; afterwards the default limit gives those
    # bits again on the same context.
    import paper_2007_00202_gb300.mf as mf
    torch = tk
    MF_ERR_TIMEOUT = -7
    rng = np.random.default_rng(99)
    m, n, k = 1024, 1024, 4096
    A = rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))
    B = rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))
    dA, dB = _planar(torch, A, k), _planar(torch, B, k)
    mn, kn = 96 * 304 * 3, 16                 # tensor-core narrow kernel: many one-chunk tiles per CTA
    An = rng.standard_normal((mn, kn)) + 1j * rng.standard_normal((mn, kn))
    Bn = rng.standard_normal((kn, 64)) + 1j * rng.standard_normal((kn, 64))
    dAn, dBn = _planar(torch, An, kn), _planar(torch, Bn, 64)

    def front():
        dC = torch.zeros(2, m, n, dtype=torch.float32, device="cuda")
        mf.mf_gemm_c64(2, m, n, k, dA.data_ptr(), k, m * k, dB.data_ptr(), k, n * k, dC.data_ptr(), n, m * n,
                       -1.0, 0.0, 0)
        torch.cuda.synchronize()
        return dC.cpu().numpy()

    def narrow():
        dC = torch.zeros(2, mn, 64, dtype=torch.float32, device="cuda")
        mf.mf_gemm_nrhs_c64(0, mn, 64, kn, dAn.data_ptr(), kn, mn * kn, dBn.data_ptr(), 64, kn * 64,
                            dC.data_ptr(), 64, mn * 64, -1.0, 0.0, -1, 0)
        torch.cuda.synchronize()
        return dC.cpu().numpy()

    for call, ref in ((front, -(A @ B.T)), (narrow, -(An @ Bn))):
        base = call()                          # default limit
        got = base[0].astype(np.float64) + 1j * base[1].astype(np.float64)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-4
        timeouts = 0
        mf.mf_set_wait_limit(1)
        try:
            for attempt in range(6):
                try:
                    out = call()
                    assert np.array_equal(out, base)
                except mf.MfError as e:
                    assert e.code == MF_ERR_TIMEOUT, e
                    timeouts += 1
        finally:
            mf.mf_set_wait_limit(0)
        assert timeouts >= 1, call.__name__
        assert np.array_equal(call(), base)
