"""bench.py's roofline objects on CPU: arithmetic from the event profile, the ALU / HBM bound
chosen by arithmetic intensity against the FP32-ALU / HBM ridge, and the DRAM-traffic figure
reported only while the narrow GEMM's source is the one the ncu capture measured."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6756.5, "bf16_tflops": 1899.9}


def test_narrow_gemm_alu_bound_arithmetic():
    # 16 right-hand sides: 8 m n k flop over 8 (m k + ...) bytes, about 16 flop/byte > ridge 11.9
    prof = {"launches": 10, "ms": 2.0, "flops": 8.0 * 4096 * 16 * 4096 * 10, "bytes": 1.358e8 * 10}
    r = bench.roofline(prof, PEAKS)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(prof["flops"] / 2e-3 / 1e12)
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["hbm_frac"] == pytest.approx(prof["bytes"] / 2e-3 / 1e9 / 6756.5)
    assert r["ms_per_launch"] == pytest.approx(0.2)
    matches = bench._device_code_sha1("gemm_nrhs.cu", "launch_nb") == bench.NARROW_SRC_SHA1
    if matches:
        assert r["traffic"] == pytest.approx(bench.NARROW_TRAFFIC_PER_ALG_BYTE * prof["bytes"] / 10)
    else:
        assert r["traffic"] is None


def test_traffic_hash_covers_the_device_code_only():
    # the counters stay valid across edits of the host launch code and lapse with any edit of the
    # kernels: the hash covers the source up to the first host launch function
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2007_00202_gb300", "csrc", "gemm_nrhs.cu")
    text = open(path).read()
    i = text.index("void launch_nb(")
    cut = text.rfind("\ntemplate", 0, i)
    assert 0 < cut < i
    assert "__global__" in text[:cut] and "__global__" not in text[cut:]


def test_narrow_gemm_hbm_bound_below_the_ridge():
    # one right-hand side: about 1 flop/byte, far below the ridge
    prof = {"launches": 4, "ms": 1.0, "flops": 1.0e9, "bytes": 1.0e9}
    r = bench.roofline(prof, PEAKS)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(1e9 / 1e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6756.5)


def test_front_gemm_tensor_roofline_and_empty_profiles():
    prof = {"launches": 3, "ms": 10.0, "flops": 1.0e12, "bytes": 0.0}
    r = bench.roofline_front(prof, PEAKS)
    assert r["bound"] == "tensor" and r["achieved"] == pytest.approx(100.0)
    # TF32 ceiling: measured bf16 x 1.1 / 2.25 (nominal dense TF32 : bf16 of a GB300)
    assert r["peak"] == pytest.approx(1899.9 * 1.1 / 2.25)
    assert r["achieved_tensor_passes"] == pytest.approx(300.0) and r["frac"] == pytest.approx(100.0 / r["peak"])
    assert bench.roofline({"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0}, PEAKS) is None
    assert bench.roofline_front(None, PEAKS) is None


def test_clock_summary_reports_median_max_and_active_reasons(tmp_path):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    rows = ["0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    open(c.path, "w").write("\n".join(rows) + "\n")
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
