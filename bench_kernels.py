"""Microbenchmarks of the library's hot kernels through their C-ABI component entry points,
and single-phase runs of the 64^3 workload for profilers.

    python bench_kernels.py [narrow|front|rowid|factor|solve] [--reps R] [--grid G]

narrow: the narrow GEMM of the solve (mf_gemm_nrhs_c64), C = -A B + C with A 4096 x 4096,
        B 4096 x 16 (complex64): one launch streams 128 MiB of A (larger than L2).
front:  the split-TF32 tcgen05 front GEMM (mf_gemm_c64 engine 2), 4096 x 4096 x 4096.
rowid:  the batched row ID (mf_row_id_c64) of 256 matrices of 128 x 72 (the randomized
        construction's sketch blocks); rowid_big: 8 matrices of 256 x 1024 (the entry
        evaluation's large proxy blocks, one thread-block cluster each).
factor: the compressed complex64 factorization of the bench workload (helmholtz7 G^3, ppw 10,
        separators >= 1024 HOD-BF at tol 1e-4, rank <= 64), once to warm up, then once between
        cudaProfilerStart/Stop (for `ncu --profile-from-start off`).
solve:  after that factorization, one preconditioner application to 16 right-hand sides
        (no refinement) between cudaProfilerStart/Stop, after three warm-up solves.
bfapply: the batched butterfly apply of `--blocks` Green's-function HOD-BF blocks (the first
        blocks of the 200-block workload, m = rint(16 * 8^u), seed 3; tol 1e-4) to 64 vectors,
        after three warm-up applies; the timed applies run between cudaProfilerStart/Stop.
peaks:  roofline denominators with library GEMMs (torch.matmul / cuBLAS): 8192^3 fp32 with
        TF32 off and on, bf16 and fp64, 4096^3 complex64, and a 1 GiB device copy.
Prints one JSON line per item: device time per call (CUDA events, after warm-up; the
component entry points include their own synchronisation) and the achieved rate against the
peaks used by bench.py.
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def _time(torch, fn, reps):
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def narrow(torch, mf, reps, m=4096, k=4096, n=16):
    g = torch.Generator(device="cuda").manual_seed(1)
    A = torch.randn(2, m, k, device="cuda", generator=g)
    B = torch.randn(2, k, n, device="cuda", generator=g)
    C = torch.randn(2, m, n, device="cuda", generator=g)
    st = torch.cuda.current_stream().cuda_stream

    def run():
        mf.mf_gemm_nrhs_c64(0, m, n, k, A.data_ptr(), k, m * k, B.data_ptr(), n, k * n, C.data_ptr(), n, m * n,
                            -1.0, 1.0, 0, st)
    ms = _time(torch, run, reps)
    flops = 8.0 * m * n * k
    by = 8.0 * (m * k + k * n + 2 * m * n)
    hbm = _peaks().get("hbm_gbs", 6800.0)
    return {"kernel": "k_gemm_nrhs", "shape": [m, n, k], "ms": ms, "tflops": flops / ms / 1e9,
            "alu_frac": flops / ms / 1e9 / FP32_ALU_TFLOPS, "gbs": by / ms / 1e6, "hbm_frac": by / ms / 1e6 / hbm,
            "alg_bytes": by}


def front(torch, mf, reps, m=4096, n=4096, k=4096):
    g = torch.Generator(device="cuda").manual_seed(2)
    A = torch.randn(2, m, k, device="cuda", generator=g)
    B = torch.randn(2, n, k, device="cuda", generator=g)
    C = torch.zeros(2, m, n, device="cuda")
    st = torch.cuda.current_stream().cuda_stream

    def run():
        mf.mf_gemm_c64(2, m, n, k, A.data_ptr(), k, m * k, B.data_ptr(), k, n * k, C.data_ptr(), n, m * n,
                       -1.0, 0.0, st)
    ms = _time(torch, run, reps)
    flops = 8.0 * m * n * k
    return {"kernel": "k_gemm_tc<1> (split TF32, 3 passes)", "shape": [m, n, k], "ms": ms,
            "tflops": flops / ms / 1e9, "tensor_tflops": 3 * flops / ms / 1e9,
            "tf32_frac": 3 * flops / ms / 1e9 / 999.0}


def rowid_big(torch, mf, reps):
    """The large-block row ID (8 matrices of 256 x 1024, rank <= 64): a thread-block cluster each."""
    r = rowid(torch, mf, reps, nmat=8, m=256, n=1024)
    r["kernel"] = "k_row_id_cluster"
    return r


def rowid(torch, mf, reps, nmat=256, m=128, n=72):
    g = torch.Generator(device="cuda").manual_seed(3)
    M = torch.randn(nmat, 2, m, n, device="cuda", generator=g)
    kmax = min(m, n)
    U = torch.zeros(nmat, 2, m, kmax, device="cuda")
    sk = torch.zeros(nmat, kmax, dtype=torch.int32, device="cuda")
    rk = torch.zeros(nmat, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream

    def run():
        mf.mf_row_id_c64(nmat, m, n, M.data_ptr(), 1e-4, 64, U.data_ptr(), sk.data_ptr(), rk.data_ptr(), st)
    ms = _time(torch, run, reps)
    return {"kernel": "k_row_id", "shape": [nmat, m, n], "ms": ms, "us_per_matrix": ms * 1e3 / nmat}


def _workload(torch, grid, nmin=1024):
    import workloads as w
    import paper_2007_00202_gb300 as g
    p = w.helmholtz7(grid, 10)
    h = g.analyze_problem(p, nmin_sep=nmin, max_rank=64, precision=g.MF_PREC_C64, refine=g.MF_REFINE_NONE)
    return g, p, h


def extend_add_bytes(h):
    """Algorithmic bytes of each extend-add launch of the dense levels, in launch order (deepest
    level first, first then second child): sum of u_child^2 x 24 B (read the child's complex64
    entry, read and write the parent's)."""
    ex = h.mf_analysis_export()
    nf = len(ex["parent"])
    u = np.diff(ex["upd_ptr"])
    depth = np.zeros(nf, np.int64)
    for f in range(nf - 1, -1, -1):
        if ex["parent"][f] >= 0:
            depth[f] = depth[ex["parent"][f]] + 1
    slot = {}
    seen = {}
    for f in range(nf):
        par = int(ex["parent"][f])
        if par < 0:
            continue
        k = seen.get(par, 0)
        seen[par] = k + 1
        key = (int(depth[par]), k)
        slot[key] = slot.get(key, 0) + int(u[f]) ** 2
    order = sorted(slot, key=lambda t: (-t[0], t[1]))
    return [(d, k, 24.0 * slot[(d, k)]) for d, k in order]


def factor(torch, mf, reps, grid=64, nmin=1024):
    import time
    g, p, h = _workload(torch, grid, nmin)
    h.mf_factor(1e-4)
    torch.cuda.synchronize()
    c0 = g.lib().mf_launch_counter()
    torch.cuda.profiler.start()
    t0 = time.perf_counter()
    h.mf_factor(1e-4)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    torch.cuda.profiler.stop()
    return {"item": "factorization", "grid": grid, "nmin_sep": nmin, "s": dt,
            "launches": g.lib().mf_launch_counter() - c0,
            "extend_add_bytes_per_launch": extend_add_bytes(h)[:4]}


def solve(torch, mf, reps, grid=64):
    import time
    import workloads as w
    g, p, h = _workload(torch, grid)
    h.mf_factor(1e-4)
    b = w.rhs_gaussian(p, 16, 7)
    bd = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()
    xd = torch.empty_like(bd)
    for _ in range(3):
        h.mf_solve_device(16, bd.data_ptr(), xd.data_ptr(), allow_no_convergence=True)
    torch.cuda.synchronize()
    c0 = g.lib().mf_launch_counter()
    torch.cuda.profiler.start()
    t0 = time.perf_counter()
    h.mf_solve_device(16, bd.data_ptr(), xd.data_ptr(), allow_no_convergence=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    torch.cuda.profiler.stop()
    return {"item": "preconditioner application, 16 RHS", "grid": grid, "ms": dt * 1e3,
            "launches": g.lib().mf_launch_counter() - c0}


def bfapply(torch, mf, reps, blocks=200, nrhs=64):
    import math
    import workloads as w
    ms_ = w.butterfly_bench_sizes(200, 3)[:blocks]
    S = mf.GreenSet([int(m) for m in ms_], math.pi / 4, 1.0, 1e-4, leaf=64,
                    stream=torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(8)
    X = w.complex_gaussian(rng, S.rows, nrhs)
    dX = torch.from_numpy(np.concatenate([X.real.ravel(), X.imag.ravel()]).astype(np.float32)).cuda()
    dY = torch.zeros_like(dX)
    for _ in range(3):
        S.apply(nrhs, dX.data_ptr(), dY.data_ptr())
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    ms = _time(torch, lambda: S.apply(nrhs, dX.data_ptr(), dY.data_ptr()), reps)
    torch.cuda.profiler.stop()
    by = 8.0 * S.storage + 2.0 * 8.0 * S.rows * nrhs
    fl, lb = S.apply_counts(nrhs)
    hbm = _peaks().get("hbm_gbs", 6800.0)
    return {"item": "butterfly apply", "blocks": blocks, "rows": S.rows, "stored_entries": S.storage,
            "nrhs": nrhs, "ms": ms, "alg_bytes": by, "gbs": by / ms / 1e6, "hbm_frac": by / ms / 1e6 / hbm,
            "level_traffic_bytes": lb, "level_traffic_gbs": lb / ms / 1e6, "tflops": fl / ms / 1e9}


def peaks(torch, mf, reps):
    out = {"item": "library peaks (cuBLAS through torch.matmul; device copy)"}

    def mm(dtype, n, tf32=False):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device="cuda").to(dtype)
        b = torch.randn(n, n, device="cuda").to(dtype)
        ms = min(_time(torch, lambda: torch.matmul(a, b), 3) for _ in range(max(1, reps // 3)))
        torch.backends.cuda.matmul.allow_tf32 = False
        return (8.0 if dtype.is_complex else 2.0) * n ** 3 / ms / 1e9
    out["fp32_tflops"] = mm(torch.float32, 8192)
    out["tf32_tflops"] = mm(torch.float32, 8192, tf32=True)
    out["bf16_tflops"] = mm(torch.bfloat16, 8192)
    out["fp64_tflops"] = mm(torch.float64, 8192)
    out["c64_tflops"] = mm(torch.complex64, 4096)
    src = torch.empty(1 << 28, device="cuda")
    dst = torch.empty_like(src)
    ms = _time(torch, lambda: dst.copy_(src), reps)
    out["copy_gbs"] = 2.0 * src.numel() * 4 / ms / 1e6
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", nargs="*", default=["narrow", "front", "rowid"])
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--grid", type=int, default=64)
    ap.add_argument("--blocks", type=int, default=200)
    ap.add_argument("--nmin", type=int, default=1024)
    args = ap.parse_args()
    import torch
    from paper_2007_00202_gb300 import build, mf
    build.build()
    for w in args.which:
        if w == "factor":
            r = factor(torch, mf, args.reps, args.grid, args.nmin)
        elif w == "solve":
            r = solve(torch, mf, args.reps, args.grid)
        elif w == "bfapply":
            r = bfapply(torch, mf, args.reps, args.blocks)
        else:
            r = {"narrow": narrow, "front": front, "rowid": rowid, "rowid_big": rowid_big,
                 "peaks": peaks}[w](torch, mf, args.reps)
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
