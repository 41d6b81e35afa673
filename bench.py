"""Benchmark of the GPU multifrontal solver on the 64^3 Helmholtz workload.

One step = the whole hot path on one problem: numeric factorization
(mf_factor) + solve of 16 right-hand sides to a true FP64 relative residual
<= 1e-8 (mf_solve*, GMRES(30) preconditioned by the complex64 factorization).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints ONE JSON line (rank 0).  Under torchrun (N > 1) every rank factors and
solves its own copy of the problem (replicas: the workload is one independent
problem per GPU, there is no data-path exchange) and value is the sum over
ranks.  --impl reference times the FP64 CPU oracle on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import queue
import subprocess
import tempfile
import threading
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "factor s and solves/s to 1e-8 residual, mixed vs FP64 GPU path; p99 latency"
UNIT = "solves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--grid", type=int, default=64)
    ap.add_argument("--problem", default="helmholtz", choices=["helmholtz", "yee", "poisson"],
                    help="helmholtz: 7-point damped Helmholtz (ppw 10), Gaussian RHS seed 7; yee: curl-curl on "
                         "grid^3 Yee cells with PEC walls (ppw 10), edge-dipole RHS seed 11; poisson: k = 0")
    ap.add_argument("--nrhs", type=int, default=16)
    ap.add_argument("--nmin", type=int, default=1024, help="separators >= nmin are HOD-BF compressed")
    ap.add_argument("--parallel-levels", type=int, default=0,
                    help="planar rule: cut the top N levels along the root separator's axis (parallel separators)")
    ap.add_argument("--ordering", default="planar", choices=["planar", "hybrid", "graph"],
                    help="planar: nested dissection by lattice planes; hybrid: lattice planes while the separators "
                         "are compressed, graph nested dissection inside boxes whose planar separator would stay "
                         "dense; graph: level-structure nested dissection of the matrix graph (coordinates withheld)")
    ap.add_argument("--no-dense", action="store_true", help="skip the all-dense complex64 comparison step")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 GPU comparison step")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving (continuous batching) measurement")
    ap.add_argument("--no-bfapply", action="store_true", help="skip the batched butterfly-apply measurement")
    ap.add_argument("--serving-full", action="store_true",
                    help="run only the full serving workload (32^3 + 64^3 + 100^3 resident, 2000 requests of "
                         "1-256 RHS) and print its JSON line; at 80 % of the measured capacity the 2000 requests "
                         "take about 40 minutes")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="with --serving-full: serve the first N requests of the seed-5 stream (the stream, its "
                         "arrival rate and the problems are those of the full workload)")
    return ap.parse_args()


def dist_setup(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, nrhs, ms_max):
    """Whole-job solves/s: every rank solves nrhs right-hand sides of its own replica per step,
    and the job's step takes as long as its slowest rank."""
    return world * nrhs / (ms_max / 1e3)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, idx):
        self.idx = idx
        self.proc = None
        # the raw samples go to MF_CLOCKS_DIR (default: the system's temporary directory)
        self.path = os.path.join(os.environ.get("MF_CLOCKS_DIR", tempfile.gettempdir()), f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [l.split(",") for l in open(self.path) if l.strip()]
        except Exception:
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# event timing of one launch (and one solve-graph replay) in PROFILE_PERIOD during the timed steps:
# the per-launch average comes from that sample, and the timing costs little of the step
PROFILE_PERIOD = 8
# nominal FP32 SIMT peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz maximum SM clock
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# DRAM traffic of the narrow GEMM per algorithmic byte, from an ncu capture of one streaming
# launch (4096 x 16 x 4096, 136 MB of A: read once), valid while the kernel's device code (the
# source file up to its first host launch function) hashes to NARROW_SRC_SHA1; scaled to the
# bench's launches by their algorithmic bytes
NARROW_TRAFFIC_PER_ALG_BYTE = 1.0204
NARROW_SRC_SHA1 = "d006306299d40ec83fe95f1fbcfd4d36babf87c6"


def _device_code_sha1(name, launcher):
    """SHA-1 of a kernel source file up to the template line that introduces its host function
    `launcher` (the device code; edits of the host launch code leave it unchanged)."""
    import hashlib
    path = os.path.join(ROOT, "paper_2007_00202_gb300", "csrc", name)
    try:
        text = open(path).read()
        i = text.index(f"void {launcher}(")
        i = text.rfind("\ntemplate", 0, i)
        return hashlib.sha1(text[:i].encode()).hexdigest() if i >= 0 else None
    except (OSError, ValueError):
        return None


def roofline(prof, peaks):
    """Roofline of the dominant kernel, the narrow GEMM (k_gemm_nrhs), from the CUDA-event
    profile of the timed steps: algorithmic flops and bytes over the summed launch time.
    Its arithmetic intensity (about 4 n flop per byte for n right-hand sides) is above the
    FP32-ALU / HBM ridge, so the ALU ceiling binds; the HBM fraction is reported beside it."""
    if not prof or prof["ms"] <= 0:
        return None
    sec = prof["ms"] / 1e3
    tflops = prof["flops"] / sec / 1e12
    gbs = prof["bytes"] / sec / 1e9
    hbm = peaks.get("hbm_gbs") or 6800.0
    ai = prof["flops"] / max(prof["bytes"], 1.0)
    traffic = None
    if NARROW_TRAFFIC_PER_ALG_BYTE is not None and _device_code_sha1("gemm_nrhs.cu", "launch_nb") == NARROW_SRC_SHA1:
        traffic = NARROW_TRAFFIC_PER_ALG_BYTE * prof["bytes"] / max(prof["launches"], 1)
    alu_bound = ai * hbm / 1e3 > FP32_ALU_TFLOPS
    r = {"kernel": "k_gemm_nrhs (narrow planar complex GEMM: solve front products, butterfly level products)",
         "launches_timed": prof["launches"], "sample": f"one launch / graph replay in {PROFILE_PERIOD}", "ms_per_launch": prof["ms"] / max(prof["launches"], 1),
         "flop_per_byte": ai, "traffic": traffic, "traffic_unit": "bytes per launch",
         "hbm_achieved_gbs": gbs, "hbm_peak_gbs": hbm, "hbm_frac": gbs / hbm,
         "peak_source": "alu: nominal FP32 SIMT peak 152 SM x 128 lanes x 2 x 2.07 GHz; "
                        "hbm: MEASURED_PEAKS.json hbm_gbs (of measured)"}
    if alu_bound:
        r.update({"bound": "alu", "achieved": tflops, "peak": FP32_ALU_TFLOPS, "unit": "TFLOP/s",
                  "frac": tflops / FP32_ALU_TFLOPS})
    else:
        r.update({"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm})
    return r


# nominal dense tensor rates of a GB300 (TF32 1.1, bf16 2.25 PFLOP/s): the TF32 ceiling is the
# measured bf16 peak scaled by their ratio
TF32_PER_BF16 = 1.1 / 2.25


def tf32_peak(peaks):
    bf16 = peaks.get("bf16_tflops") or 1900.0
    return bf16 * TF32_PER_BF16


def roofline_front(prof, peaks):
    """The dense fronts' Schur-update GEMMs of the factorization (tcgen05, split TF32: three
    passes per product) against the TF32 tensor peak (the measured bf16 peak x 1.1 / 2.25)."""
    if not prof or prof["ms"] <= 0:
        return None
    sec = prof["ms"] / 1e3
    alg = prof["flops"] / sec / 1e12
    peak = tf32_peak(peaks)
    return {"kernel": "k_gemm_tc<1> (tcgen05 kind::tf32, split precision) + SIMT trailing updates",
            "bound": "tensor", "achieved": alg, "achieved_tensor_passes": 3 * alg, "peak": peak,
            "unit": "TFLOP/s", "frac": alg / peak, "frac_tensor_passes": 3 * alg / peak,
            "launches": prof["launches"], "traffic": None,
            "peak_source": "TF32 = MEASURED_PEAKS.json bf16_tflops x 1.1/2.25 (nominal TF32:bf16 ratio; of measured)"}


def _rel(x, ref):
    import numpy as np
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def oracle_sample(n=20, nrhs=16):
    """The FP64 oracle on a bounded sample of the 64^3 workload: the same Helmholtz operator
    (ppw 10) at n^3, separators >= 128 HOD-BF compressed at tol 1e-4 with rank cap 64, factor +
    GMRES(30) solve of nrhs Gaussian RHS (seed 7) to 1e-8, timed on the host cores.  Also returns
    the oracle's exact solution of the same system (dense multifrontal LU in FP64, untimed), the
    reference of every GPU result's error."""
    import numpy as np
    import workloads as w
    from oracle.analysis import analyze
    from oracle import compressed_mf as cm, dense_mf as dm, gmres as gm
    p = w.helmholtz7(n, 10)
    b = w.rhs_gaussian(p, nrhs, 7)
    A = p.to_scipy()
    t0 = time.perf_counter()
    an = analyze(p, 64, 128, 64)
    fac, st = cm.compressed_factor(p, an, 1e-4, max_rank=64)
    X, its, res = gm.gmres(A, b, cm.preconditioner(an, fac), rtol=1e-8)
    dt = time.perf_counter() - t0
    ane = analyze(p, 64, 10 ** 9)
    x_exact = dm.solve(p, ane, dm.multifrontal_factor(p, ane)[0], b)
    cores = len(os.sched_getaffinity(0))
    return p, b, x_exact, {
        "value": nrhs / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
        "sample": f"FP64 oracle: HOD-BF multifrontal factor (tol 1e-4, rank <= 64, separators >= 128) + "
                  f"GMRES(30) of {nrhs} RHS to 1e-8 on helmholtz7 {n}^3 (N={p.n}); {dt:.1f} s, "
                  f"{max(its)} iterations, residual {max(res):.1e}",
        "seconds": dt, "err_vs_oracle_exact": _rel(X, x_exact)}


def direct_16cube(g, torch):
    """The 16^3 direct-solver configuration: helmholtz7 16^3 (ppw 8), separators >= 128 HOD-BF at
    tol 1e-6, complex128 factors, no refinement, RHS a point source at (8, 8, 8) plus a Gaussian
    column (seed 42); error against the oracle's exact solution (Alg. 1, FP64)."""
    import numpy as np
    import workloads as w
    from oracle.analysis import analyze
    from oracle import dense_mf as dm
    p = w.helmholtz7(16, 8)
    b = w.rhs_point_plus_gaussian(p, 42)
    an = analyze(p, 64, 10 ** 9)
    xe = dm.solve(p, an, dm.multifrontal_factor(p, an)[0], b)
    h = g.analyze_problem(p, nmin_sep=128, precision=g.MF_PREC_C128, refine=g.MF_REFINE_NONE,
                          stream=torch.cuda.current_stream().cuda_stream)
    h.mf_factor(1e-6)
    h.mf_solve(b, allow_no_convergence=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h.mf_factor(1e-6)
    torch.cuda.synchronize()
    tf = time.perf_counter() - t0
    t0 = time.perf_counter()
    x, _ = h.mf_solve(b, allow_no_convergence=True)
    ts = time.perf_counter() - t0
    A = p.to_scipy()
    st = h.mf_stats()
    return {"workload": "helmholtz7 16^3 (N=4096), ppw 8, separators >= 128 HOD-BF at tol 1e-6, complex128, "
                        "no refinement, point source + Gaussian RHS (seed 42)",
            "compressed_fronts": st["ncompressed"], "factor_s": tf, "solve_s": ts,
            "max_rel_residual": float(np.max(np.linalg.norm(A @ x - b, axis=0) / np.linalg.norm(b, axis=0))),
            "err_vs_oracle": _rel(x, xe)}


def gpu_paths_on(g, torch, p, b, x_exact, nmin, tol=1e-4):
    """The four GPU variants on one problem: factor s, solve s, solves/s, iterations, residual and
    the error against the oracle's exact solution x_exact."""
    import numpy as np
    nrhs = b.shape[1]
    stream = torch.cuda.current_stream().cuda_stream
    variants = {
        "compressed_c64": dict(nmin_sep=nmin, max_rank=64, precision=g.MF_PREC_C64, refine=g.MF_REFINE_GMRES),
        "dense_c64": dict(nmin_sep=10 ** 9, precision=g.MF_PREC_C64, refine=g.MF_REFINE_GMRES),
        "fp64_exact": dict(nmin_sep=10 ** 9, precision=g.MF_PREC_C128, refine=g.MF_REFINE_IR),
        "fp64_butterfly": dict(nmin_sep=nmin, max_rank=64, precision=g.MF_PREC_C128, refine=g.MF_REFINE_GMRES),
    }
    A = p.to_scipy()
    out = {}
    for name, kw in variants.items():
        h = g.analyze_problem(p, stream=stream, **kw)
        ftol = 0.0 if name == "fp64_exact" else tol
        h.mf_factor(ftol)                       # warm-up (allocations, graphs)
        h.mf_solve(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.mf_factor(ftol)
        torch.cuda.synchronize()
        tf = time.perf_counter() - t0
        t0 = time.perf_counter()
        x, info = h.mf_solve(b)
        ts = time.perf_counter() - t0
        res = float(np.max(np.linalg.norm(A @ x - b, axis=0) / np.linalg.norm(b, axis=0)))
        out[name] = {"factor_s": tf, "solve_s": ts, "solves_per_s": nrhs / (tf + ts), "iters": int(info.iters),
                     "max_rel_residual": res, "err_vs_oracle": _rel(x, x_exact)}
        del h
    return out


def serving(g, w, torch):
    """Continuous batching over resident factorizations (the serving workload, bounded): the
    helmholtz7 32^3 and 64^3 problems (complex64, separators >= 1024 HOD-BF at tol 1e-4, rank
    <= 64) factored and kept on the device, each on its own stream; 60 requests with Poisson
    arrivals (mean gap 100 ms, seed 5), each 1-16 complex Gaussian right-hand sides for a problem
    drawn uniformly; solved to 1e-8 by GMRES in the batches the server forms.  Latency is
    arrival to completion."""
    import numpy as np
    probs = [w.helmholtz7(32, 10), w.helmholtz7(64, 10)]
    streams = [torch.cuda.Stream() for _ in probs]
    hs = []
    for p, st in zip(probs, streams):
        h = g.analyze_problem(p, nmin_sep=1024, max_rank=64, precision=g.MF_PREC_C64, refine=g.MF_REFINE_GMRES,
                              stream=st.cuda_stream)
        h.mf_factor(1e-4)
        hs.append(h)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    pools = [np.asfortranarray(w.complex_gaussian(rng, p.n, 16)) for p in probs]
    nreq = 60
    gaps = rng.exponential(0.1, nreq)
    which = rng.integers(0, len(probs), nreq)
    widths = rng.integers(1, 17, nreq)
    srv = g.Server(hs, max_batch_rhs=256, mem_budget_bytes=96 << 30)
    ids, t0 = [], time.perf_counter()
    t = t0
    for k in range(nreq):
        t += gaps[k]
        while time.perf_counter() < t:
            time.sleep(max(0.0, min(1e-3, t - time.perf_counter())))
        ids.append((srv.submit(int(which[k]), pools[which[k]][:, :widths[k]]), int(which[k]), int(widths[k])))
    lat, batches, worst = [], [], 0.0
    checked = set()
    for rid, pi, k in ids:
        x, info = srv.wait(rid)
        lat.append((info["t_done"] - info["t_arrival"]) * 1e3)
        batches.append(info["batch_rhs"])
        if pi not in checked:
            A = probs[pi].to_scipy()
            bb = pools[pi][:, :k]
            worst = max(worst, float(np.max(np.linalg.norm(A @ x - bb, axis=0) / np.linalg.norm(bb, axis=0))))
            checked.add(pi)
    wall = time.perf_counter() - t0
    srv.close()
    lat.sort()
    return {"workload": "helmholtz7 32^3 + 64^3 resident, complex64 HOD-BF tol 1e-4; 60 Poisson requests "
                        "(mean gap 100 ms, seed 5) of 1-16 RHS each, GMRES to 1e-8",
            "requests": nreq, "rhs": int(widths.sum()), "p50_ms": lat[len(lat) // 2],
            "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))], "solves_per_s": float(widths.sum()) / wall,
            "mean_batch_rhs": float(np.mean(batches)), "max_rel_residual_checked": worst}


def serving_full(g, w, torch, nserve=2000, nreq=2000):
    """The serving workload at its stated size: helmholtz7 32^3, 64^3 and 100^3 (complex64, separators
    >= 1024 HOD-BF at tol 1e-4, rank <= 64) factored and resident on the device, each on its own
    stream; nreq requests (seed 5, of which the first nserve are served): problem rng.integers(3), nrhs = rint(exp(U(0, ln 256))) complex
    Gaussian right-hand sides, exponential inter-arrival times at 80 % of the measured single-stream
    capacity; batches admitted by free device memory; GMRES to 1e-8.  50 sampled requests are checked
    with an FP64 residual on the host."""
    import numpy as np
    # three factorizations stay resident: one construction context each (one work arena per handle),
    # so that the batches' GMRES workspace fits beside them
    os.environ["MF_SERIAL_FRONTS"] = "1"
    probs = [w.helmholtz7(32, 10), w.helmholtz7(64, 10), w.helmholtz7(100, 10)]
    streams = [torch.cuda.Stream() for _ in probs]
    hs = []
    for p, st in zip(probs, streams):
        h = g.analyze_problem(p, nmin_sep=1024, max_rank=64, precision=g.MF_PREC_C64, refine=g.MF_REFINE_GMRES,
                              stream=st.cuda_stream)
        h.mf_factor(1e-4)
        hs.append(h)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    which = rng.integers(0, len(probs), nreq)
    widths = np.rint(np.exp(rng.uniform(0.0, math.log(256.0), nreq))).astype(int)
    pools = [np.asfortranarray(w.complex_gaussian(rng, p.n, 256)) for p in probs]
    # single-stream capacity: solves/s of one full batch (64 columns: the tensor-core width of the
    # preconditioner's level products) per problem, averaged over the mix
    batch = 64
    cap = []
    for p, h, pool in zip(probs, hs, pools):
        h.mf_solve(pool[:, :batch])
        t0 = time.perf_counter()
        h.mf_solve(pool[:, :batch])
        cap.append(batch / (time.perf_counter() - t0))
    mix = np.bincount(which, minlength=len(probs)) / nreq
    capacity = 1.0 / float(np.sum(mix / np.array(cap)))          # RHS per second over the request mix
    rate = 0.8 * capacity / float(np.mean(widths))                # requests per second
    gaps = rng.exponential(1.0 / rate, nreq)
    print(f"serving: capacity {cap} RHS/s per problem", file=sys.stderr, flush=True)
    srv = g.Server(hs, max_batch_rhs=batch, mem_budget_bytes=1 << 62)   # admission by free device memory
    sample = set(np.random.default_rng(6).choice(nserve, min(50, nserve), replace=False).tolist())
    As = [p.to_scipy() for p in probs]
    # results are collected while requests keep arriving (each solution is dropped once checked),
    # so the host holds only the solutions of requests in flight
    pending = queue.Queue()
    lat, statuses, worst = [], [], [0.0]

    def collect():
        while True:
            item = pending.get()
            if item is None:
                return
            q, rid, pi, k = item
            x, info = srv.wait(rid)
            lat.append((info["t_done"] - info["t_arrival"]) * 1e3)
            statuses.append(info["status"])
            if q in sample:
                bb = pools[pi][:, :k]
                worst[0] = max(worst[0], float(np.max(np.linalg.norm(As[pi] @ x - bb, axis=0) /
                                                      np.linalg.norm(bb, axis=0))))
            del x
    collector = threading.Thread(target=collect)
    collector.start()
    t0 = time.perf_counter()
    t = t0
    for k in range(nserve):
        t += gaps[k]
        while time.perf_counter() < t:
            time.sleep(max(0.0, min(1e-3, t - time.perf_counter())))
        pending.put((k, srv.submit(int(which[k]), pools[which[k]][:, :widths[k]]), int(which[k]), int(widths[k])))
        if k % 100 == 99:
            done = sorted(lat)
            pq = (f", p50 {done[len(done) // 2]:.0f} ms, p99 {done[min(len(done) - 1, int(0.99 * len(done)))]:.0f} ms"
                  if done else "")
            print(f"serving: {k + 1} requests submitted, {len(done)} done, {time.perf_counter() - t0:.0f} s{pq}",
                  file=sys.stderr, flush=True)
    pending.put(None)
    collector.join()
    wall = time.perf_counter() - t0
    srv.close()
    worst = worst[0]
    lat.sort()
    served = int(widths[:nserve].sum())
    return {"workload": "helmholtz7 32^3 + 64^3 + 100^3 resident, complex64 HOD-BF tol 1e-4; "
                        f"{nreq} Poisson requests (seed 5) of rint(exp(U(0, ln 256))) RHS, arrivals at 80 % of the "
                        f"measured capacity ({capacity:.0f} RHS/s), admission by free device memory, GMRES to 1e-8"
                        + ("" if nserve == nreq else f"; the first {nserve} requests of the stream served"),
            "requests": nserve, "rhs": served, "arrival_rate_per_s": rate, "max_batch_rhs": batch,
            "capacity_rhs_per_s": capacity,
            "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "solves_per_s": served / wall, "wall_s": wall,
            "all_converged": bool(all(s_ == 0 for s_ in statuses)),
            "max_rel_residual_sampled": worst, "sampled": len(sample)}


def butterfly_apply(g, w, torch, peaks, nrhs=64):
    """The batched butterfly-apply workload: 200 compressed blocks of the Helmholtz Green's function
    between two parallel m x m point planes one spacing apart (m = rint(16 * 8^u), u ~ U(0,1),
    seed 3; k = pi/4; ID tolerance 1e-4, leaf 64), built on the GPU and applied to 64 complex
    Gaussian vectors per block (all blocks and levels in stage-merged launches).  Bytes =
    stored factor entries x 8 + input and output vectors; error against the dense FP64 product
    on three blocks of at most 48 x 48 points."""
    import numpy as np
    import paper_2007_00202_gb300.mf as mf
    ms = w.butterfly_bench_sizes(200, 3)
    S = mf.GreenSet([int(m) for m in ms], math.pi / 4, 1.0, 1e-4, leaf=64,
                    stream=torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(8)
    X = w.complex_gaussian(rng, S.rows, nrhs)
    dX = torch.from_numpy(np.concatenate([X.real.ravel(), X.imag.ravel()]).astype(np.float32)).cuda()
    dY = torch.zeros_like(dX)
    for _ in range(3):
        S.apply(nrhs, dX.data_ptr(), dY.data_ptr())
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record()
    for _ in range(reps):
        S.apply(nrhs, dX.data_ptr(), dY.data_ptr())
    e1.record()
    torch.cuda.synchronize()
    ms_apply = e0.elapsed_time(e1) / reps
    Yg = dY.cpu().numpy().astype(np.float64)
    Yg = (Yg[:S.rows * nrhs] + 1j * Yg[S.rows * nrhs:]).reshape(S.rows, nrhs)
    P, Q = S.points()
    offs = np.concatenate([[0], np.cumsum(ms.astype(np.int64) ** 2)])
    err = 0.0
    small = [int(b) for b in np.argsort(ms) if ms[b] <= 48]   # dense K of at most 2304^2 entries
    for b in [small[0], small[len(small) // 2], small[-1]]:
        a, e = int(offs[b]), int(offs[b + 1])
        K = w.green_entries(P[a:e], Q[a:e], math.pi / 4, np.arange(e - a), np.arange(e - a))
        ref = K @ X[a:e]
        err = max(err, float(np.linalg.norm(Yg[a:e] - ref) / np.linalg.norm(ref)))
    alg_bytes = 8.0 * S.storage + 2.0 * 8.0 * S.rows * nrhs
    flops = 8.0 * S.storage * nrhs
    # with the level vectors in device memory: every level product's factor block, input and output
    # (inter-level vector traffic, part of the apply's algorithmic bytes when levels are not kept on chip)
    _, level_bytes = S.apply_counts(nrhs)
    hbm = peaks.get("hbm_gbs") or 6800.0
    gbs = alg_bytes / (ms_apply / 1e3) / 1e9
    return {"workload": f"200 Green's-function blocks (m = rint(16*8^u), seed 3), tol 1e-4, {nrhs} vectors each",
            "rows": S.rows, "stored_entries": S.storage, "max_rank": S.max_rank, "build_s": S.build_seconds,
            "apply_ms": ms_apply, "alg_gbs": gbs, "hbm_frac": gbs / hbm,
            "level_traffic_bytes": level_bytes, "level_traffic_gbs": level_bytes / (ms_apply / 1e3) / 1e9,
            "level_traffic_hbm_frac": level_bytes / (ms_apply / 1e3) / 1e9 / hbm,
            "tflops": flops / (ms_apply / 1e3) / 1e12, "alu_frac": flops / (ms_apply / 1e3) / 1e12 / FP32_ALU_TFLOPS,
            "max_rel_err_vs_dense_fp64": err, "err_vs_oracle": err,
            "err_reference": "dense FP64 product K X of the kernel's closed form on three blocks"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    vals = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample()[3]
        if i >= args.warmup:
            vals.append(r["value"])
    v = sum(vals) / len(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 16 / v * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": "helmholtz7 20^3 sample of the 64^3 workload (FP64 CPU oracle, HOD-BF tol 1e-4)",
                       "nrhs": 16},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": r["cores"], "kind": "oracle", "sample": r["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import numpy as np
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_2007_00202_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    barrier(world)
    import paper_2007_00202_gb300 as g
    import workloads as w

    if args.serving_full:
        if rank == 0:
            print(json.dumps({"metric": "serving p50/p99 latency and solves/s (full serving workload)",
                              "serving_full": serving_full(g, w, torch, args.serving_requests)}), flush=True)
        barrier(world)
        return

    n = args.grid
    nrhs = args.nrhs
    if args.problem == "yee":
        p = w.yee_maxwell(n, 10)
        b = w.rhs_dipoles(p, nrhs, 11)
        wname = f"Yee curl-curl {n}^3 cells, PEC (N={p.n}), ppw 10, {nrhs} edge-dipole RHS seed 11"
    else:
        p = w.helmholtz7(n, 10, k=0.0) if args.problem == "poisson" else w.helmholtz7(n, 10)
        b = w.rhs_gaussian(p, nrhs, 7)
        wname = (f"{'poisson7 (k = 0)' if args.problem == 'poisson' else 'helmholtz7'} {n}^3 (N={p.n})"
                 f"{'' if args.problem == 'poisson' else ', ppw 10'}, {nrhs} Gaussian RHS seed 7")
    stream = torch.cuda.current_stream()
    # complex64 factors, separators >= 1024 in HOD-BF at tol 1e-4 (rank <= 64), FP64 GMRES(30) to 1e-8
    nmin = args.nmin
    tol = 1e-4
    okw = {"planar": {}, "graph": {"graph": True}, "hybrid": {"ordering": g.MF_ORDER_HYBRID}}[args.ordering]
    if args.parallel_levels:
        okw = dict(okw, parallel_levels=args.parallel_levels)
    h = g.analyze_problem(p, **okw, nmin_sep=nmin, max_rank=64, precision=g.MF_PREC_C64, refine=g.MF_REFINE_GMRES,
                          stream=stream.cuda_stream)
    bd = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()     # N x nrhs column-major, resident
    xd = torch.empty_like(bd)
    A = p.to_scipy()

    def step():
        h.mf_factor(tol)
        return h.mf_solve_device(nrhs, bd.data_ptr(), xd.data_ptr())

    for _ in range(args.warmup):
        info = step()
    torch.cuda.synchronize()
    h.mf_profile(True, period=PROFILE_PERIOD)
    barrier(world)
    torch.cuda.synchronize()
    c0 = g.lib().mf_launch_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.profiler.start()   # under `ncu --profile-from-start off`: the timed steps only
        e0.record(stream)
        for _ in range(args.steps):
            info = step()
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    launches = g.lib().mf_launch_counter() - c0
    ms = e0.elapsed_time(e1) / args.steps
    prof = h.mf_profile_read(g.MF_PROF_NARROW_GEMM)
    prof_front = h.mf_profile_read(g.MF_PROF_FRONT_GEMM)
    h.mf_profile(False)
    barrier(world)
    ms_max = allmax(ms, world)
    x = xd.cpu().numpy().T
    res = float(np.max(np.linalg.norm(A @ x - b, axis=0) / np.linalg.norm(b, axis=0)))
    value = replica_throughput(world, nrhs, ms_max)
    st = h.mf_stats()
    # factor-only timing (one extra untimed pass, for the factor-seconds part of the metric)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h.mf_factor(tol)
    torch.cuda.synchronize()
    factor_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    h.mf_solve_device(nrhs, bd.data_ptr(), xd.data_ptr())
    torch.cuda.synchronize()
    solve_s = time.perf_counter() - t0

    # e2e: the public host-buffer call (H2D of b and D2H of x inside the timed region)
    for _ in range(1):
        h.mf_factor(tol)
        h.mf_solve(b)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        h.mf_factor(tol)
        xe, _ = h.mf_solve(b)
    torch.cuda.synchronize()
    e2e_ms = allmax((time.perf_counter() - t0) / args.steps * 1e3, world)

    line = None
    if rank == 0:
        peaks = measured_peaks()
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "c64", "data": "synthetic",
                "config": {"workload": f"{wname}, complex64 factors, separators >= {nmin} HOD-BF at tol 1e-4 "
                                       f"(rank <= 64), FP64 GMRES(30) to 1e-8",
                           "compressed_fronts": st["ncompressed"], "max_rank": st["max_rank"],
                           "arena_peak_gb": st["arena_peak_bytes"] / 1e9,
                           "arena_capacity_gb": st["arena_capacity_bytes"] / 1e9,
                           "nrhs": nrhs, "nmin_sep": nmin, "ordering": args.ordering,
                           "parallel_levels": args.parallel_levels,
                           "l2": "inputs larger than L2 (factors "
                           f"{st['factor_bytes'] / 1e9:.1f} GB)", "parallelism": "replicas" if world > 1 else "1gpu"},
                "factor_s": factor_s, "solve_s": solve_s, "solve_iters": int(info.iters),
                "max_rel_residual_host_check": res,
                "gpu_launches": int(launches),
                "roofline": roofline(prof, peaks),
                "roofline_front_gemm": roofline_front(prof_front, peaks),
                "e2e": {"value": world * nrhs / (e2e_ms / 1e3), "unit": UNIT,
                        "h2d_bytes_per_step": int(16 * p.n * nrhs), "d2h_bytes_per_step": int(16 * p.n * nrhs)}}
        c = clk.summary()
        if c:
            line["clocks"] = c
    # the comparison paths below each hold a factorization of their own: free this one first
    h.close()
    torch.cuda.synchronize()
    # all-dense complex64 path (same solver without compression), one step
    if rank == 0 and not args.no_dense:
      try:
        hd = g.analyze_problem(p, **okw, nmin_sep=10 ** 9, precision=g.MF_PREC_C64, refine=g.MF_REFINE_GMRES,
                               stream=stream.cuda_stream)
        hd.mf_factor(tol)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hd.mf_factor(tol)
        torch.cuda.synchronize()
        fd = time.perf_counter() - t0
        t0 = time.perf_counter()
        infod = hd.mf_solve_device(nrhs, bd.data_ptr(), xd.data_ptr())
        torch.cuda.synchronize()
        sd = time.perf_counter() - t0
        line["dense_c64_path"] = {"factor_s": fd, "solve_s": sd, "solves_per_s": nrhs / (fd + sd),
                                  "gmres_iters": int(infod.iters), "max_rel_residual": infod.max_rel_residual}
        del hd
      except Exception as e:   # the comparison path failed (e.g. out of memory): record it, keep the line
        line["dense_c64_path"] = {"error": str(e)[:300]}
    # FP64 GPU path (same code in complex128), one step, for the mixed-vs-FP64 comparison
    if rank == 0 and not args.no_fp64:
      try:
        h64 = g.analyze_problem(p, **okw, nmin_sep=10 ** 9, precision=g.MF_PREC_C128, refine=g.MF_REFINE_IR,
                                stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h64.mf_factor(0.0)
        torch.cuda.synchronize()
        f64 = time.perf_counter() - t0
        t0 = time.perf_counter()
        info64 = h64.mf_solve_device(nrhs, bd.data_ptr(), xd.data_ptr())
        torch.cuda.synchronize()
        s64 = time.perf_counter() - t0
        line["fp64_path"] = {"variant": "exact (all-dense) multifrontal in complex128 + iterative refinement",
                             "factor_s": f64, "solve_s": s64, "solves_per_s": nrhs / (f64 + s64),
                             "refinement_steps": int(info64.iters), "max_rel_residual": info64.max_rel_residual}
        del h64
      except Exception as e:
        line["fp64_path"] = {"error": str(e)[:300]}
      try:
        # FP64 butterfly variant: the compressed path in complex128 + GMRES
        hb = g.analyze_problem(p, **okw, nmin_sep=nmin, max_rank=64, precision=g.MF_PREC_C128, refine=g.MF_REFINE_GMRES,
                               stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hb.mf_factor(tol)
        torch.cuda.synchronize()
        fb = time.perf_counter() - t0
        t0 = time.perf_counter()
        infob = hb.mf_solve_device(nrhs, bd.data_ptr(), xd.data_ptr())
        torch.cuda.synchronize()
        sb = time.perf_counter() - t0
        line["fp64_butterfly_path"] = {"factor_s": fb, "solve_s": sb, "solves_per_s": nrhs / (fb + sb),
                                       "gmres_iters": int(infob.iters), "max_rel_residual": infob.max_rel_residual}
        del hb
      except Exception as e:
        line["fp64_butterfly_path"] = {"error": str(e)[:300]}
    if rank == 0 and not args.no_serving:
        line["serving"] = serving(g, w, torch)
    if rank == 0 and not args.no_bfapply:
        line["butterfly_apply"] = butterfly_apply(g, w, torch, measured_peaks())
    if rank == 0 and not args.no_cpu:
        # the cpu_baseline leg: the oracle timed on the 20^3 sample, the GPU paths on the same problem
        # beside it, and every GPU path's error against the oracle's exact solution of that problem
        ps, bs, xs, cb = oracle_sample()
        same = gpu_paths_on(g, torch, ps, bs, xs, nmin=128)
        cb["gpu_same_problem"] = same
        cb["gpu_over_oracle"] = same["compressed_c64"]["solves_per_s"] / cb["value"]
        line["cpu_baseline"] = cb
        for key, name in (("dense_c64_path", "dense_c64"), ("fp64_path", "fp64_exact"),
                          ("fp64_butterfly_path", "fp64_butterfly")):
            if key in line:
                line[key]["err_vs_oracle_20cube"] = same[name]["err_vs_oracle"]
        line["err_vs_oracle_20cube"] = same["compressed_c64"]["err_vs_oracle"]
        line["direct_16cube"] = direct_16cube(g, torch)
    if rank == 0:
        print(json.dumps(line), flush=True)
    barrier(world)


if __name__ == "__main__":
    main()
