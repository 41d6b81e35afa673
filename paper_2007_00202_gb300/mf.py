"""Thin Python binding of the C ABI in include/mf.h (argument marshalling only).

Every computation runs in libmf.so; this module converts numpy arrays and
raw device pointers into the C calls of the same names and raises MfError on
a negative return code.  Importing it does not need a GPU; calls that touch
the device (mf_factor, mf_solve*) do.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmf.so")

MF_OK = 0
ERRORS = {-1: "MF_ERR_ARG", -2: "MF_ERR_STATE", -3: "MF_ERR_UNSUPPORTED", -4: "MF_ERR_OOM",
          -5: "MF_ERR_SINGULAR", -6: "MF_ERR_NO_CONVERGENCE", -7: "MF_ERR_TIMEOUT", -8: "MF_ERR_CUDA"}
MF_LATTICE_NODE, MF_LATTICE_EDGE = 0, 1
MF_PREC_C64, MF_PREC_C128 = 0, 1
MF_REFINE_NONE, MF_REFINE_GMRES, MF_REFINE_IR = 0, 1, 2
MF_PROF_NARROW_GEMM, MF_PROF_FRONT_GEMM = 0, 1
MF_OP_F11, MF_OP_F11_INV, MF_OP_F12, MF_OP_F21, MF_OP_C = 0, 1, 2, 3, 4
MF_OPTIONS_V1, MF_OPTIONS_V2 = 1, 2
MF_ORDER_AUTO, MF_ORDER_HYBRID, MF_ORDER_GRAPH = 0, 1, 2


class MfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class mf_options(C.Structure):
    _fields_ = [("version", C.c_int32), ("leaf_size", C.c_int32), ("nmin_sep", C.c_int32),
                ("hodbf_leaf", C.c_int32), ("max_rank", C.c_int32), ("alpha", C.c_int32), ("knn", C.c_int32),
                ("precision", C.c_int32), ("refine", C.c_int32), ("gmres_restart", C.c_int32),
                ("max_iters", C.c_int32), ("lattice", C.c_int32), ("rtol", C.c_double), ("seed", C.c_uint64),
                ("coords", C.POINTER(C.c_int32)), ("ordering", C.c_int32), ("parallel_levels", C.c_int32)]


class mf_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("max_rel_residual", C.c_double)]


class mf_stats_t(C.Structure):
    _fields_ = [("n", C.c_int64), ("nfronts", C.c_int64), ("ncompressed", C.c_int64), ("tree_levels", C.c_int32),
                ("max_rank", C.c_int32), ("factor_flops", C.c_double), ("factor_bytes", C.c_double),
                ("factor_seconds", C.c_double), ("precision", C.c_int32), ("gpu_launches_factor", C.c_int32),
                ("gpu_launches_solve", C.c_int32), ("reserved", C.c_int32), ("arena_peak_bytes", C.c_double),
                ("arena_capacity_bytes", C.c_double)]


class mf_kernel_profile_t(C.Structure):
    _fields_ = [("launches", C.c_int64), ("ms", C.c_double), ("flops", C.c_double), ("bytes", C.c_double)]


class mf_request_info(C.Structure):
    _fields_ = [("id", C.c_int64), ("problem", C.c_int32), ("nrhs", C.c_int32), ("iters", C.c_int32),
                ("converged", C.c_int32), ("batch_rhs", C.c_int32), ("reserved", C.c_int32),
                ("max_rel_residual", C.c_double), ("t_arrival", C.c_double), ("t_start", C.c_double),
                ("t_done", C.c_double)]


class mf_analysis_sizes_t(C.Structure):
    _fields_ = [("n", C.c_int64), ("nfronts", C.c_int64), ("upd_total", C.c_int64), ("tree_total", C.c_int64),
                ("nn_total", C.c_int64)]


_P = C.c_void_p
_I64P = C.POINTER(C.c_int64)
_I32P = C.POINTER(C.c_int32)
_DP = C.POINTER(C.c_double)

# name -> (restype, argtypes); every name here must be exported by libmf.so
SIGNATURES = {
    "mf_options_init": (C.c_int, [C.POINTER(mf_options)]),
    "mf_analyze": (C.c_int, [C.c_int64, _I64P, _I32P, _DP, C.POINTER(mf_options), _P, C.POINTER(_P)]),
    "mf_factor": (C.c_int, [_P, C.c_double]),
    "mf_solve": (C.c_int, [_P, C.c_int32, _DP, C.c_int64, _DP, C.c_int64, C.POINTER(mf_solve_info)]),
    "mf_solve_device": (C.c_int, [_P, C.c_int32, _P, _P, C.POINTER(mf_solve_info)]),
    "mf_stats": (C.c_int, [_P, C.POINTER(mf_stats_t)]),
    "mf_solve_columns": (C.c_int, [_P, C.c_int32, _I32P, _I32P, _DP]),
    "mf_last_error": (C.c_char_p, [_P]),
    "mf_destroy": (None, [_P]),
    "mf_launch_counter": (C.c_int64, []),
    "mf_profile": (C.c_int, [_P, C.c_int32]),
    "mf_server_create": (C.c_int, [C.c_int32, C.POINTER(_P), C.c_int32, C.c_int64, C.POINTER(_P)]),
    "mf_server_submit": (C.c_int, [_P, C.c_int32, C.c_int32, _P, _P, _I64P]),
    "mf_server_wait": (C.c_int, [_P, C.c_int64, C.POINTER(mf_request_info)]),
    "mf_server_destroy": (None, [_P]),
    "mf_green_build": (C.c_int, [C.c_int32, _I32P, C.c_double, C.c_double, C.c_double, C.c_int32, C.c_int32,
                                 C.c_int32, C.c_int32, _P, C.POINTER(_P)]),
    "mf_green_info": (C.c_int, [_P, _I64P, _DP, _I32P, _DP]),
    "mf_green_points": (C.c_int, [_P, _DP, _DP]),
    "mf_green_apply": (C.c_int, [_P, C.c_int32, _P, _P]),
    "mf_green_apply_counts": (C.c_int, [_P, C.c_int32, _DP, _DP]),
    "mf_green_destroy": (None, [_P]),
    "mf_row_id_c64": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, _P, C.c_double, C.c_int32, _P, _P, _P, _P]),
    "mf_row_id_c64_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, _P, C.c_double, C.c_int32, _P, _P, _P,
                                        _P]),
    "mf_gemm_c64": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P, C.c_int64, C.c_int64, _P, C.c_int64,
                              C.c_int64, _P, C.c_int64, C.c_int64, C.c_float, C.c_float, _P]),
    "mf_gemm_nrhs_c64": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P, C.c_int64, C.c_int64, _P,
                                   C.c_int64, C.c_int64, _P, C.c_int64, C.c_int64, C.c_float, C.c_float, C.c_int32,
                                   _P]),
    "mf_profile_read": (C.c_int, [_P, C.c_int32, C.POINTER(mf_kernel_profile_t)]),
    "mf_analysis_sizes": (C.c_int, [_P, C.POINTER(mf_analysis_sizes_t)]),
    "mf_analysis_export": (C.c_int, [_P, _I64P, _I64P, _I64P, _I32P, _I64P, _I64P]),
    "mf_front_trees": (C.c_int, [_P, C.c_int64, _I64P, _I64P]),
    "mf_front_apply": (C.c_int, [_P, C.c_int64, C.c_int32, C.c_int32, _DP, _DP]),
    "mf_set_wait_limit": (C.c_int, [C.c_int64]),
    "mf_front_neighbours": (C.c_int, [_P, C.c_int64, C.c_int32, _I64P, _I64P, _I64P]),
}

_lib = None


def lib():
    """The loaded libmf.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2007_00202_gb300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def _check(rc, h=None):
    if rc != MF_OK:
        msg = lib().mf_last_error(h).decode(errors="replace")
        raise MfError(rc, msg)
    return rc


def mf_options_init(**kw) -> mf_options:
    o = mf_options()
    _check(lib().mf_options_init(C.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class Handle:
    """Owns one mf_handle*."""

    def __init__(self, ptr, keep):
        self.ptr = ptr
        self._keep = keep

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "ptr", None):
            lib().mf_destroy(self.ptr)
            self.ptr = None

    # ---------------- numeric phases ----------------
    def mf_factor(self, tol: float):
        _check(lib().mf_factor(self.ptr, float(tol)), self.ptr)

    def mf_solve(self, b: np.ndarray, allow_no_convergence=False):
        """b: (N,) or (N, nrhs) complex128 host array -> (x, info)."""
        b = np.asarray(b, dtype=np.complex128)
        vec = b.ndim == 1
        B = np.asfortranarray(b[:, None] if vec else b)
        n, nrhs = B.shape
        X = np.empty_like(B, order="F")
        info = mf_solve_info()
        dp = C.POINTER(C.c_double)
        rc = lib().mf_solve(self.ptr, nrhs, C.cast(B.ctypes.data, dp), n, C.cast(X.ctypes.data, dp), n,
                            C.byref(info))
        if not (allow_no_convergence and rc == -6):
            _check(rc, self.ptr)
        return (X[:, 0] if vec else X), info

    def mf_solve_device(self, nrhs: int, d_b: int, d_x: int, allow_no_convergence=False):
        """d_b, d_x: device pointers (int) to interleaved complex128 N x nrhs column-major."""
        info = mf_solve_info()
        rc = lib().mf_solve_device(self.ptr, nrhs, C.c_void_p(d_b), C.c_void_p(d_x), C.byref(info))
        if not (allow_no_convergence and rc == -6):
            _check(rc, self.ptr)
        return info

    def mf_solve_columns(self, nrhs: int) -> dict:
        """Per-column iterations, converged flags and true relative residuals of the last solve."""
        it = np.zeros(nrhs, np.int32)
        cv = np.zeros(nrhs, np.int32)
        rr = np.zeros(nrhs, np.float64)
        _check(lib().mf_solve_columns(self.ptr, nrhs, _p(it, C.c_int32), _p(cv, C.c_int32), _p(rr, C.c_double)),
               self.ptr)
        return {"iters": it, "converged": cv, "rel_residual": rr}

    def mf_stats(self) -> dict:
        s = mf_stats_t()
        _check(lib().mf_stats(self.ptr, C.byref(s)), self.ptr)
        return {k: getattr(s, k) for k, _ in s._fields_}

    def mf_profile(self, enable, period: int = 1):
        """enable: False stops; True times one launch (and one graph replay) in `period`."""
        _check(lib().mf_profile(self.ptr, int(period) if enable else 0), self.ptr)

    def mf_profile_read(self, kernel: int = 0) -> dict:
        """kernel: MF_PROF_NARROW_GEMM (0) or MF_PROF_FRONT_GEMM (1); see include/mf.h."""
        p = mf_kernel_profile_t()
        _check(lib().mf_profile_read(self.ptr, kernel, C.byref(p)), self.ptr)
        return dict(launches=p.launches, ms=p.ms, flops=p.flops, bytes=p.bytes)

    # ---------------- inspection (host only) ----------------
    def mf_analysis_export(self) -> dict:
        sz = mf_analysis_sizes_t()
        _check(lib().mf_analysis_sizes(self.ptr, C.byref(sz)), self.ptr)
        n, nf = sz.n, sz.nfronts
        perm = np.empty(n, np.int64)
        parent = np.empty(nf, np.int64)
        sep = np.empty(2 * nf, np.int64)
        flags = np.empty(nf, np.int32)
        uptr = np.empty(nf + 1, np.int64)
        uidx = np.empty(max(sz.upd_total, 1), np.int64)
        _check(lib().mf_analysis_export(self.ptr, _p(perm, C.c_int64), _p(parent, C.c_int64), _p(sep, C.c_int64),
                                        _p(flags, C.c_int32), _p(uptr, C.c_int64), _p(uidx, C.c_int64)), self.ptr)
        return dict(perm=perm, parent=parent, sep=sep.reshape(nf, 2), compressed=flags.astype(bool),
                    upd_ptr=uptr, upd_idx=uidx[:sz.upd_total])

    def mf_front_apply(self, f: int, which: int, x: np.ndarray, out_rows: int) -> np.ndarray:
        """Y = K x for operator `which` (MF_OP_*) of compressed front f; x: (in, nrhs) complex."""
        X = np.asfortranarray(np.asarray(x, dtype=np.complex128))
        Y = np.empty((out_rows, X.shape[1]), np.complex128, order="F")
        dp = C.POINTER(C.c_double)
        _check(lib().mf_front_apply(self.ptr, f, which, X.shape[1], C.cast(X.ctypes.data, dp),
                                    C.cast(Y.ctypes.data, dp)), self.ptr)
        return Y

    def mf_front_trees(self, f: int):
        nlev = np.zeros(2, np.int64)
        _check(lib().mf_front_trees(self.ptr, f, _p(nlev, C.c_int64), None), self.ptr)
        tot = sum(2 * ((1 << int(L)) - 1) for L in nlev)
        rng = np.empty(max(tot, 1), np.int64)
        _check(lib().mf_front_trees(self.ptr, f, _p(nlev, C.c_int64), _p(rng, C.c_int64)), self.ptr)
        out, p = [], 0
        for L in nlev:
            tree = []
            for l in range(int(L)):
                cnt = 1 << l
                tree.append([(int(rng[p + 2 * i]), int(rng[p + 2 * i + 1])) for i in range(cnt)])
                p += 2 * cnt
            out.append(tree)
        return out

    def mf_front_neighbours(self, f: int, knn: int, s: int, u: int):
        counts = np.zeros(4, np.int64)
        _check(lib().mf_front_neighbours(self.ptr, f, knn, _p(counts, C.c_int64), None, None), self.ptr)
        ptr = np.empty(2 * (s + 1) + 2 * (u + 1), np.int64)
        idx = np.empty(max(int(counts.sum()), 1), np.int64)
        _check(lib().mf_front_neighbours(self.ptr, f, knn, _p(counts, C.c_int64), _p(ptr, C.c_int64),
                                         _p(idx, C.c_int64)), self.ptr)
        lens = [s, u, s, u]
        out, pp, ip = [], 0, 0
        for k in range(4):
            rp = ptr[pp:pp + lens[k] + 1]
            pp += lens[k] + 1
            ent = idx[ip:ip + counts[k]]
            ip += int(counts[k])
            out.append([ent[rp[i]:rp[i + 1]].tolist() for i in range(lens[k])])
        return dict(zip(("nn11", "nn22", "nn12", "nn21"), out))


def mf_analyze(n, rowptr, colind, vals, coords, lattice=MF_LATTICE_NODE, stream=0, **opts) -> Handle:
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.complex128)
    o = mf_options_init(lattice=lattice, **opts)
    if coords is not None:          # None: general CSR input, graph nested dissection
        coords = np.ascontiguousarray(coords, dtype=np.int32)
        if coords.shape != (n, 3):
            raise ValueError("coords must be N x 3")
        o.coords = _p(coords, C.c_int32)
    h = C.c_void_p()
    rc = lib().mf_analyze(n, _p(rowptr, C.c_int64), _p(colind, C.c_int32), C.cast(vals.ctypes.data, C.POINTER(C.c_double)),
                          C.byref(o), C.c_void_p(stream), C.byref(h))
    _check(rc, None)
    return Handle(h, (rowptr, colind, vals, coords))


def analyze_problem(prob, graph=False, **opts) -> Handle:
    """mf_analyze on a workloads.SparseProblem-like object (n, rowptr, colind, vals, coords, lattice);
    graph=True withholds the coordinates (graph nested dissection of the CSR pattern); the ordering
    option (MF_ORDER_*) picks planar, hybrid or graph nested dissection when coordinates are given."""
    return mf_analyze(prob.n, prob.rowptr, prob.colind, prob.vals, None if graph else prob.coords, prob.lattice,
                      **opts)


def mf_gemm_c64(engine, m, n, k, A, lda, pla, B, ldb, plb, C_, ldc, plc, alpha, beta, stream=0):
    """Component GEMM on device pointers (ints); see include/mf.h."""
    _check(lib().mf_gemm_c64(engine, m, n, k, C.c_void_p(A), lda, pla, C.c_void_p(B), ldb, plb, C.c_void_p(C_), ldc,
                             plc, alpha, beta, C.c_void_p(stream)))


def mf_gemm_nrhs_c64(trans_a, m, n, k, A, lda, pla, B, ldb, plb, C_, ldc, plc, alpha, beta, ksplit=0, stream=0):
    """Component narrow GEMM (solve / butterfly level products) on device pointers (ints); see include/mf.h."""
    _check(lib().mf_gemm_nrhs_c64(trans_a, m, n, k, C.c_void_p(A), lda, pla, C.c_void_p(B), ldb, plb, C.c_void_p(C_),
                                  ldc, plc, alpha, beta, ksplit, C.c_void_p(stream)))


def mf_row_id_c64(nmat, m, n, M, tol, max_rank, U, sk, rank, stream=0):
    """Component batched row ID on device pointers (ints); see include/mf.h."""
    _check(lib().mf_row_id_c64(nmat, m, n, C.c_void_p(M), tol, max_rank, C.c_void_p(U), C.c_void_p(sk),
                               C.c_void_p(rank), C.c_void_p(stream)))


def mf_set_wait_limit(spins: int):
    """Poll limit of the tensor-core kernels' bounded waits (0: the default); see include/mf.h."""
    _check(lib().mf_set_wait_limit(int(spins)))


def mf_row_id_c64_noalloc(nmat, m, n, M, tol, max_rank, U, sk, rank, stream=0):
    """mf_row_id_c64 with the library's fixed scratch array (no device allocation); see include/mf.h."""
    _check(lib().mf_row_id_c64_noalloc(nmat, m, n, C.c_void_p(M), tol, max_rank, C.c_void_p(U), C.c_void_p(sk),
                                       C.c_void_p(rank), C.c_void_p(stream)))


class GreenSet:
    """Set of HOD-BF compressed Green's-function blocks built on the GPU (mf_green_*)."""

    def __init__(self, m_list, k, h=1.0, tol=1e-4, leaf=64, max_rank=0, alpha=2, knn=8, stream=0):
        m = np.ascontiguousarray(m_list, dtype=np.int32)
        self.ptr = C.c_void_p()
        _check(lib().mf_green_build(len(m), _p(m, C.c_int32), k, h, tol, leaf, max_rank, alpha, knn,
                                    C.c_void_p(stream), C.byref(self.ptr)))
        rows = C.c_int64(); st = C.c_double(); mr = C.c_int32(); bs = C.c_double()
        _check(lib().mf_green_info(self.ptr, C.byref(rows), C.byref(st), C.byref(mr), C.byref(bs)))
        self.rows, self.storage, self.max_rank, self.build_seconds = rows.value, st.value, mr.value, bs.value

    def points(self):
        P = np.empty((self.rows, 3)); Q = np.empty((self.rows, 3))
        _check(lib().mf_green_points(self.ptr, _p(P, C.c_double), _p(Q, C.c_double)))
        return P, Q

    def apply(self, nrhs, d_x, d_y):
        _check(lib().mf_green_apply(self.ptr, nrhs, C.c_void_p(d_x), C.c_void_p(d_y)))

    def apply_counts(self, nrhs):
        """(flops, bytes) of one apply with nrhs vectors: bytes with each level's vectors in memory."""
        f, b = C.c_double(), C.c_double()
        _check(lib().mf_green_apply_counts(self.ptr, nrhs, C.byref(f), C.byref(b)))
        return f.value, b.value

    def __del__(self):
        if getattr(self, "ptr", None):
            lib().mf_green_destroy(self.ptr)
            self.ptr = None


class Server:
    """Continuous-batching solve server over resident factorizations (mf_server_*)."""

    def __init__(self, handles, max_batch_rhs=256, mem_budget_bytes=64 << 30):
        self.handles = list(handles)
        arr = (C.c_void_p * len(self.handles))(*[h.ptr for h in self.handles])
        self.ptr = C.c_void_p()
        _check(lib().mf_server_create(len(self.handles), arr, max_batch_rhs, mem_budget_bytes, C.byref(self.ptr)))
        self._bufs = {}

    def submit(self, problem, b):
        """b: (N, nrhs) complex128 host array; returns a request id."""
        B = np.asfortranarray(np.asarray(b, dtype=np.complex128).reshape(b.shape[0], -1))
        X = np.empty_like(B, order="F")
        rid = C.c_int64()
        _check(lib().mf_server_submit(self.ptr, problem, B.shape[1], C.c_void_p(B.ctypes.data),
                                      C.c_void_p(X.ctypes.data), C.byref(rid)))
        self._bufs[rid.value] = (B, X)
        return rid.value

    def wait(self, rid):
        info = mf_request_info()
        rc = lib().mf_server_wait(self.ptr, rid, C.byref(info))
        B, X = self._bufs.pop(rid)
        if rc not in (0, -6):
            _check(rc)
        out = {k: getattr(info, k) for k, _ in info._fields_}
        out["status"] = rc
        return X, out

    def close(self):
        if getattr(self, "ptr", None):
            lib().mf_server_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        self.close()
