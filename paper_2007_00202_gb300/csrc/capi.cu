// C ABI (include/mf.h): handle, analysis, factorization, solve with FP64
// refinement (right-preconditioned GMRES(m) with modified Gram-Schmidt, or
// iterative refinement; Sec. 6), statistics and inspection.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstddef>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/mf.h"
#include "analysis.h"
#include "bf_kernels.h"
#include "engine.h"

using mf::CudaError;
using mf::DevMem;

struct mf_handle {
  mf_options opt{};
  std::vector<int32_t> coords;
  cudaStream_t stream = nullptr;
  mf::Analysis an;
  std::string err;
  // host copy of the permuted matrix values (interleaved) for the device upload
  std::vector<double> pvals;
  std::vector<int32_t> pcol32;
  mf::DeviceMatrix A;
  bool on_device = false;
  std::unique_ptr<mf::EngineBase> eng;
  bool factored = false;
  int profile = 0;   // profiling period (0: off)
  double factor_seconds = 0;
  // solve work (FP64, new numbering)
  DevMem wb, wx, wr, wz, wV, wH, wsc, wy;
  DevMem perm_d, io_tmp, io_b, io_x;     // permutation and I/O staging of the solve calls
  int64_t io_nrhs = 0;
  int64_t work_nrhs = 0;
  int32_t work_restart = 0;
  // per-column results of the last solve (mf_solve_columns)
  std::vector<int32_t> col_iters, col_converged;
  std::vector<double> col_rel_residual;
};

namespace {

thread_local std::string g_err;

int fail(mf_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  g_err = msg;
  return code;
}

template <typename F>
int guarded(mf_handle* h, F&& fn) {
  try {
    return fn();
  } catch (const mf::SingularError& e) {
    return fail(h, MF_ERR_SINGULAR, e.what());
  } catch (const mf::TimeoutError& e) {
    return fail(h, MF_ERR_TIMEOUT, e.what());
  } catch (const CudaError& e) {
    std::string m = e.what();
    int code = (m.find("out of memory") != std::string::npos || m.find("cudaMalloc") != std::string::npos)
                   ? MF_ERR_OOM
                   : MF_ERR_CUDA;
    return fail(h, code, m);
  } catch (const std::bad_alloc&) {
    return fail(h, MF_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(h, MF_ERR_ARG, e.what());
  }
}

void ensure_device(mf_handle* h) {
  if (h->on_device) return;
  cudaStream_t st = h->stream;
  auto& A = h->A;
  A.n = h->an.n;
  A.nnz = (int64_t)h->an.pcol.size();
  mf::upload(A.rowptr, h->an.prow, st);
  mf::upload(A.col64, h->an.pcol, st);
  mf::upload(A.col32, h->pcol32, st);
  mf::upload(A.vals, h->pvals, st);
  mf::upload(h->perm_d, h->an.perm, st);
  MF_CUDA(cudaStreamSynchronize(st));
  h->on_device = true;
}

void ensure_work(mf_handle* h, int nrhs, int restart) {
  if (h->work_nrhs >= nrhs && h->work_restart >= restart) return;
  const int64_t n = h->an.n;
  size_t vec = sizeof(double) * 2 * (size_t)n * nrhs;
  h->wb.alloc(vec);
  h->wx.alloc(vec);
  h->wr.alloc(vec);
  h->wz.alloc(vec);
  h->wV.alloc(vec * (restart + 1));
  h->wH.alloc(sizeof(double) * 2 * (size_t)(restart + 2) * (restart + 1) * nrhs);
  h->wsc.alloc(sizeof(double) * 2 * (size_t)nrhs * 4);
  h->wy.alloc(sizeof(double) * 2 * (size_t)nrhs * (restart + 1));
  h->work_nrhs = nrhs;
  h->work_restart = restart;
}

using cplx = std::complex<double>;

// True residual norms ||b - A x|| per column; r receives b - A x.
void residual(mf_handle* h, const double* b, const double* x, double* r, int nrhs, std::vector<double>& nrm) {
  const int64_t n = h->an.n;
  cudaStream_t st = h->stream;
  mf::launch_spmv_residual(n, h->A.rowptr.as<int64_t>(), h->A.col32.as<int32_t>(), h->A.vals.as<double>(), x, b, r,
                           nrhs, n, st);
  double* d = h->wsc.as<double>();
  mf::launch_colnorm2(n, nrhs, r, n, d, st);
  nrm.resize(nrhs);
  MF_CUDA(cudaMemcpyAsync(nrm.data(), d, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
  MF_CUDA(cudaStreamSynchronize(st));
  for (auto& v : nrm) v = std::sqrt(v);
}

// Solve on device buffers in the new numbering: B (n x nrhs) -> X.
int solve_new_numbering(mf_handle* h, int nrhs, const double* B, double* X, mf_solve_info* info) {
  const int64_t n = h->an.n;
  cudaStream_t st = h->stream;
  const int restart = std::max(1, h->opt.gmres_restart);
  const int refine = h->opt.refine;
  ensure_work(h, nrhs, refine == MF_REFINE_GMRES ? restart : 1);
  const size_t vec = sizeof(double) * 2 * (size_t)n * nrhs;
  std::vector<double> bn;
  double* R = h->wr.as<double>();
  double* Z = h->wz.as<double>();
  // ||b||
  {
    double* d = h->wsc.as<double>();
    mf::launch_colnorm2(n, nrhs, B, n, d, st);
    bn.resize(nrhs);
    MF_CUDA(cudaMemcpyAsync(bn.data(), d, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    for (auto& v : bn) v = std::sqrt(v);
  }
  const double rtol = h->opt.rtol;
  int iters = 0;
  std::vector<double> rn;
  std::vector<int> its_col(nrhs, 0);   // iterations (or refinement steps) of each column
  auto rel_ok = [&](const std::vector<double>& r, int c) { return bn[c] == 0 || r[c] <= rtol * bn[c]; };
  h->col_iters.clear();
  h->col_converged.clear();
  h->col_rel_residual.clear();

  if (refine == MF_REFINE_NONE || refine == MF_REFINE_IR) {
    h->eng->apply_precond(B, X, nrhs);
    residual(h, B, X, R, nrhs, rn);
    if (refine == MF_REFINE_IR) {
      while (iters < h->opt.max_iters) {
        bool all = true;
        for (int c = 0; c < nrhs; ++c) all = all && rel_ok(rn, c);
        if (all) break;
        // a column's step count: the refinement steps taken while it was above rtol
        for (int c = 0; c < nrhs; ++c) its_col[c] += rel_ok(rn, c) ? 0 : 1;
        h->eng->apply_precond(R, Z, nrhs);
        // X += Z
        std::vector<double> one(2 * nrhs, 0.0);
        for (int c = 0; c < nrhs; ++c) one[2 * c] = -1.0;
        MF_CUDA(cudaMemcpyAsync(h->wsc.as<double>(), one.data(), sizeof(double) * 2 * nrhs, cudaMemcpyHostToDevice, st));
        mf::launch_colaxpy(n, nrhs, h->wsc.as<double>(), Z, n, X, n, 1.0, st);
        residual(h, B, X, R, nrhs, rn);
        ++iters;
      }
    }
  } else {
    // right-preconditioned restarted GMRES, all columns in lockstep, per-column Givens
    MF_CUDA(cudaMemsetAsync(X, 0, vec, st));
    MF_CUDA(cudaMemcpyAsync(R, B, vec, cudaMemcpyDeviceToDevice, st));
    rn = bn;
    double* V = h->wV.as<double>();
    double* Hd = h->wH.as<double>();
    double* sc = h->wsc.as<double>();
    double* yd = h->wy.as<double>();
    const size_t vstride = (size_t)2 * n * nrhs;   // doubles per Krylov vector block
    while (true) {
      std::vector<int> active;
      for (int c = 0; c < nrhs; ++c)
        if (!rel_ok(rn, c) && its_col[c] < h->opt.max_iters) active.push_back(c);
      if (active.empty()) break;
      // v0 = r / ||r||  (all columns; converged ones are carried but not used)
      std::vector<double> inv(2 * nrhs, 0.0);
      for (int c = 0; c < nrhs; ++c) inv[2 * c] = rn[c] > 0 ? 1.0 / rn[c] : 0.0;
      MF_CUDA(cudaMemcpyAsync(sc, inv.data(), sizeof(double) * 2 * nrhs, cudaMemcpyHostToDevice, st));
      mf::launch_colscale(n, nrhs, sc, R, n, V, n, st);
      std::vector<std::vector<cplx>> Hh(nrhs, std::vector<cplx>((restart + 1) * restart));
      std::vector<std::vector<cplx>> cs(nrhs, std::vector<cplx>(restart)), sn(nrhs, std::vector<cplx>(restart));
      std::vector<std::vector<cplx>> g(nrhs, std::vector<cplx>(restart + 1));
      std::vector<int> jused(nrhs, 0);
      std::vector<char> live(nrhs, 0);
      for (int c : active) { live[c] = 1; g[c][0] = rn[c]; }
      std::vector<double> hcol(2 * (restart + 1) * nrhs);
      for (int j = 0; j < restart; ++j) {
        bool any = false;
        for (int c = 0; c < nrhs; ++c) any = any || live[c];
        if (!any) break;
        double* vj = V + j * vstride;
        double* w = V + (j + 1) * vstride;
        h->eng->apply_precond(vj, Z, nrhs);
        mf::launch_spmv(n, h->A.rowptr.as<int64_t>(), h->A.col32.as<int32_t>(), h->A.vals.as<double>(), Z, w, nrhs, n,
                        st);
        // modified Gram-Schmidt
        for (int i = 0; i <= j; ++i) {
          double* hij = Hd + (size_t)2 * nrhs * (i + (restart + 1) * j);
          mf::launch_coldot(n, nrhs, V + i * vstride, n, w, n, hij, st);
          mf::launch_colaxpy(n, nrhs, hij, V + i * vstride, n, w, n, 1.0, st);
        }
        mf::launch_colnorm2(n, nrhs, w, n, sc, st);
        std::vector<double> wn(nrhs);
        MF_CUDA(cudaMemcpyAsync(wn.data(), sc, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
        MF_CUDA(cudaMemcpyAsync(hcol.data(), Hd + (size_t)2 * nrhs * (restart + 1) * j,
                                sizeof(double) * 2 * nrhs * (j + 1), cudaMemcpyDeviceToHost, st));
        MF_CUDA(cudaStreamSynchronize(st));
        std::vector<double> scl(2 * nrhs, 0.0);
        for (int c = 0; c < nrhs; ++c) {
          double hn = std::sqrt(wn[c]);
          scl[2 * c] = hn > 0 ? 1.0 / hn : 0.0;
          if (!live[c]) continue;
          auto& H = Hh[c];
          for (int i = 0; i <= j; ++i)
            H[i + (restart + 1) * j] = cplx(hcol[2 * (nrhs * i + c)], hcol[2 * (nrhs * i + c) + 1]);
          H[j + 1 + (restart + 1) * j] = hn;
          // complex Givens rotations G_i = [[conj(c), conj(s)], [-s, c]], c = a / d, s = b / d,
          // d = sqrt(|a|^2 + |b|^2): G_i (a, b) = (d, 0), so G H is upper triangular
          for (int i = 0; i < j; ++i) {
            cplx a = H[i + (restart + 1) * j], bb = H[i + 1 + (restart + 1) * j];
            H[i + (restart + 1) * j] = std::conj(cs[c][i]) * a + std::conj(sn[c][i]) * bb;
            H[i + 1 + (restart + 1) * j] = -sn[c][i] * a + cs[c][i] * bb;
          }
          cplx a = H[j + (restart + 1) * j], bb = H[j + 1 + (restart + 1) * j];
          double den = std::sqrt(std::norm(a) + std::norm(bb));
          cs[c][j] = den > 0 ? a / den : cplx(1);
          sn[c][j] = den > 0 ? bb / den : cplx(0);
          H[j + (restart + 1) * j] = den > 0 ? cplx(den) : a;
          H[j + 1 + (restart + 1) * j] = 0;
          g[c][j + 1] = -sn[c][j] * g[c][j];
          g[c][j] = std::conj(cs[c][j]) * g[c][j];
          jused[c] = j + 1;
          its_col[c]++;
          if (std::abs(g[c][j + 1]) <= rtol * bn[c] || its_col[c] >= h->opt.max_iters || hn == 0) live[c] = 0;
        }
        MF_CUDA(cudaMemcpyAsync(sc, scl.data(), sizeof(double) * 2 * nrhs, cudaMemcpyHostToDevice, st));
        mf::launch_colscale(n, nrhs, sc, w, n, w, n, st);
        iters = std::max(iters, j + 1);
      }
      // y = H^-1 g per column; t = V y ; X += M^-1 t
      int jmax = 0;
      for (int c : active) jmax = std::max(jmax, jused[c]);
      std::vector<double> yh(2 * (size_t)nrhs * jmax, 0.0);
      for (int c : active) {
        int m = jused[c];
        std::vector<cplx> y(m);
        for (int i = m - 1; i >= 0; --i) {
          cplx acc = g[c][i];
          for (int k = i + 1; k < m; ++k) acc -= Hh[c][i + (restart + 1) * k] * y[k];
          y[i] = acc / Hh[c][i + (restart + 1) * i];
        }
        for (int i = 0; i < m; ++i) {
          yh[2 * ((size_t)nrhs * i + c)] = -y[i].real();
          yh[2 * ((size_t)nrhs * i + c) + 1] = -y[i].imag();
        }
      }
      MF_CUDA(cudaMemcpyAsync(yd, yh.data(), sizeof(double) * yh.size(), cudaMemcpyHostToDevice, st));
      MF_CUDA(cudaMemsetAsync(R, 0, vec, st));
      for (int i = 0; i < jmax; ++i)
        mf::launch_colaxpy(n, nrhs, yd + (size_t)2 * nrhs * i, V + i * vstride, n, R, n, 1.0, st);
      h->eng->apply_precond(R, Z, nrhs);
      std::vector<double> one(2 * nrhs, 0.0);
      for (int c = 0; c < nrhs; ++c) one[2 * c] = -1.0;
      MF_CUDA(cudaMemcpyAsync(sc, one.data(), sizeof(double) * 2 * nrhs, cudaMemcpyHostToDevice, st));
      mf::launch_colaxpy(n, nrhs, sc, Z, n, X, n, 1.0, st);
      residual(h, B, X, R, nrhs, rn);
      iters = 0;
      for (int c = 0; c < nrhs; ++c) iters = std::max(iters, its_col[c]);
    }
    if (rn.size() != (size_t)nrhs) residual(h, B, X, R, nrhs, rn);
  }
  MF_CUDA(cudaGetLastError());
  double worst = 0;
  bool conv = true;
  for (int c = 0; c < nrhs; ++c) {
    double rr = bn[c] > 0 ? rn[c] / bn[c] : 0.0;
    worst = std::max(worst, rr);
    conv = conv && rel_ok(rn, c);
  }
  if (info) {
    info->iters = iters;
    info->converged = conv ? 1 : 0;
    info->max_rel_residual = worst;
  }
  h->col_iters.assign(its_col.begin(), its_col.end());
  h->col_converged.resize(nrhs);
  h->col_rel_residual.resize(nrhs);
  for (int c = 0; c < nrhs; ++c) {
    h->col_converged[c] = rel_ok(rn, c) ? 1 : 0;
    h->col_rel_residual[c] = bn[c] > 0 ? rn[c] / bn[c] : 0.0;
  }
  if (!conv && refine != MF_REFINE_NONE)
    return fail(h, MF_ERR_NO_CONVERGENCE, "refinement stopped above rtol (max rel. residual " + std::to_string(worst) + ")");
  return MF_OK;
}

}  // namespace

extern "C" {

int mf_options_init(mf_options* o) {
  if (!o) return fail(nullptr, MF_ERR_ARG, "opt is NULL");
  std::memset(o, 0, sizeof(*o));
  o->version = MF_OPTIONS_V2;
  o->leaf_size = 64;
  o->nmin_sep = 1024;
  o->hodbf_leaf = 64;
  o->max_rank = 0;
  o->alpha = 2;
  o->knn = 8;
  o->precision = MF_PREC_C64;
  o->refine = MF_REFINE_GMRES;
  o->gmres_restart = 30;
  o->max_iters = 300;
  o->lattice = MF_LATTICE_NODE;
  o->rtol = 1e-8;
  o->seed = 1;
  o->coords = nullptr;
  o->ordering = MF_ORDER_AUTO;
  return MF_OK;
}

int mf_analyze(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* vals, const mf_options* opt,
               void* cuda_stream, mf_handle** out) {
  if (!out) return fail(nullptr, MF_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!opt || (opt->version != MF_OPTIONS_V1 && opt->version != MF_OPTIONS_V2))
    return fail(nullptr, MF_ERR_ARG, "options missing or wrong version");
  const int ordering = opt->version >= MF_OPTIONS_V2 ? opt->ordering : MF_ORDER_AUTO;   // V1 structs end at coords
  if (n <= 0 || !rowptr || !colind || !vals) return fail(nullptr, MF_ERR_ARG, "invalid CSR arguments");
  std::unique_ptr<mf_handle> h(new (std::nothrow) mf_handle());
  if (!h) return fail(nullptr, MF_ERR_OOM, "host allocation failed");
  int rc = guarded(h.get(), [&]() -> int {
    if (opt->version >= MF_OPTIONS_V2) {
      h->opt = *opt;
    } else {   // a version-1 struct ends at coords
      std::memset(&h->opt, 0, sizeof(h->opt));
      std::memcpy(&h->opt, opt, offsetof(mf_options, ordering));
      h->opt.version = MF_OPTIONS_V2;
      h->opt.ordering = MF_ORDER_AUTO;
    }
    if (opt->coords) {
      h->coords.assign(opt->coords, opt->coords + 3 * n);
      h->opt.coords = h->coords.data();
    }
    h->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    try {
      // with lattice coordinates: planar separators; without: graph nested dissection
      mf::analyze(n, rowptr, colind, opt->coords ? h->coords.data() : nullptr, opt->lattice, opt->leaf_size,
                  opt->nmin_sep, opt->hodbf_leaf, h->an, ordering,
                  opt->version >= MF_OPTIONS_V2 ? opt->parallel_levels : 0);
    } catch (const std::runtime_error& e) {
      std::string m = e.what();
      if (m.find("empty separator") != std::string::npos) return fail(h.get(), MF_ERR_UNSUPPORTED, m);
      return fail(h.get(), MF_ERR_ARG, m);
    }
    // permuted values, aligned with the permuted (sorted) pattern
    const auto& an = h->an;
    h->pvals.resize(2 * an.pcol.size());
    h->pcol32.resize(an.pcol.size());
    std::vector<std::pair<int64_t, int64_t>> row;
    for (int64_t r = 0; r < n; ++r) {
      int64_t o = an.perm[r];
      row.clear();
      for (int64_t k = rowptr[o]; k < rowptr[o + 1]; ++k) row.push_back({an.iperm[colind[k]], k});
      std::sort(row.begin(), row.end());
      int64_t p = an.prow[r];
      for (auto& e : row) {
        h->pvals[2 * p] = vals[2 * e.second];
        h->pvals[2 * p + 1] = vals[2 * e.second + 1];
        h->pcol32[p] = (int32_t)e.first;
        ++p;
      }
    }
    return MF_OK;
  });
  if (rc != MF_OK) return rc;
  *out = h.release();
  return MF_OK;
}

int mf_factor(mf_handle* h, double tol) {
  if (!h) return fail(nullptr, MF_ERR_ARG, "handle is NULL");
  if (!(tol > 0) && !(tol == 0)) return fail(h, MF_ERR_ARG, "tol must be >= 0");
  return guarded(h, [&]() -> int {
    auto t0 = std::chrono::steady_clock::now();
    ensure_device(h);
    if (!h->eng) {
      mf::EngineOptions eo;
      eo.max_rank = h->opt.max_rank;
      eo.alpha = h->opt.alpha;
      eo.knn = h->opt.knn;
      eo.seed = h->opt.seed;
      bool any_comp = false;
      size_t comp_n = 0, max_n = 0;
      for (auto& f : h->an.fronts)
        if (f.compressed) {
          any_comp = true;
          comp_n += (size_t)(f.s() + f.u());
          max_n = std::max(max_n, (size_t)(f.s() + f.u()));
        }
      // arenas for the compressed fronts, sized from their dimensions: one persistent arena for every
      // compressed front's factors, and per construction context a work arena for the largest front
      // (released after each front)
      size_t el = h->opt.precision == MF_PREC_C128 ? 16 : 8;
      // without a rank cap the sketch widths may double several times: give the work arena room
      // (measured work of one front: 1.6 GB at s + u = 6144 (64^3), more than 9.6 GB at 15000 (100^3))
      const size_t per = h->opt.max_rank > 0 ? 320000 : 1280000;
      eo.persist_bytes = any_comp ? std::max<size_t>(size_t(4) << 30, comp_n * 24000 * el) : 0;
      eo.scratch_bytes = any_comp ? std::max<size_t>(size_t(2) << 30, max_n * per * el) : 0;
      // the persistent arena takes at most 40 % of the free memory; as many work arenas as fit in
      // 70 % of it beside it (1 to 8) set the number of construction contexts
      size_t fr = 0, tot = 0;
      if (any_comp && cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
        const double room = 0.7 * (double)fr;
        eo.persist_bytes = std::min(eo.persist_bytes, (size_t)(0.4 * (double)fr));
        const double left = room - (double)eo.persist_bytes;
        int nc = (int)(left / (double)eo.scratch_bytes);
        if (nc < 1) {
          nc = 1;
          eo.scratch_bytes = (size_t)std::max(0.0, left);
        }
        eo.max_contexts = std::min(nc, 8);
      }
      h->eng = h->opt.precision == MF_PREC_C128 ? mf::make_engine_c128(h->an, h->A, h->stream, eo)
                                               : mf::make_engine_c64(h->an, h->A, h->stream, eo);
      h->eng->set_profiling(h->profile);
    }
    h->factored = false;
    h->eng->factor(tol);
    h->factored = true;
    h->factor_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return MF_OK;
  });
}

int mf_solve_device(mf_handle* h, int32_t nrhs, const void* d_b, void* d_x, mf_solve_info* info) {
  if (!h) return fail(nullptr, MF_ERR_ARG, "handle is NULL");
  if (!h->factored) return fail(h, MF_ERR_STATE, "mf_solve before mf_factor");
  if (nrhs <= 0 || !d_b || !d_x) return fail(h, MF_ERR_ARG, "invalid solve arguments");
  return guarded(h, [&]() -> int {
    const int64_t n = h->an.n;
    ensure_work(h, nrhs, h->opt.refine == MF_REFINE_GMRES ? std::max(1, h->opt.gmres_restart) : 1);
    cudaStream_t st = h->stream;
    // permute into the new numbering: wb[new] = b[perm[new]]
    double* B = h->wb.as<double>();
    double* X = h->wx.as<double>();
    const int64_t* perm = h->perm_d.as<int64_t>();
    if (h->io_nrhs < nrhs) {
      h->io_tmp.alloc(sizeof(double) * 2 * n * nrhs);
      h->io_b.alloc(sizeof(double) * 2 * n * nrhs);
      h->io_x.alloc(sizeof(double) * 2 * n * nrhs);
      h->io_nrhs = nrhs;
    }
    DevMem& tmp = h->io_tmp;
    mf::launch_to_planar<double>(static_cast<const double*>(d_b), n, n, nrhs, perm, tmp.as<double>(), n * nrhs, st);
    mf::launch_from_planar<double>(tmp.as<double>(), n * nrhs, n, nrhs, nullptr, B, n, st);
    int rc = solve_new_numbering(h, nrhs, B, X, info);
    mf::launch_to_planar<double>(X, n, n, nrhs, nullptr, tmp.as<double>(), n * nrhs, st);
    mf::launch_from_planar<double>(tmp.as<double>(), n * nrhs, n, nrhs, perm, static_cast<double*>(d_x), n, st);
    MF_CUDA(cudaStreamSynchronize(st));
    return rc;
  });
}

int mf_solve(mf_handle* h, int32_t nrhs, const double* b, int64_t ldb, double* x, int64_t ldx, mf_solve_info* info) {
  if (!h) return fail(nullptr, MF_ERR_ARG, "handle is NULL");
  if (!h->factored) return fail(h, MF_ERR_STATE, "mf_solve before mf_factor");
  const int64_t n = h->an.n;
  if (nrhs <= 0 || !b || !x || ldb < n || ldx < n) return fail(h, MF_ERR_ARG, "invalid solve arguments");
  return guarded(h, [&]() -> int {
    cudaStream_t st = h->stream;
    if (h->io_nrhs < nrhs) {
      h->io_tmp.alloc(sizeof(double) * 2 * n * nrhs);
      h->io_b.alloc(sizeof(double) * 2 * n * nrhs);
      h->io_x.alloc(sizeof(double) * 2 * n * nrhs);
      h->io_nrhs = nrhs;
    }
    DevMem& db = h->io_b;
    DevMem& dx = h->io_x;
    MF_CUDA(cudaMemcpy2DAsync(db.p, sizeof(double) * 2 * n, b, sizeof(double) * 2 * ldb, sizeof(double) * 2 * n, nrhs,
                              cudaMemcpyHostToDevice, st));
    int rc = mf_solve_device(h, nrhs, db.p, dx.p, info);
    if (rc != MF_OK && rc != MF_ERR_NO_CONVERGENCE) return rc;
    MF_CUDA(cudaMemcpy2DAsync(x, sizeof(double) * 2 * ldx, dx.p, sizeof(double) * 2 * n, sizeof(double) * 2 * n, nrhs,
                              cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    return rc;
  });
}

int mf_solve_columns(const mf_handle* h, int32_t nrhs, int32_t* iters, int32_t* converged, double* rel_residual) {
  if (!h) return fail(nullptr, MF_ERR_ARG, "handle is NULL");
  if (h->col_iters.empty()) return fail(const_cast<mf_handle*>(h), MF_ERR_STATE, "no solve has run on this handle");
  if (nrhs != (int32_t)h->col_iters.size())
    return fail(const_cast<mf_handle*>(h), MF_ERR_ARG, "nrhs differs from the last solve's");
  for (int c = 0; c < nrhs; ++c) {
    if (iters) iters[c] = h->col_iters[c];
    if (converged) converged[c] = h->col_converged[c];
    if (rel_residual) rel_residual[c] = h->col_rel_residual[c];
  }
  return MF_OK;
}

int mf_stats(const mf_handle* h, mf_stats_t* out) {
  if (!h || !out) return fail(const_cast<mf_handle*>(h), MF_ERR_ARG, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  out->n = h->an.n;
  out->nfronts = (int64_t)h->an.fronts.size();
  int lv = 0;
  for (auto& f : h->an.fronts) {
    out->ncompressed += f.compressed ? 1 : 0;
    lv = std::max(lv, f.level + 1);
  }
  out->tree_levels = lv;
  out->precision = h->opt.precision;
  if (h->eng) {
    out->factor_flops = h->eng->factor_flops();
    out->factor_bytes = h->eng->factor_bytes();
    h->eng->arena_usage(out->arena_peak_bytes, out->arena_capacity_bytes);
    out->gpu_launches_factor = h->eng->launches_factor();
    out->max_rank = h->eng->max_rank();
  }
  out->factor_seconds = h->factor_seconds;
  return MF_OK;
}

int mf_profile(mf_handle* h, int32_t enable) {
  if (!h) return fail(nullptr, MF_ERR_ARG, "handle is NULL");
  if (enable < 0) return fail(h, MF_ERR_ARG, "enable must be >= 0");
  h->profile = enable;
  if (h->eng) return guarded(h, [&]() -> int {
    h->eng->set_profiling(h->profile);
    return MF_OK;
  });
  return MF_OK;
}

int mf_profile_read(mf_handle* h, int32_t kernel, mf_kernel_profile_t* out) {
  if (!h || !out) return fail(h, MF_ERR_ARG, "NULL argument");
  if (kernel != MF_PROF_NARROW_GEMM && kernel != MF_PROF_FRONT_GEMM) return fail(h, MF_ERR_ARG, "unknown kernel");
  std::memset(out, 0, sizeof(*out));
  if (!h->eng) return MF_OK;
  return guarded(h, [&]() -> int {
    mf::LaunchProfiler& p = h->eng->prof[kernel];
    p.collect();
    out->launches = p.launches;
    out->ms = p.ms;
    out->flops = p.flops;
    out->bytes = p.bytes;
    return MF_OK;
  });
}

int mf_gemm_c64(int32_t engine, int32_t m, int32_t n, int32_t k, const float* A, int64_t lda, int64_t pla,
                const float* B, int64_t ldb, int64_t plb, float* C, int64_t ldc, int64_t plc, float alpha, float beta,
                void* stream) {
  if (m <= 0 || n <= 0 || k <= 0 || !A || !B || !C || lda < k || ldb < k || ldc < n)
    return fail(nullptr, MF_ERR_ARG, "invalid GEMM arguments");
  if (engine < 0 || engine > 2) return fail(nullptr, MF_ERR_ARG, "engine must be 0, 1 or 2");
  if (engine >= 1 && ((lda | ldb | pla | plb) % 4 != 0 || ((uintptr_t)A | (uintptr_t)B) % 16 != 0))
    return fail(nullptr, MF_ERR_ARG, "tensor-core GEMM needs 16-byte aligned operands (ld, plane % 4 == 0)");
  return guarded(nullptr, [&]() -> int {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    mf::GemmDesc<float> d;
    d.m = m; d.n = n; d.k = k; d.transA = 0; d.transB = 1; d.alpha = alpha; d.beta = beta;
    d.A = {const_cast<float*>(A), pla, lda};
    d.B = {const_cast<float*>(B), plb, ldb};
    d.C = {C, plc, ldc};
    int tile = engine >= 1 ? mf::gemm_tc_tile() : mf::GEMM_TILE;
    std::vector<mf::GemmTile> tl;
    for (int i = 0; i < (m + tile - 1) / tile; ++i)
      for (int j = 0; j < (n + tile - 1) / tile; ++j) tl.push_back({0, i, j, 0});
    DevMem dd, dt, ds;
    mf::upload(dd, std::vector<mf::GemmDesc<float>>{d}, st);
    mf::upload(dt, tl, st);
    ds.alloc(sizeof(int32_t));
    MF_CUDA(cudaMemsetAsync(ds.p, 0, sizeof(int32_t), st));
    if (engine >= 1) mf::launch_gemm_tc(dd.as<mf::GemmDesc<float>>(), dt.as<mf::GemmTile>(), (int)tl.size(),
                                        ds.as<int32_t>(), st, engine == 2);
    else mf::launch_gemm<float>(dd.as<mf::GemmDesc<float>>(), dt.as<mf::GemmTile>(), (int)tl.size(), st);
    MF_CUDA(cudaGetLastError());
    int32_t stat = 0;
    MF_CUDA(cudaMemcpyAsync(&stat, ds.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    if (stat) return fail(nullptr, MF_ERR_TIMEOUT, "a bounded wait in the tensor-core GEMM expired");
    return MF_OK;
  });
}

int mf_gemm_nrhs_c64(int32_t trans_a, int32_t m, int32_t n, int32_t k, const float* A, int64_t lda, int64_t pla,
                     const float* B, int64_t ldb, int64_t plb, float* C, int64_t ldc, int64_t plc, float alpha,
                     float beta, int32_t ksplit, void* stream) {
  if (m <= 0 || n <= 0 || n > 128 || k <= 0 || !A || !B || !C || (trans_a != 0 && trans_a != 1) ||
      lda < (trans_a ? m : k) || ldb < n || ldc < n)
    return fail(nullptr, MF_ERR_ARG, "invalid narrow-GEMM arguments");
  if (ksplit != -1 && ksplit != 0 && ksplit != 1 && ksplit != 2 && ksplit != 4 && ksplit != 8)
    return fail(nullptr, MF_ERR_ARG, "ksplit must be -1, 0, 1, 2, 4 or 8");
  if (ksplit == -1 && n > 64) return fail(nullptr, MF_ERR_ARG, "the tensor-core kernel takes n <= 64");
  return guarded(nullptr, [&]() -> int {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    mf::GemmDesc<float> d;
    d.m = m; d.n = n; d.k = k; d.transA = trans_a; d.transB = 0; d.alpha = alpha; d.beta = beta;
    d.A = {const_cast<float*>(A), pla, lda};
    d.B = {const_cast<float*>(B), plb, ldb};
    d.C = {C, plc, ldc};
    std::vector<mf::GemmTile> tl;
    if (ksplit == -1) {
      const int tr = mf::gemm_nrhs_tc_rows();
      for (int i = 0; i < (m + tr - 1) / tr; ++i) tl.push_back({0, i, 0, 0});
      DevMem dd, dt, ds;
      mf::upload(dd, std::vector<mf::GemmDesc<float>>{d}, st);
      mf::upload(dt, tl, st);
      ds.alloc(sizeof(int32_t));
      MF_CUDA(cudaMemsetAsync(ds.p, 0, sizeof(int32_t), st));
      mf::launch_gemm_nrhs_tc(dd.as<mf::GemmDesc<float>>(), dt.as<mf::GemmTile>(), (int)tl.size(), ds.as<int32_t>(), st);
      MF_CUDA(cudaGetLastError());
      int32_t stat = 0;
      MF_CUDA(cudaMemcpyAsync(&stat, ds.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      MF_CUDA(cudaStreamSynchronize(st));
      if (stat) return fail(nullptr, MF_ERR_TIMEOUT, "a bounded wait in the tensor-core kernel expired");
      return MF_OK;
    }
    const int nb = mf::gemm_nrhs_width(n, sizeof(float));
    for (int i = 0; i < (m + mf::GEMM_NRHS_ROWS - 1) / mf::GEMM_NRHS_ROWS; ++i)
      for (int j = 0; j < (n + nb - 1) / nb; ++j) tl.push_back({0, i, j, 0});
    const int ks = ksplit ? ksplit : mf::gemm_nrhs_split((int)tl.size(), k);
    DevMem dd, dt;
    mf::upload(dd, std::vector<mf::GemmDesc<float>>{d}, st);
    mf::upload(dt, tl, st);
    mf::launch_gemm_nrhs<float>(dd.as<mf::GemmDesc<float>>(), dt.as<mf::GemmTile>(), (int)tl.size(), nb, ks, k, st);
    MF_CUDA(cudaGetLastError());
    MF_CUDA(cudaStreamSynchronize(st));
    return MF_OK;
  });
}

int mf_row_id_c64(int32_t nmat, int32_t m, int32_t n, const float* M, double tol, int32_t max_rank, float* U,
                  int32_t* sk, int32_t* rank, void* stream) {
  if (nmat <= 0 || m <= 0 || n <= 0 || m > 2048 || n > 8192 || !M || !U || !sk || !rank || !(tol >= 0))
    return fail(nullptr, MF_ERR_ARG, "invalid row-ID arguments");
  return guarded(nullptr, [&]() -> int {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int kmax = std::min(m, n);
    if (max_rank > 0) kmax = std::min(kmax, (int)max_rank);
    DevMem work, jobs;
    const bool in_smem = (m <= 128 && n <= 128) || mf::row_id_smem_bytes(m, n, sizeof(float), true) <= mf::kRowIdSmemCap;
    if (!in_smem) work.alloc(sizeof(float) * 2 * (size_t)m * n * nmat);
    std::vector<mf::IdJob<float>> jb(nmat);
    for (int q = 0; q < nmat; ++q) {
      auto& j = jb[q];
      j.M = M + (size_t)2 * m * n * q;
      j.plane = (int64_t)m * n;
      j.ld = n;
      j.m = m;
      j.n = n;
      j.U = U + (size_t)2 * m * kmax * q;
      j.uplane = (int64_t)m * kmax;
      j.ldu = kmax;
      j.sk = sk + (size_t)kmax * q;
      j.rank = rank + q;
      j.work = in_smem ? nullptr : work.as<float>() + (size_t)2 * m * n * q;
      j.wplane = (int64_t)m * n;
    }
    mf::upload(jobs, jb, st);
    if (m <= 128 && n <= 128) {   // the solver's register-resident kernel for small blocks
      if (mf::launch_row_id_reg<float>(jobs.as<mf::IdJob<float>>(), nmat, m, n, (float)tol, max_rank, st) != 0)
        return fail(nullptr, MF_ERR_ARG, "matrix too large for the row-ID kernel");
    } else if (mf::launch_row_id<float>(jobs.as<mf::IdJob<float>>(), nmat, m, n, (float)tol, max_rank, st, in_smem) != 0)
      return fail(nullptr, MF_ERR_ARG, "matrix too large for the row-ID kernel");
    MF_CUDA(cudaGetLastError());
    MF_CUDA(cudaStreamSynchronize(st));
    return MF_OK;
  });
}

int64_t mf_launch_counter(void) { return mf::launch_count(); }

const char* mf_last_error(const mf_handle* h) { return h ? h->err.c_str() : g_err.c_str(); }

void mf_destroy(mf_handle* h) {
  if (!h) return;
  delete h;
}

int mf_analysis_sizes(const mf_handle* h, mf_analysis_sizes_t* out) {
  if (!h || !out) return fail(const_cast<mf_handle*>(h), MF_ERR_ARG, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  out->n = h->an.n;
  out->nfronts = (int64_t)h->an.fronts.size();
  for (auto& f : h->an.fronts) {
    out->upd_total += f.u();
    for (auto& l : f.th_tree) out->tree_total += (int64_t)l.size();
    for (auto& l : f.f22_tree) out->tree_total += (int64_t)l.size();
  }
  return MF_OK;
}

int mf_analysis_export(const mf_handle* h, int64_t* perm, int64_t* front_parent, int64_t* front_sep,
                       int32_t* front_flags, int64_t* upd_ptr, int64_t* upd_idx) {
  if (!h) return fail(nullptr, MF_ERR_ARG, "handle is NULL");
  const auto& an = h->an;
  if (perm) std::copy(an.perm.begin(), an.perm.end(), perm);
  int64_t p = 0;
  if (upd_ptr) upd_ptr[0] = 0;
  for (size_t i = 0; i < an.fronts.size(); ++i) {
    const auto& f = an.fronts[i];
    if (front_parent) front_parent[i] = f.parent;
    if (front_sep) { front_sep[2 * i] = f.sep_begin; front_sep[2 * i + 1] = f.sep_end; }
    if (front_flags) front_flags[i] = f.compressed ? 1 : 0;
    if (upd_idx) std::copy(f.upd.begin(), f.upd.end(), upd_idx + p);
    p += f.u();
    if (upd_ptr) upd_ptr[i + 1] = p;
  }
  return MF_OK;
}

int mf_set_wait_limit(int64_t spins) {
  if (spins < 0) return fail(nullptr, MF_ERR_ARG, "spins must be >= 0");
  mf::set_wait_limit((long long)spins);
  return MF_OK;
}

int mf_front_apply(mf_handle* h, int64_t f, int32_t which, int32_t nrhs, const double* x, double* y) {
  if (!h || !x || !y || nrhs <= 0) return fail(h, MF_ERR_ARG, "invalid argument");
  if (!h->factored) return fail(h, MF_ERR_STATE, "mf_front_apply before mf_factor");
  if (f < 0 || f >= (int64_t)h->an.fronts.size()) return fail(h, MF_ERR_ARG, "bad front id");
  return guarded(h, [&]() -> int {
    if (h->eng->front_apply((int)f, which, nrhs, x, y) != 0)
      return fail(h, MF_ERR_ARG, "front is not compressed or has no such operator");
    return MF_OK;
  });
}

int mf_front_trees(const mf_handle* h, int64_t f, int64_t* nlev, int64_t* ranges) {
  if (!h || !nlev) return fail(const_cast<mf_handle*>(h), MF_ERR_ARG, "NULL argument");
  if (f < 0 || f >= (int64_t)h->an.fronts.size()) return fail(const_cast<mf_handle*>(h), MF_ERR_ARG, "bad front id");
  const auto& fr = h->an.fronts[f];
  nlev[0] = (int64_t)fr.th_tree.size();
  nlev[1] = (int64_t)fr.f22_tree.size();
  if (ranges) {
    int64_t p = 0;
    for (auto* t : {&fr.th_tree, &fr.f22_tree})
      for (auto& l : *t)
        for (auto& r : l) { ranges[p++] = r.a; ranges[p++] = r.b; }
  }
  return MF_OK;
}

int mf_front_neighbours(const mf_handle* h, int64_t f, int32_t knn, int64_t* counts, int64_t* ptr, int64_t* idx) {
  if (!h || !counts || knn < 0) return fail(const_cast<mf_handle*>(h), MF_ERR_ARG, "invalid argument");
  if (f < 0 || f >= (int64_t)h->an.fronts.size()) return fail(const_cast<mf_handle*>(h), MF_ERR_ARG, "bad front id");
  return guarded(const_cast<mf_handle*>(h), [&]() -> int {
    mf::FrontNeighbours nb;
    mf::front_neighbours(h->an, h->an.fronts[f], knn, nb);
    const std::vector<int64_t>* P[4] = {&nb.nn11_ptr, &nb.nn22_ptr, &nb.nn12_ptr, &nb.nn21_ptr};
    const std::vector<int64_t>* I[4] = {&nb.nn11, &nb.nn22, &nb.nn12, &nb.nn21};
    for (int k = 0; k < 4; ++k) counts[k] = (int64_t)I[k]->size();
    if (ptr) {
      int64_t p = 0;
      for (int k = 0; k < 4; ++k)
        for (int64_t v : *P[k]) ptr[p++] = v;
    }
    if (idx) {
      int64_t p = 0;
      for (int k = 0; k < 4; ++k)
        for (int64_t v : *I[k]) idx[p++] = v;
    }
    return MF_OK;
  });
}

}  // extern "C"
