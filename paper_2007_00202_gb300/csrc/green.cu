// Sets of HOD-BF compressed blocks of the 3-D Helmholtz Green's function
// G(x, y) = exp(i k |x - y|) / (4 pi |x - y|) between two parallel m x m point
// grids (Sec. 3.1 names this kernel as the model of butterfly-compressible
// interactions).  Every block is built on the GPU by HOD-BF entry evaluation
// (Sec. 4.1: Alg. 2 on all off-diagonal blocks, all blocks of all matrices with
// the same level count in lockstep) and applied to blocks of vectors.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "../../include/mf.h"
#include "bf_engine.h"

namespace mf {

namespace {

template <typename T>
struct GreenJob {
  const int32_t* X;
  const int32_t* Y;
  int32_t nx, ny;
  T* dst;
  int64_t dplane, dld;
};

template <typename T>
__global__ void k_green(const GreenJob<T>* jobs, const double* P, const double* Q, double k) {
  const GreenJob<T> j = jobs[blockIdx.y];
  const int64_t total = (int64_t)j.nx * j.ny;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / j.ny), b = (int)(e % j.ny);
    const int x = j.X[a], y = j.Y[b];
    const double dx = P[3 * x] - Q[3 * y], dy = P[3 * x + 1] - Q[3 * y + 1], dz = P[3 * x + 2] - Q[3 * y + 2];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    double sn, cs;
    sincos(k * r, &sn, &cs);
    const double s = 1.0 / (4.0 * 3.14159265358979323846 * r);
    j.dst[(int64_t)a * j.dld + b] = (T)(cs * s);
    j.dst[(int64_t)a * j.dld + b + j.dplane] = (T)(sn * s);
  }
}

// geometric bisection of 2-D lattice points (uniform depth), as the separator reordering of Sec. 5.1
void cluster2d(const std::vector<std::array<int64_t, 2>>& pts, int64_t leaf, std::vector<int64_t>& order, Tree& lv) {
  std::vector<std::vector<int64_t>> cl(1);
  for (size_t i = 0; i < pts.size(); ++i) cl[0].push_back((int64_t)i);
  std::vector<std::vector<std::vector<int64_t>>> hist{cl};
  for (;;) {
    size_t mx = 0;
    for (auto& c : cl) mx = std::max(mx, c.size());
    if ((int64_t)mx <= leaf) break;
    std::vector<std::vector<int64_t>> nw;
    for (auto& c : cl) {
      if (c.empty()) { nw.emplace_back(); nw.emplace_back(); continue; }
      std::array<int64_t, 2> lo = pts[c[0]], hi = pts[c[0]];
      for (int64_t id : c)
        for (int d = 0; d < 2; ++d) { lo[d] = std::min(lo[d], pts[id][d]); hi[d] = std::max(hi[d], pts[id][d]); }
      int a = (hi[1] - lo[1] > hi[0] - lo[0]) ? 1 : 0;
      int64_t cut = lo[a] + (hi[a] - lo[a] + 1) / 2;
      std::vector<int64_t> l, r;
      for (int64_t id : c) (pts[id][a] < cut ? l : r).push_back(id);
      nw.push_back(l);
      nw.push_back(r);
    }
    cl.swap(nw);
    hist.push_back(cl);
  }
  lv.clear();
  for (auto& h : hist) {
    std::vector<Range> rs;
    int64_t p = 0;
    for (auto& c : h) { rs.push_back({p, p + (int64_t)c.size()}); p += (int64_t)c.size(); }
    lv.push_back(rs);
  }
  order.clear();
  for (auto& c : cl) order.insert(order.end(), c.begin(), c.end());
}

}  // namespace
}  // namespace mf

// The apply for one (nrhs, x, y): eager on its first call (sizing the job tables), captured into a
// CUDA graph on a private stream on the second, replayed afterwards (state 3: eager only).
struct GreenPlan {
  int32_t nrhs = 0;
  const float* x = nullptr;
  float* y = nullptr;
  int state = 0;
  size_t blob = 0, mark = 0;
  char* hblob = nullptr;
  mf::DevMem dblob;
  cudaGraphExec_t exec = nullptr;
  int glaunch = 0;
  double flops = 0, bytes = 0;   // counted over the eager first call
  ~GreenPlan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (hblob) cudaFreeHost(hblob);
  }
};

struct mf_bfset {
  ~mf_bfset() {
    plans.clear();
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
    if (gs) cudaStreamDestroy(gs);
  }
  cudaStream_t st = nullptr;
  cudaStream_t gs = nullptr;          // stream of the apply graphs (forked from and joined to st)
  cudaEvent_t ev[2] = {nullptr, nullptr};
  std::vector<std::unique_ptr<GreenPlan>> plans;
  std::unique_ptr<mf::BFContext<float>> cx;
  std::vector<std::unique_ptr<mf::DHODBF<float>>> H;
  std::vector<int64_t> off;
  int64_t rows = 0;
  std::vector<double> P, Q;   // host copies, set row order
  mf::DevMem dP, dQ;
  double build_seconds = 0, k = 0;
  std::string err;
};

using mf::Blk;

extern "C" {

int mf_green_build(int32_t nblk, const int32_t* m, double k, double spacing, double tol, int32_t leaf,
                   int32_t max_rank, int32_t alpha, int32_t knn, void* stream, mf_bfset** out) {
  if (!out || nblk <= 0 || !m || leaf < 4 || !(tol > 0) || !(spacing > 0)) return MF_ERR_ARG;
  *out = nullptr;
  for (int b = 0; b < nblk; ++b)
    if (m[b] < 2 || m[b] > 512) return MF_ERR_ARG;
  auto s = std::make_unique<mf_bfset>();
  try {
    auto t0 = std::chrono::steady_clock::now();
    s->st = reinterpret_cast<cudaStream_t>(stream);
    s->k = k;
    std::vector<mf::HProblem<float>> probs(nblk);
    std::vector<std::vector<mf::IdxVec>> nns(nblk);   // the problems' neighbour lists (kept for the build)
    int64_t off = 0;
    for (int b = 0; b < nblk; ++b) {
      const int mb = m[b];
      std::vector<std::array<int64_t, 2>> pts;
      for (int j = 0; j < mb; ++j)
        for (int i = 0; i < mb; ++i) pts.push_back({i, j});
      std::vector<int64_t> order;
      mf::Tree tree;
      mf::cluster2d(pts, leaf, order, tree);
      const int n = mb * mb;
      std::vector<int64_t> pos(n);
      for (int t = 0; t < n; ++t) pos[order[t]] = t;
      for (int t = 0; t < n; ++t) {
        const auto& p = pts[order[t]];
        s->P.insert(s->P.end(), {p[0] * spacing, p[1] * spacing, 0.0});
        s->Q.insert(s->Q.end(), {p[0] * spacing, p[1] * spacing, spacing});
      }
      // geometric nearest neighbours (in-plane distance), in set-local order
      std::vector<mf::IdxVec> nn(n);
      const int R = 3;
      for (int t = 0; t < n; ++t) {
        const auto& p = pts[order[t]];
        std::vector<std::pair<int64_t, int32_t>> cand;
        for (int dj = -R; dj <= R; ++dj)
          for (int di = -R; di <= R; ++di) {
            int64_t i2 = p[0] + di, j2 = p[1] + dj;
            if (i2 < 0 || j2 < 0 || i2 >= mb || j2 >= mb) continue;
            cand.push_back({(int64_t)di * di + (int64_t)dj * dj, (int32_t)pos[j2 * mb + i2]});
          }
        std::sort(cand.begin(), cand.end());
        for (int c = 0; c < (int)cand.size() && c < knn; ++c) nn[t].push_back(cand[c].second);
      }
      probs[b].n = n;
      probs[b].off = off;
      probs[b].tree = tree;
      nns[b] = std::move(nn);
      probs[b].nn = &nns[b];
      s->off.push_back(off);
      off += n;
    }
    s->rows = off;
    // memory: factors are O(n log n) per block; reserve generously
    size_t persist = std::max<size_t>((size_t)off * 4096 * sizeof(float), size_t(1) << 30);
    size_t scratch = std::max<size_t>((size_t)off * 8192 * sizeof(float), size_t(2) << 30);
    s->cx = std::make_unique<mf::BFContext<float>>(s->st, persist, scratch);
    mf::upload(s->dP, s->P, s->st);
    mf::upload(s->dQ, s->Q, s->st);
    const double* dP = s->dP.as<double>();
    const double* dQ = s->dQ.as<double>();
    mf::BFContext<float>* cx = s->cx.get();
    cudaStream_t st = s->st;
    mf::DExtract<float> ext = [cx, dP, dQ, k, st](const std::vector<std::pair<mf::IdxVec, mf::IdxVec>>& lst,
                                                  std::vector<Blk<float>>& dst) {
      std::vector<mf::GreenJob<float>> jobs;
      int64_t mx = 0;
      for (size_t q = 0; q < lst.size(); ++q) {
        if (lst[q].first.empty() || lst[q].second.empty()) continue;
        mf::GreenJob<float> j;
        j.X = static_cast<const int32_t*>(cx->upload(lst[q].first.data(), lst[q].first.size() * 4));
        j.Y = static_cast<const int32_t*>(cx->upload(lst[q].second.data(), lst[q].second.size() * 4));
        j.nx = (int)lst[q].first.size(); j.ny = (int)lst[q].second.size();
        j.dst = dst[q].p; j.dplane = dst[q].plane; j.dld = dst[q].ld;
        jobs.push_back(j);
        mx = std::max<int64_t>(mx, (int64_t)j.nx * j.ny);
      }
      if (jobs.empty()) return;
      auto* dj = cx->scratch.takeT<mf::GreenJob<float>>(jobs.size());
      cx->h2d(dj, jobs.data(), jobs.size() * sizeof(jobs[0]));
      int bx = (int)std::min<int64_t>(512, (mx + 255) / 256);
      mf::count_launches(1);
      mf::k_green<float><<<dim3(bx, (unsigned)jobs.size()), 256, 0, st>>>(dj, dP, dQ, k);
    };
    mf::BFParams P;
    P.tol = tol;
    P.max_rank = max_rank;
    P.alpha = alpha;
    P.knn = knn;
    cx->hodbf_entry_eval_batch(ext, probs, P);
    for (auto& hp : probs) s->H.push_back(std::move(hp.out));
    MF_CUDA(cudaStreamSynchronize(st));
    s->build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  } catch (const mf::CudaError& e) {
    return std::string(e.what()).find("out of memory") != std::string::npos ? MF_ERR_OOM : MF_ERR_CUDA;
  } catch (const std::exception&) {
    return MF_ERR_ARG;
  }
  *out = s.release();
  return MF_OK;
}

int mf_green_info(const mf_bfset* s, int64_t* rows, double* storage, int32_t* max_rank, double* build_seconds) {
  if (!s) return MF_ERR_ARG;
  double st = 0;
  int mr = 0;
  for (auto& h : s->H) { st += h->storage(); mr = std::max(mr, h->max_rank()); }
  if (rows) *rows = s->rows;
  if (storage) *storage = st;
  if (max_rank) *max_rank = mr;
  if (build_seconds) *build_seconds = s->build_seconds;
  return MF_OK;
}

int mf_green_apply_counts(const mf_bfset* s, int32_t nrhs, double* flops, double* bytes) {
  if (!s) return MF_ERR_ARG;
  for (auto& p : s->plans)
    if (p->nrhs == nrhs && p->state > 0) {
      if (flops) *flops = p->flops;
      if (bytes) *bytes = p->bytes;
      return MF_OK;
    }
  return MF_ERR_STATE;
}

int mf_green_points(const mf_bfset* s, double* P, double* Q) {
  if (!s) return MF_ERR_ARG;
  if (P) std::memcpy(P, s->P.data(), s->P.size() * sizeof(double));
  if (Q) std::memcpy(Q, s->Q.data(), s->Q.size() * sizeof(double));
  return MF_OK;
}

int mf_green_apply(mf_bfset* s, int32_t nrhs, const float* x, float* y) {
  if (!s || nrhs <= 0 || !x || !y) return MF_ERR_ARG;
  try {
    auto& cx = *s->cx;
    // leaves of every block in one launch, then each HOD-BF level of every block in one stage-merged apply
    auto body = [&]() {
      const size_t mk = cx.scratch.mark();
      Blk<float> X, Y;
      X.p = const_cast<float*>(x); X.rows = (int)s->rows; X.cols = nrhs; X.ld = nrhs; X.plane = s->rows * nrhs;
      Y = X;
      Y.p = y;
      std::vector<mf::GemmDesc<float>> g;
      int maxLH = 0;
      for (size_t b = 0; b < s->H.size(); ++b) {
        const auto& H = *s->H[b];
        maxLH = std::max(maxLH, H.LH);
        for (size_t q = 0; q < H.D.size(); ++q) {
          const mf::Range r = H.tree[H.LH][q];
          const int nr = (int)(r.b - r.a);
          mf::GemmDesc<float> d;
          d.m = nr; d.n = nrhs; d.k = nr; d.transA = 0; d.transB = 0; d.alpha = 1.f; d.beta = 0.f;
          d.A = H.D[q].pm();
          d.B = X.sub((int)(s->off[b] + r.a), 0, nr, nrhs).pm();
          d.C = Y.sub((int)(s->off[b] + r.a), 0, nr, nrhs).pm();
          g.push_back(d);
        }
      }
      cx.gemm(g);
      // every off-diagonal butterfly of every level in one stage-merged apply: the butterflies of
      // one block's levels have different level counts, so their last (accumulating) stages fall
      // in different launches and never write the same rows at once
      std::vector<const mf::DBF<float>*> bfs;
      std::vector<Blk<float>> xs, ys;
      for (int l = 1; l <= maxLH; ++l) {
        for (size_t b = 0; b < s->H.size(); ++b) {
          const auto& H = *s->H[b];
          if (l > H.LH) continue;
          for (int i = 0; i < (1 << l); ++i) {
            const mf::Range rr = H.tree[l][i], cr = H.tree[l][i ^ 1];
            bfs.push_back(H.off[l][i].get());
            xs.push_back(X.sub((int)(s->off[b] + cr.a), 0, (int)(cr.b - cr.a), nrhs));
            ys.push_back(Y.sub((int)(s->off[b] + rr.a), 0, (int)(rr.b - rr.a), nrhs));
          }
        }
      }
      cx.apply(bfs, xs, ys, false, true);
      cx.scratch.release(mk);   // stream order makes later reuse of the scratch safe
    };
    GreenPlan* pl = nullptr;
    for (auto& p : s->plans)
      if (p->nrhs == nrhs && p->x == x && p->y == y) pl = p.get();
    if (!pl) {
      s->plans.push_back(std::make_unique<GreenPlan>());
      pl = s->plans.back().get();
      pl->nrhs = nrhs;
      pl->x = x;
      pl->y = y;
    }
    if (pl->state == 2 && cx.scratch.mark() != pl->mark) pl->state = 3;   // scratch moved under the graph
    if (pl->state == 0 || pl->state == 3) {
      const double f0 = cx.flops, b0 = cx.bytes;
      if (pl->state == 0) cx.count_begin();
      body();
      if (pl->state == 0) {
        pl->blob = cx.count_end();
        pl->state = 1;
        pl->flops = cx.flops - f0;
        pl->bytes = cx.bytes - b0;
      }
    } else {
      if (pl->state == 1) {   // capture on the private stream
        if (!s->gs) {
          MF_CUDA(cudaStreamCreateWithFlags(&s->gs, cudaStreamNonBlocking));
          for (auto& e : s->ev) MF_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        }
        const size_t cap = pl->blob + 4096;
        MF_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&pl->hblob), cap, cudaHostAllocDefault));
        pl->dblob.alloc(cap);
        cx.flush();
        pl->mark = cx.scratch.mark();
        cx.st = s->gs;
        cx.capture_begin(pl->hblob, pl->dblob.as<char>(), cap);
        cudaGraph_t gr = nullptr;
        const int64_t c0 = mf::launch_count();
        bool ok = cudaStreamBeginCapture(s->gs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
          try {
            body();
          } catch (...) {
            ok = false;
          }
          if (cudaStreamEndCapture(s->gs, &gr) != cudaSuccess || !gr) ok = false;
        }
        pl->glaunch = (int)(mf::launch_count() - c0);
        mf::count_launches(-pl->glaunch);   // captured, not run
        cx.st = s->st;
        cx.scratch.release(pl->mark);
        if (!cx.capture_end()) ok = false;
        if (ok && cudaGraphInstantiate(&pl->exec, gr, 0) != cudaSuccess) {
          pl->exec = nullptr;
          ok = false;
        }
        if (gr) cudaGraphDestroy(gr);
        cudaGetLastError();
        pl->state = ok ? 2 : 3;
        if (!ok) body();
      }
      if (pl->state == 2) {
        MF_CUDA(cudaEventRecord(s->ev[0], s->st));
        MF_CUDA(cudaStreamWaitEvent(s->gs, s->ev[0], 0));
        MF_CUDA(cudaGraphLaunch(pl->exec, s->gs));
        mf::count_launches(pl->glaunch);
        MF_CUDA(cudaEventRecord(s->ev[1], s->gs));
        MF_CUDA(cudaStreamWaitEvent(s->st, s->ev[1], 0));
      }
    }
    MF_CUDA(cudaGetLastError());
    MF_CUDA(cudaStreamSynchronize(s->st));
  } catch (const std::exception&) {
    return MF_ERR_CUDA;
  }
  return MF_OK;
}

void mf_green_destroy(mf_bfset* s) { delete s; }

}  // extern "C"
