// Continuous-batching solve server over resident factorizations.
//
// Several factorizations stay resident on the device (one mf_handle each, each
// on its own CUDA stream).  Requests carry right-hand sides for one of them.
// One worker thread per factorization takes every request that is waiting for
// it when the previous batch finishes (continuous batching: requests that
// arrive while a batch is on the GPU join the next batch), admits them while
// the device workspace of the batch fits the memory budget and the device's free
// memory (cudaMemGetInfo, read when the batch is formed), solves the batch
// with one mf_solve call (columns converge independently inside GMRES), and
// completes each request.  Batches of different factorizations overlap on the
// device because the workers run concurrently on different streams.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mf.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id;
  int32_t problem, nrhs;
  const double* b;
  double* x;
  double t_arrival = 0, t_start = 0, t_done = 0;
  int32_t iters = 0, converged = 0, batch_rhs = 0, status = 1;   // status 1 = pending
  double max_rel_residual = 0;
};

struct Worker {
  mf_handle* h = nullptr;
  int64_t n = 0;
  std::deque<std::shared_ptr<Request>> q;
  std::thread th;
  std::vector<double> bbuf, xbuf;
};

}  // namespace

struct mf_server {
  std::vector<std::unique_ptr<Worker>> w;
  int device = 0;                         // the device of the handles (current at mf_server_create)
  int32_t max_batch = 256;
  int64_t budget = 0;
  std::atomic<int64_t> reserved{0};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  int64_t next_id = 0;
  std::map<int64_t, std::shared_ptr<Request>> reqs;
  Clock::time_point t0 = Clock::now();
  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  int64_t bytes_for(int64_t n, int32_t nrhs) const {
    return (int64_t)(30 + 10) * n * std::min<int32_t>(nrhs, max_batch) * 16;
  }
  void run(int p);
};

void mf_server::run(int p) {
  Worker& wk = *w[p];
  cudaSetDevice(device);
  for (;;) {
    std::vector<std::shared_ptr<Request>> batch;
    int64_t bytes = 0;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stop || !wk.q.empty(); });
      if (stop && wk.q.empty()) return;
      // admission by the device's free memory as well as the caller's budget: a batch's workspace
      // must fit in what the device has left (keeping 1 GiB of headroom)
      size_t fr = 0, total = 0;
      int64_t room = budget;
      if (cudaMemGetInfo(&fr, &total) == cudaSuccess)
        room = std::min<int64_t>(budget, reserved.load() + std::max<int64_t>(0, (int64_t)fr - (int64_t(1) << 30)));
      int tot = 0;
      while (!wk.q.empty()) {
        auto& r = wk.q.front();
        int64_t need = bytes_for(wk.n, tot + r->nrhs) - bytes;
        bool first = batch.empty();
        if (!first && (tot + r->nrhs > max_batch || reserved.load() + need > room)) break;
        if (first && reserved.load() + need > room && reserved.load() > 0) break;   // wait for memory
        bytes += need;
        reserved += need;
        tot += r->nrhs;
        batch.push_back(r);
        wk.q.pop_front();
      }
      if (batch.empty()) {
        cv_done.wait_for(lk, std::chrono::milliseconds(1));
        continue;
      }
    }
    const double ts = now();
    int tot = 0;
    for (auto& r : batch) tot += r->nrhs;
    wk.bbuf.resize((size_t)2 * wk.n * tot);
    wk.xbuf.resize((size_t)2 * wk.n * tot);
    size_t off = 0;
    for (auto& r : batch) {
      std::memcpy(wk.bbuf.data() + off, r->b, sizeof(double) * 2 * wk.n * r->nrhs);
      off += (size_t)2 * wk.n * r->nrhs;
    }
    // each request reports its own columns: what it returns does not depend on the batch it ran in.
    // A request wider than max_batch runs alone, in slices of max_batch columns (its columns are
    // independent), so that the solve's workspace stays bounded.
    mf_solve_info info{};
    std::vector<int32_t> cit(tot, 0), cconv(tot, 0);
    std::vector<double> cres(tot, 0.0);
    int rc = MF_OK;
    bool have_cols = true;
    for (int c0 = 0; c0 < tot && (rc == MF_OK || rc == MF_ERR_NO_CONVERGENCE); c0 += max_batch) {
      const int nc = std::min(max_batch, tot - c0);
      const size_t o = (size_t)2 * wk.n * c0;
      mf_solve_info part{};
      const int r = mf_solve(wk.h, nc, wk.bbuf.data() + o, wk.n, wk.xbuf.data() + o, wk.n, &part);
      if (r != MF_OK && r != MF_ERR_NO_CONVERGENCE) {
        rc = r;
        break;
      }
      if (r == MF_ERR_NO_CONVERGENCE) rc = r;
      info.iters = std::max(info.iters, part.iters);
      info.max_rel_residual = std::max(info.max_rel_residual, part.max_rel_residual);
      have_cols = have_cols && mf_solve_columns(wk.h, nc, cit.data() + c0, cconv.data() + c0, cres.data() + c0) == MF_OK;
    }
    have_cols = have_cols && (rc == MF_OK || rc == MF_ERR_NO_CONVERGENCE);
    const double td = now();
    off = 0;
    for (auto& r : batch) {
      if (rc == MF_OK || rc == MF_ERR_NO_CONVERGENCE)
        std::memcpy(r->x, wk.xbuf.data() + off, sizeof(double) * 2 * wk.n * r->nrhs);
      off += (size_t)2 * wk.n * r->nrhs;
    }
    reserved -= bytes;
    {
      std::lock_guard<std::mutex> lk(mu);
      int c0 = 0;
      for (auto& r : batch) {
        r->t_start = ts;
        r->t_done = td;
        r->batch_rhs = tot;
        if (have_cols) {
          int it = 0, conv = 1;
          double worst = 0;
          for (int c = c0; c < c0 + r->nrhs; ++c) {
            it = std::max(it, cit[c]);
            conv = conv && cconv[c];
            worst = std::max(worst, cres[c]);
          }
          r->iters = it;
          r->converged = conv;
          r->max_rel_residual = worst;
          r->status = conv ? MF_OK : MF_ERR_NO_CONVERGENCE;
        } else {
          r->iters = info.iters;
          r->converged = 0;
          r->max_rel_residual = info.max_rel_residual;
          r->status = rc == MF_OK ? MF_ERR_CUDA : rc;
        }
        c0 += r->nrhs;
      }
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
}

extern "C" {

int mf_server_create(int32_t nproblems, mf_handle* const* handles, int32_t max_batch_rhs, int64_t mem_budget_bytes,
                     mf_server** out) {
  if (!out || nproblems <= 0 || !handles || max_batch_rhs <= 0 || mem_budget_bytes <= 0) return MF_ERR_ARG;
  auto s = std::make_unique<mf_server>();
  s->max_batch = max_batch_rhs;
  if (cudaGetDevice(&s->device) != cudaSuccess) return MF_ERR_CUDA;
  s->budget = mem_budget_bytes;
  for (int p = 0; p < nproblems; ++p) {
    mf_stats_t st;
    if (!handles[p] || mf_stats(handles[p], &st) != MF_OK) return MF_ERR_ARG;
    auto wk = std::make_unique<Worker>();
    wk->h = handles[p];
    wk->n = st.n;
    s->w.push_back(std::move(wk));
  }
  mf_server* sp = s.get();
  for (int p = 0; p < nproblems; ++p) sp->w[p]->th = std::thread([sp, p] { sp->run(p); });
  *out = s.release();
  return MF_OK;
}

int mf_server_submit(mf_server* s, int32_t problem, int32_t nrhs, const double* b, double* x, int64_t* id) {
  if (!s || problem < 0 || problem >= (int32_t)s->w.size() || nrhs <= 0 || !b || !x || !id) return MF_ERR_ARG;
  if (s->bytes_for(s->w[problem]->n, nrhs) > s->budget) return MF_ERR_OOM;
  auto r = std::make_shared<Request>();
  r->problem = problem;
  r->nrhs = nrhs;
  r->b = b;
  r->x = x;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    r->t_arrival = s->now();
    s->reqs[r->id] = r;
    s->w[problem]->q.push_back(r);
    *id = r->id;
  }
  s->cv_work.notify_all();
  return MF_OK;
}

int mf_server_wait(mf_server* s, int64_t id, mf_request_info* info) {
  if (!s) return MF_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return MF_ERR_ARG;
  auto r = it->second;
  s->cv_done.wait(lk, [&] { return r->status != 1; });
  if (info) {
    info->id = r->id;
    info->problem = r->problem;
    info->nrhs = r->nrhs;
    info->iters = r->iters;
    info->converged = r->converged;
    info->batch_rhs = r->batch_rhs;
    info->max_rel_residual = r->max_rel_residual;
    info->t_arrival = r->t_arrival;
    info->t_start = r->t_start;
    info->t_done = r->t_done;
  }
  s->reqs.erase(it);
  return r->status;
}

void mf_server_destroy(mf_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& w : s->w)
    if (w->th.joinable()) w->th.join();
  delete s;
}

}  // extern "C"
