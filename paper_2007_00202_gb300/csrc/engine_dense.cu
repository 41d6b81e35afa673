// Dense-front engine: the multifrontal factorization of Alg. 1 (Sec. 2), one
// batched launch sequence per assembly-tree level (deepest level first), and
// the forward/backward solve of Alg. 1's last line.
//
// Per level:  assemble A entries, extend-add children (Sec. 2 step 1);
// blocked right-looking LU of F11 with partial pivoting inside F11 (step 2);
// explicit L^-1 and U^-1 by recursive 2 x 2 block inversion; F12 <- L^-1 P^T F12,
// F21 <- F21 U^-1 (step 3) and C = F22 - F21 F12 (step 4) as batched GEMMs.
// The whole sequence is built once per analysis ("launch program") and
// replayed by every factorization.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <thread>

#include "engine.h"
#include "engine_comp.h"

namespace mf {

namespace {

constexpr int LU_NB = 32;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <typename T>
class DenseEngine : public EngineBase {
 public:
  DenseEngine(const Analysis& an, const DeviceMatrix& A, cudaStream_t st, const EngineOptions& eo)
      : an_(an), A_(A), st_(st), eo_(eo) {
    plan();
  }

  int max_rank() const override { return max_rank_; }
  double compressed_seconds() const override { return comp_seconds_; }

  void factor(double tol) override {
    const int64_t c0 = launch_count();
    const auto tf0 = std::chrono::steady_clock::now();
    MF_CUDA(cudaMemsetAsync(arena_.p, 0, zero_bytes_, st_));
    MF_CUDA(cudaMemsetAsync(status_.p, 0, sizeof(int32_t), st_));
    BFParams P;
    P.tol = tol > 0 ? tol : 1e-12;
    P.max_rank = eo_.max_rank;
    P.alpha = eo_.alpha;
    P.knn = eo_.knn;
    comp_flops_ = 0;
    comp_seconds_ = 0;
    prof[0].collect();   // pending records may name the events of the graphs dropped next
    for (auto& kv : sprog_) kv.second->drop_graph();   // compressed fronts move with every factorization
    if (comp_) {
      comp_->fronts.clear();
      for (int w = 0; w < comp_->contexts(); ++w) {
        comp_->ctx(w).persist.release(0);
        comp_->ctx(w).scratch.release(0);
        comp_->ctx(w).flops = 0;
      }
    }
    static const bool serial = getenv("MF_SERIAL_FRONTS") && getenv("MF_SERIAL_FRONTS")[0] == '1';
    for (size_t lv = 0; lv < levels_.size(); ++lv) {
      const auto& lvl = comp_levels_[lv];
      // the dense fronts of a level with compressed fronts run on their own stream: neither
      // depends on the other (both read only lower levels), and the compressed fronts' host-driven
      // construction would otherwise start behind the dense fronts' LU
      const bool side = !lvl.empty() && lvl_begin_[lv + 1] > lvl_begin_[lv] && !serial;
      cudaStream_t dst = st_;
      if (side) {
        MF_CUDA(cudaEventRecord(lev_ev_[1], st_));
        MF_CUDA(cudaStreamWaitEvent(ds_, lev_ev_[1], 0));
        dst = ds_;
      }
      for (size_t i = lvl_begin_[lv]; i < lvl_begin_[lv + 1]; ++i) {
        if (gemm_flops_[i] > 0) prof[1].time(dst, gemm_flops_[i], gemm_bytes_[i], [&] { fops_[i](dst); });
        else fops_[i](dst);
      }
      if (side) MF_CUDA(cudaEventRecord(lev_ev_[2], ds_));
      if (lvl.empty()) continue;
      auto t0 = std::chrono::steady_clock::now();
      const auto& F = an_.fronts;
      // front list[i] with execution context w (and helper context `helper` for its F12 / F21, -1:
      // none); densify on the same context
      const int ctx_cap = std::min<int>(CompressedPart<T>::kMaxContexts, std::max(1, eo_.max_contexts));
      auto run = [&](const std::vector<int32_t>& list, size_t i0, size_t step, int w, int helper) {
        for (size_t i = i0; i < list.size(); i += step) {
          const int fid = list[i];
          comp_->factor_front(fid, fr_, P, eo_.seed, w, helper);
          if (F[fid].parent >= 0 && !F[F[fid].parent].compressed) comp_->densify_C(fid, fr_[fid], w);
        }
      };
      if (lvl.size() == 1 || serial || eo_.max_contexts <= 1) {
        const int helper = (!serial && ctx_cap >= 2) ? 1 : -1;
        if (helper > 0) comp_->ensure_contexts(2);
        run(lvl, 0, 1, 0, helper);
      } else {
        // the fronts of one level are independent: up to kMaxContexts host threads build them, each
        // with its own stream and scratch arena, taking the next front of the level when done, so
        // that one thread's host work overlaps the others' GPU work
        const int nctx = std::min<int>((int)lvl.size(), ctx_cap);
        const int nhelp = std::max(0, std::min(nctx, ctx_cap - nctx));   // contexts left for F12 / F21
        comp_->ensure_contexts(nctx + nhelp);
        MF_CUDA(cudaEventRecord(lev_ev_[0], st_));                  // children and dense fronts below
        for (int w = 1; w < nctx; ++w) MF_CUDA(cudaStreamWaitEvent(comp_->stream(w), lev_ev_[0], 0));
        int dev = 0;
        MF_CUDA(cudaGetDevice(&dev));
        std::atomic<size_t> next{0};
        std::vector<std::exception_ptr> errs(nctx);
        auto worker = [&](int w) {
          try {
            for (size_t i = next++; i < lvl.size(); i = next++) run(lvl, i, lvl.size(), w, w < nhelp ? nctx + w : -1);
          } catch (...) {
            errs[w] = std::current_exception();
          }
        };
        std::vector<std::thread> th;
        for (int w = 1; w < nctx; ++w)
          th.emplace_back([&, w, dev] {
            if (cudaSetDevice(dev) != cudaSuccess) {
              errs[w] = std::make_exception_ptr(CudaError("cudaSetDevice failed"));
              return;
            }
            worker(w);
            if (!errs[w] && cudaStreamSynchronize(comp_->stream(w)) != cudaSuccess)
              errs[w] = std::make_exception_ptr(CudaError("construction stream failed"));
          });
        worker(0);
        for (auto& t : th) t.join();
        for (auto& e : errs)
          if (e) std::rethrow_exception(e);
      }
      if (side) MF_CUDA(cudaStreamWaitEvent(st_, lev_ev_[2], 0));   // the next level needs both
      for (int32_t fid : lvl) max_rank_ = std::max(max_rank_, comp_->fronts.at(fid)->max_rank);
      comp_seconds_ += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (comp_) {
      comp_flops_ = 0;
      for (int w = 0; w < comp_->contexts(); ++w) comp_flops_ += comp_->ctx(w).flops;
    }
    if (getenv("MF_TRACE") && getenv("MF_TRACE")[0] == '1') {
      MF_CUDA(cudaStreamSynchronize(st_));
      fprintf(stderr, "[mf] factor: %.3f s, compressed fronts %.3f s (host-issued, synchronised per phase)\n",
              std::chrono::duration<double>(std::chrono::steady_clock::now() - tf0).count(), comp_seconds_);
      if (comp_)
        for (int w = 0; w < comp_->contexts(); ++w)
          fprintf(stderr, "[mf] context %d: persistent arena peak %.2f of %.2f GB, work arena peak %.2f of %.2f GB\n",
                  w, comp_->ctx(w).persist.peak() / 1e9, comp_->ctx(w).persist.capacity() / 1e9,
                  comp_->ctx(w).scratch.peak() / 1e9, comp_->ctx(w).scratch.capacity() / 1e9);
    }
    MF_CUDA(cudaGetLastError());
    nlaunch_factor_ = (int)(launch_count() - c0);
    int32_t stat = 0;
    MF_CUDA(cudaMemcpyAsync(&stat, status_.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st_));
    MF_CUDA(cudaStreamSynchronize(st_));
    prof[0].collect();
    prof[1].collect();
    if (stat == 2) throw TimeoutError("a bounded wait in a tensor-core kernel expired");
    if (stat != DEV_OK) throw SingularError("zero pivot in a dense front");
  }

  // Solve programs exist for column counts 16, 32, 64, ...: a call with nrhs columns runs the
  // smallest one that holds them (the extra columns stay zero; columns never mix).
  static int nrhs_bucket(int nrhs) {
    int nb = 16;
    while (nb < nrhs) nb *= 2;
    return nb;
  }

  int front_apply(int fid, int which, int nrhs, const double* x, double* y) override {
    if (!comp_ || nrhs <= 0) return -1;
    auto it = comp_->fronts.find(fid);
    if (it == comp_->fronts.end()) return -1;
    CompFront<T>& cf = *it->second;
    const int s = cf.s, u = cf.u;
    int rin = s, rout = s;
    if (which == 2) rin = u;
    if (which == 3) rout = u;
    if (which == 4) rin = rout = u;
    if (which < 0 || which > 4 || rin == 0 || rout == 0) return -1;
    if ((which == 2 && !cf.F12) || (which == 3 && !cf.F21) || (which == 4 && !cf.C)) return -1;
    BFContext<T>& cx = comp_->cx;
    const int ld = (nrhs + 3) & ~3;
    const int64_t pin = (int64_t)rin * ld, pout = (int64_t)rout * ld;
    std::vector<T> hx(2 * (size_t)pin, T(0)), hy(2 * (size_t)pout);
    for (int c = 0; c < nrhs; ++c)
      for (int r = 0; r < rin; ++r) {
        hx[(size_t)r * ld + c] = (T)x[2 * ((size_t)c * rin + r)];
        hx[pin + (size_t)r * ld + c] = (T)x[2 * ((size_t)c * rin + r) + 1];
      }
    DevMem dx, dy;
    dx.alloc(sizeof(T) * hx.size());
    dy.alloc(sizeof(T) * hy.size());
    MF_CUDA(cudaMemcpyAsync(dx.p, hx.data(), sizeof(T) * hx.size(), cudaMemcpyHostToDevice, cx.st));
    Blk<T> X, Y;
    X.p = dx.as<T>(); X.rows = rin; X.cols = nrhs; X.ld = ld; X.plane = pin;
    Y.p = dy.as<T>(); Y.rows = rout; Y.cols = nrhs; Y.ld = ld; Y.plane = pout;
    const size_t mk = cx.scratch.mark();
    if (which == 0) cx.hodbf_apply(*cf.F11, X, Y, false);
    if (which == 1) cx.inv_apply(*cf.F11inv, X, Y, false);
    if (which == 2 || which == 3) {
      std::vector<const DBF<T>*> b{which == 2 ? cf.F12.get() : cf.F21.get()};
      std::vector<Blk<T>> xs{X}, ys{Y};
      cx.apply(b, xs, ys, false, false);
    }
    if (which == 4) cx.hodbf_apply(*cf.C, X, Y, false);
    cx.flush();
    MF_CUDA(cudaMemcpyAsync(hy.data(), dy.p, sizeof(T) * hy.size(), cudaMemcpyDeviceToHost, cx.st));
    MF_CUDA(cudaStreamSynchronize(cx.st));
    cx.scratch.release(mk);
    for (int c = 0; c < nrhs; ++c)
      for (int r = 0; r < rout; ++r) {
        y[2 * ((size_t)c * rout + r)] = (double)hy[(size_t)r * ld + c];
        y[2 * ((size_t)c * rout + r) + 1] = (double)hy[pout + (size_t)r * ld + c];
      }
    return 0;
  }

  void apply_precond(const double* x, double* y, int nrhs) override {
    const int nb = nrhs_bucket(nrhs);
    SolveProg& sp = solve_prog(nb);
    const int64_t n = an_.n;
    T* X = sp.X.template as<T>();
    const int64_t xpl = n * nb;
    static const bool trace = getenv("MF_TRACE") && getenv("MF_TRACE")[0] == '1';
    std::chrono::steady_clock::time_point t0;
    const int state0 = sp.state;
    if (trace) {
      MF_CUDA(cudaStreamSynchronize(st_));
      t0 = std::chrono::steady_clock::now();
    }
    launch_to_planar<T>(x, n, n, nrhs, nullptr, X, xpl, st_, nb);
    run_solve_ops(sp);
    launch_from_planar<T>(X, xpl, n, nrhs, nullptr, y, n, st_, nb);
    MF_CUDA(cudaGetLastError());
    if (trace) {
      auto t1 = std::chrono::steady_clock::now();
      MF_CUDA(cudaStreamSynchronize(st_));
      auto t2 = std::chrono::steady_clock::now();
      fprintf(stderr, "[mf] precond nrhs %d state %d->%d  issue %.3f ms  total %.3f ms  (%d kernels)\n", nrhs, state0,
              sp.state, std::chrono::duration<double, std::milli>(t1 - t0).count(),
              std::chrono::duration<double, std::milli>(t2 - t0).count(), sp.glaunch);
    }
  }

  double factor_flops() const override { return flops_ + comp_flops_; }
  double factor_bytes() const override { return factor_bytes_; }
  void arena_usage(double& peak, double& capacity) const override {
    peak = capacity = 0;
    if (!comp_) return;
    for (int w = 0; w < comp_->contexts(); ++w) {
      const BFContext<T>& c = w == 0 ? comp_->cx : *comp_->extra_[w - 1];
      peak += (double)c.persist.peak() + (double)c.scratch.peak();
      capacity += (double)c.persist.capacity() + (double)c.scratch.capacity();
    }
  }
  int launches_factor() const override { return nlaunch_factor_; }
  int launches_solve(int nrhs) override { return solve_prog(nrhs_bucket(nrhs)).nlaunch + 2; }

 private:
  struct SolveProg {
    DevMem X, tmp, ptrs, descs, tiles;
    std::vector<std::function<void(cudaStream_t)>> ops;
    int nlaunch = 0;
    // CUDA graph of ops: state 0 = the next call runs eagerly and counts the staged bytes of
    // the compressed fronts, 1 = the next call captures, 2 = replay, 3 = eager only
    int state = 0;
    cudaGraphExec_t exec = nullptr;
    cudaGraphExec_t exec_prof = nullptr;   // the same program with timing events (profiling)
    int64_t nrep = 0;
    size_t blob = 0, blob_cap = 0, mark = 0;
    int glaunch = 0;
    int64_t nrec = 0;                                  // timed launches of one run (profiling)
    std::vector<LaunchProfiler::Rec> prof_recs;        // event pairs recorded by the graph
    char* hblob = nullptr;
    DevMem dblob;
    void drop_graph() {
      if (exec) cudaGraphExecDestroy(exec);
      if (exec_prof) cudaGraphExecDestroy(exec_prof);
      exec = exec_prof = nullptr;
      state = 0;
      nrep = 0;
      for (auto& r : prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
      }
      prof_recs.clear();
    }
    ~SolveProg() {
      drop_graph();
      if (hblob) cudaFreeHost(hblob);
    }
  };

  const Analysis& an_;
  const DeviceMatrix& A_;
  cudaStream_t st_;
  DevMem arena_, fronts_d_, flists_d_, status_, descs_d_, tiles_d_, ea_d_;
  size_t zero_bytes_ = 0;
  std::vector<FrontDev<T>> fr_;             // indexed by front id
  std::vector<std::vector<int32_t>> levels_;  // front ids per level, deepest first
  std::vector<size_t> level_off_;           // offsets of the level lists in flists_d_
  std::vector<std::function<void(cudaStream_t)>> fops_;
  std::vector<GemmDesc<T>> descs_;
  std::vector<GemmTile> tiles_;
  double flops_ = 0, factor_bytes_ = 0;
  int nlaunch_factor_ = 0;
  std::map<int, std::unique_ptr<SolveProg>> sprog_;
  std::vector<double> gemm_flops_;          // per factor op: algorithmic flops if it is a GEMM launch, else 0
  std::vector<double> gemm_bytes_;          // and its algorithmic bytes
  EngineOptions eo_;
  std::vector<std::vector<int32_t>> comp_levels_;   // compressed fronts per level
  std::vector<size_t> lvl_begin_;           // factor ops of level lv: [lvl_begin_[lv], lvl_begin_[lv+1])
  std::unique_ptr<CompressedPart<T>> comp_;
  double comp_flops_ = 0, comp_seconds_ = 0;
  int max_rank_ = 0;
  cudaStream_t gs_ = nullptr;               // stream of the solve graphs (forked from and joined to st_)
  // the engine stream's progress before a level's compressed fronts [0] and dense fronts [1]; the
  // dense fronts' completion on ds_ [2]
  cudaEvent_t lev_ev_[3] = {nullptr, nullptr, nullptr};
  cudaStream_t ds_ = nullptr;               // dense fronts of the levels that also hold compressed fronts
  cudaEvent_t gev_[2] = {nullptr, nullptr};

 public:
  ~DenseEngine() override {
    sprog_.clear();
    for (auto e : gev_)
      if (e) cudaEventDestroy(e);
    for (auto e : lev_ev_)
      if (e) cudaEventDestroy(e);
    if (ds_) cudaStreamDestroy(ds_);
    if (gs_) cudaStreamDestroy(gs_);
  }

 private:
  void set_profiling(int period) override {
    prof[0].collect();
    for (auto& kv : sprog_) kv.second->drop_graph();   // recaptured with (or without) timing events
    EngineBase::set_profiling(period);
  }

  // The solve program is the same launch sequence for every call with the same nrhs: the
  // first call runs it eagerly (and sizes the job tables of the compressed fronts), the
  // second captures it into a CUDA graph on gs_, later calls replay the graph.  A capture
  // that fails (a synchronizing call inside, an error) leaves the program eager.
  void run_solve_ops(SolveProg& sp) {
    static const bool no_graph = getenv("MF_NO_GRAPH") && getenv("MF_NO_GRAPH")[0] == '1';
    BFContext<T>* cx = comp_ ? &comp_->cx : nullptr;
    auto eager = [&] {
      for (auto& op : sp.ops) op(st_);
    };
    if (no_graph || sp.state == 3) return eager();
    if (sp.state == 2 && cx && cx->scratch.mark() != sp.mark) sp.drop_graph();
    if (sp.state == 2) {
      // with profiling on, one replay in prof[0].every runs the copy with timing events
      const bool timed = prof[0].on && sp.exec_prof && (sp.nrep++ % prof[0].every) == 0;
      if (timed) prof[0].collect();   // the previous timed replay's events are recorded again
      MF_CUDA(cudaEventRecord(gev_[0], st_));
      MF_CUDA(cudaStreamWaitEvent(gs_, gev_[0], 0));
      MF_CUDA(cudaGraphLaunch(timed ? sp.exec_prof : sp.exec, gs_));
      count_launches(sp.glaunch);   // the kernel nodes the replay runs
      MF_CUDA(cudaEventRecord(gev_[1], gs_));
      MF_CUDA(cudaStreamWaitEvent(st_, gev_[1], 0));
      if (timed) prof[0].replayed(sp.prof_recs);
      return;
    }
    if (sp.state == 0) {
      if (cx) cx->count_begin();
      const int64_t r0 = prof[0].calls;
      eager();
      sp.nrec = prof[0].calls - r0;   // narrow-GEMM launches of one run (event pairs a timed graph needs)
      if (cx) sp.blob = cx->count_end();
      sp.state = 1;
      return;
    }
    // capture
    if (!gs_) {
      MF_CUDA(cudaStreamCreateWithFlags(&gs_, cudaStreamNonBlocking));
      for (auto& e : gev_) MF_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    const size_t need = sp.blob + 4096;
    if (cx && sp.blob_cap < need) {
      if (sp.hblob) cudaFreeHost(sp.hblob);
      sp.hblob = nullptr;
      MF_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&sp.hblob), need, cudaHostAllocDefault));
      sp.dblob.alloc(need);
      sp.blob_cap = need;
    }
    if (cx) {
      cx->flush();
      sp.mark = cx->scratch.mark();
    }
    // one capture of the program; with_events: the copy with timing events for profiled replays
    auto capture = [&](bool with_events) -> cudaGraphExec_t {
      if (cx) {
        cx->st = gs_;
        comp_->st_ = gs_;
        cx->capture_begin(sp.hblob, sp.dblob.template as<char>(), sp.blob_cap);
      }
      const bool prof_on = prof[0].on;
      if (with_events) {
        prof[0].collect();
        prof[0].reserve_graph((size_t)sp.nrec);
        sp.prof_recs.clear();
        prof[0].capture_into = &sp.prof_recs;
      } else {
        prof[0].on = false;
      }
      cudaGraph_t g = nullptr;
      const int64_t c0 = launch_count();
      bool ok = cudaStreamBeginCapture(gs_, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        try {
          for (auto& op : sp.ops) op(gs_);
        } catch (...) {
          ok = false;
        }
        if (cudaStreamEndCapture(gs_, &g) != cudaSuccess || !g) ok = false;
      }
      sp.glaunch = (int)(launch_count() - c0);
      count_launches(-sp.glaunch);   // captured, not run
      prof[0].on = prof_on;
      if (with_events) {             // reserved event pairs the capture did not use
        for (size_t i = sp.prof_recs.size(); i < prof[0].graph_reserve.size(); ++i) {
          cudaEventDestroy(prof[0].graph_reserve[i].a);
          cudaEventDestroy(prof[0].graph_reserve[i].b);
        }
        prof[0].graph_reserve.clear();
        prof[0].capture_into = nullptr;
      }
      if (cx) {
        cx->st = st_;
        comp_->st_ = st_;
        cx->scratch.release(sp.mark);
        if (!cx->capture_end()) ok = false;   // copies the job tables to their device twin
      }
      cudaGraphExec_t ex = nullptr;
      if (ok && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) ex = nullptr;
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();   // a failed capture leaves its error behind
      return ex;
    };
    sp.exec = capture(false);
    if (!sp.exec) {
      sp.state = 3;
      return eager();
    }
    if (prof[0].on) sp.exec_prof = capture(true);   // without it, replays are simply not timed
    sp.state = 2;
    run_solve_ops(sp);
  }

  const int32_t* flist(size_t lv) const { return flists_d_.template as<int32_t>() + level_off_[lv]; }

  // Register a batched GEMM launch in the program being built (descs, tiles collected in vectors).
  struct GemmRef {
    size_t d0, t0;
    int nt;
    size_t nd;
  };
  GemmRef add_gemm(std::vector<GemmDesc<T>>& D, std::vector<GemmTile>& Tl, const std::vector<GemmDesc<T>>& batch,
                   int tile = GEMM_TILE, int col_tile = 0) {
    GemmRef r{D.size(), Tl.size(), 0, 0};
    for (auto& d : batch) {
      if (d.m <= 0 || d.n <= 0) continue;
      int idx = (int)(D.size() - r.d0);
      D.push_back(d);
      const int ct = col_tile ? col_tile : tile;
      int tm = (d.m + tile - 1) / tile, tn = (d.n + ct - 1) / ct;
      for (int i = 0; i < tm; ++i)
        for (int j = 0; j < tn; ++j) Tl.push_back({idx, i, j, 0});
    }
    r.nt = (int)(Tl.size() - r.t0);
    r.nd = D.size() - r.d0;
    return r;
  }

  // "NT" products (both operands K-contiguous): tcgen05 tensor cores for complex64, SIMT for complex128
  static bool use_tc() {
    if (sizeof(T) != 4) return false;
    const char* e = getenv("MF_NO_TC");
    return !(e && e[0] == '1');
  }
  void push_gemm_nt(std::vector<GemmDesc<T>>& D, std::vector<GemmTile>& Tl, const std::vector<GemmDesc<T>>& b) {
    const bool tc = use_tc();
    GemmRef g = add_gemm(D, Tl, b, tc ? gemm_tc_tile() : GEMM_TILE);
    if (!g.nt) return;
    if (tc)
      push_op([this, g](cudaStream_t st) { launch_nt(g, st); }, ref_flops(D, g), ref_bytes(D, g));
    else
      push_op([this, g](cudaStream_t st) {
        launch_gemm<T>(descs_d_.template as<GemmDesc<T>>() + g.d0, tiles_d_.template as<GemmTile>() + g.t0, g.nt, st);
      }, ref_flops(D, g), ref_bytes(D, g));
  }
  void launch_nt(const GemmRef& g, cudaStream_t st);

  void push_op(std::function<void(cudaStream_t)> fn, double fl = 0, double by = 0) {
    gemm_bytes_.push_back(by);
    fops_.push_back(std::move(fn));
    gemm_flops_.push_back(fl);
  }

  double ref_flops(const std::vector<GemmDesc<T>>& D, const GemmRef& g) const {
    double f = 0;
    for (size_t i = g.d0; i < g.d0 + g.nd; ++i) f += 8.0 * D[i].m * D[i].n * D[i].k;
    return f;
  }
  double ref_bytes(const std::vector<GemmDesc<T>>& D, const GemmRef& g) const {
    double b = 0;
    for (size_t i = g.d0; i < g.d0 + g.nd; ++i) b += gemm_bytes(D[i]);
    return b;
  }

  static GemmDesc<T> gd(int m, int n, int k, int ta, int tb, T alpha, T beta, PMat<T> a, PMat<T> b, PMat<T> c) {
    GemmDesc<T> d;
    d.m = m; d.n = n; d.k = k; d.transA = ta; d.transB = tb; d.alpha = alpha; d.beta = beta;
    d.A = a; d.B = b; d.C = c;
    return d;
  }

  void plan() {
    const auto& F = an_.fronts;
    const size_t nf = F.size();
    fr_.resize(nf);
    // ---- memory plan: one arena; the zeroed part first
    size_t off = 0;
    auto take = [&](size_t elems) {
      size_t o = off;
      off = align_up(off + elems * sizeof(T), 256);
      return o;
    };
    struct Offs { size_t LU, Linv, UinvT, F12w, F21w, C, UT, W, F12p, F12T, F21f, piv, perm, upd; };
    std::vector<Offs> o(nf);
    for (size_t i = 0; i < nf; ++i) {
      int64_t s = F[i].compressed ? 0 : F[i].s(), u = F[i].u();
      const int64_t ls = (s + 3) & ~3ll, lu = (u + 3) & ~3ll;
      o[i].LU = take(2 * s * ls);
      o[i].Linv = take(2 * s * ls);
      o[i].UinvT = take(2 * s * ls);
      o[i].F12w = take(2 * (s ? u : 0) * ls);
      o[i].F21w = take(2 * (s ? u : 0) * ls);
      o[i].C = take(F[i].parent >= 0 ? 2 * u * lu : 0);
    }
    zero_bytes_ = off;
    for (size_t i = 0; i < nf; ++i) {
      int64_t s = F[i].compressed ? 0 : F[i].s(), u = F[i].compressed ? 0 : F[i].u();
      const int64_t ls = (s + 3) & ~3ll;
      o[i].UT = take(2 * s * ls);
      o[i].W = take(4 * s * ls);   // two s x s planar work matrices (L and U inversions)
      o[i].F12p = take(2 * u * ls);
      o[i].F12T = take(2 * u * ls);
      o[i].F21f = take(2 * u * ls);
      o[i].piv = off; off = align_up(off + s * 4, 256);
      o[i].perm = off; off = align_up(off + s * 4, 256);
      o[i].upd = off; off = align_up(off + F[i].u() * 8, 256);
      factor_bytes_ += sizeof(T) * 2.0 * (2.0 * s * s + 2.0 * s * u) + 8.0 * s;
    }
    arena_.alloc(off);
    char* base = arena_.template as<char>();
    for (size_t i = 0; i < nf; ++i) {
      int64_t s = F[i].s(), u = F[i].u();
      const int64_t sa = F[i].compressed ? 0 : s;   // dense buffers of compressed fronts are empty
      FrontDev<T>& f = fr_[i];
      f.sep_begin = F[i].sep_begin;
      f.s = (int32_t)s;
      f.u = (int32_t)u;
      f.upd = reinterpret_cast<const int64_t*>(base + o[i].upd);
      f.LU = reinterpret_cast<T*>(base + o[i].LU);
      f.UT = reinterpret_cast<T*>(base + o[i].UT);
      f.Linv = reinterpret_cast<T*>(base + o[i].Linv);
      f.UinvT = reinterpret_cast<T*>(base + o[i].UinvT);
      f.F12w = reinterpret_cast<T*>(base + o[i].F12w);
      f.F12p = reinterpret_cast<T*>(base + o[i].F12p);
      f.F12T = reinterpret_cast<T*>(base + o[i].F12T);
      f.F21w = reinterpret_cast<T*>(base + o[i].F21w);
      f.F21f = reinterpret_cast<T*>(base + o[i].F21f);
      f.C = reinterpret_cast<T*>(base + o[i].C);
      f.W = reinterpret_cast<T*>(base + o[i].W);
      f.piv = reinterpret_cast<int32_t*>(base + o[i].piv);
      f.perm = reinterpret_cast<int32_t*>(base + o[i].perm);
      const int64_t ls = (sa + 3) & ~3ll, lu = (u + 3) & ~3ll;
      f.ls = (int32_t)ls;
      f.lu = (int32_t)lu;
      f.pl_ss = sa * ls;
      f.pl_us = (sa ? u : 0) * ls;
      f.pl_uu = u * lu;
      if (u) MF_CUDA(cudaMemcpyAsync(base + o[i].upd, F[i].upd.data(), u * 8, cudaMemcpyHostToDevice, st_));
      if (!F[i].compressed) flops_ += 8.0 * ((double)s * s * s / 3.0 + (double)s * s * u + (double)s * u * u);
    }
    upload(fronts_d_, fr_, st_);
    status_.alloc(sizeof(int32_t));
    // ---- levels
    int depth = 0;
    for (auto& f : F) depth = std::max(depth, f.level + 1);
    levels_.assign(depth, {});
    comp_levels_.assign(depth, {});
    bool any_comp = false;
    for (auto& f : F) {
      if (f.compressed) { comp_levels_[depth - 1 - f.level].push_back((int32_t)f.id); any_comp = true; }
      else levels_[depth - 1 - f.level].push_back((int32_t)f.id);
    }
    if (any_comp) {
      comp_ = std::make_unique<CompressedPart<T>>(an_, A_, st_, eo_.persist_bytes, eo_.scratch_bytes);
      comp_->prepare_neighbours(eo_.knn);   // symbolic proxy candidates, part of the analysis
      comp_->cx.prof = &prof[0];
      for (auto& e : lev_ev_) MF_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      MF_CUDA(cudaStreamCreateWithFlags(&ds_, cudaStreamNonBlocking));
    }
    std::vector<int32_t> all;
    for (auto& lv : levels_) {
      level_off_.push_back(all.size());
      all.insert(all.end(), lv.begin(), lv.end());
    }
    upload(flists_d_, all, st_);
    // ---- extend-add items (children of the fronts of each level; slot 0 / slot 1)
    std::vector<ExtendAddItem<T>> items;
    std::vector<int32_t> rel_all;
    struct EaRef { size_t i0; int n; int maxuc; };
    std::vector<std::array<EaRef, 2>> ea_refs(depth);
    std::vector<std::vector<std::pair<int64_t, int64_t>>> rel_spans;   // per item: rel offset
    std::vector<size_t> rel_off_of_item;
    for (int lv = 0; lv < depth; ++lv) {
      for (int slot = 0; slot < 2; ++slot) {
        EaRef r{items.size(), 0, 0};
        for (int32_t fid : levels_[lv]) {
          const auto& pf = F[fid];
          if ((int)pf.children.size() <= slot) continue;
          const auto& cf = F[pf.children[slot]];
          // rel map: position of the child's I^u entries in the parent front
          size_t ro = rel_all.size();
          for (int64_t g : cf.upd) {
            int64_t pos;
            if (g >= pf.sep_begin && g < pf.sep_end) pos = g - pf.sep_begin;
            else {
              auto it = std::lower_bound(pf.upd.begin(), pf.upd.end(), g);
              if (it == pf.upd.end() || *it != g) throw std::runtime_error("child update set not in parent front");
              pos = pf.s() + (it - pf.upd.begin());
            }
            rel_all.push_back((int32_t)pos);
          }
          ExtendAddItem<T> it;
          it.Cc = fr_[cf.id].C;
          it.plane_c = fr_[cf.id].pl_uu;
          it.ldc = fr_[cf.id].lu;
          it.rel = nullptr;
          it.uc = (int32_t)cf.u();
          it.parent = fid;
          rel_off_of_item.push_back(ro);
          items.push_back(it);
          r.n++;
          r.maxuc = std::max(r.maxuc, (int)cf.u());
        }
        ea_refs[lv][slot] = r;
      }
    }
    upload(rel_, rel_all, st_);
    for (size_t k = 0; k < items.size(); ++k) items[k].rel = rel_.template as<int32_t>() + rel_off_of_item[k];
    upload(ea_d_, items, st_);

    // ---- the factor program
    std::vector<GemmDesc<T>> D;
    std::vector<GemmTile> Tl;
    struct PendingGemm { GemmRef r; };
    for (int lv = 0; lv < depth; ++lv) {
      lvl_begin_.push_back(fops_.size());
      const auto& L = levels_[lv];
      const int nfl = (int)L.size();
      int max_s = 0, max_u = 0, max_rows = 0;
      for (int32_t fid : L) {
        max_s = std::max<int>(max_s, (int)F[fid].s());
        max_u = std::max<int>(max_u, (int)F[fid].u());
      }
      max_rows = max_s + max_u;
      const int32_t* fl_lv = nullptr;   // resolved at run time
      const size_t lvi = lv;
      // assemble
      push_op([this, lvi, nfl, max_rows](cudaStream_t st) {
        launch_assemble_A<T>(fronts_d_.template as<FrontDev<T>>(), flist(lvi), nfl, max_rows, A_.rowptr.template as<int64_t>(),
                             A_.col64.template as<int64_t>(), A_.vals.template as<double>(), st);
      });
      nlaunch_factor_++;
      for (int slot = 0; slot < 2; ++slot) {
        EaRef r = ea_refs[lv][slot];
        if (r.n == 0) continue;
        push_op([this, r](cudaStream_t st) {
          launch_extend_add<T>(ea_d_.template as<ExtendAddItem<T>>() + r.i0, r.n, fronts_d_.template as<FrontDev<T>>(), r.maxuc, st);
        });
        nlaunch_factor_++;
      }
      (void)fl_lv;
      // blocked LU
      for (int kb = 0; kb < max_s; kb += LU_NB) {
        push_op([this, lvi, nfl, kb, max_s](cudaStream_t st) {
          launch_panel_lu<T>(fronts_d_.template as<FrontDev<T>>(), flist(lvi), nfl, kb, LU_NB, max_s - kb,
                             status_.template as<int32_t>(), st);
        });
        push_op([this, lvi, nfl, kb, max_s](cudaStream_t st) {
          launch_panel_trsm<T>(fronts_d_.template as<FrontDev<T>>(), flist(lvi), nfl, kb, LU_NB, max_s, st);
        });
        nlaunch_factor_ += 2;
        std::vector<GemmDesc<T>> batch;
        for (int32_t fid : L) {
          const FrontDev<T>& f = fr_[fid];
          int s = f.s;
          int w = std::min(LU_NB, s - kb);
          int rem = s - kb - w;
          if (kb >= s || rem <= 0) continue;
          const int ls = f.ls;
          PMat<T> a{f.LU + (int64_t)(kb + w) * ls + kb, f.pl_ss, ls};
          PMat<T> b{f.LU + (int64_t)kb * ls + kb + w, f.pl_ss, ls};
          PMat<T> c{f.LU + (int64_t)(kb + w) * ls + kb + w, f.pl_ss, ls};
          batch.push_back(gd(rem, rem, w, 0, 0, T(-1), T(1), a, b, c));
        }
        GemmRef g = add_gemm(D, Tl, batch);
        if (g.nt) {
          push_op([this, g](cudaStream_t st) {
            launch_gemm<T>(descs_d_.template as<GemmDesc<T>>() + g.d0, tiles_d_.template as<GemmTile>() + g.t0, g.nt, st);
          }, ref_flops(D, g), ref_bytes(D, g));
          nlaunch_factor_++;
        }
      }
      push_op([this, lvi, nfl, max_s, max_u](cudaStream_t st) {
        launch_post_lu<T>(fronts_d_.template as<FrontDev<T>>(), flist(lvi), nfl, max_s, max_u, st);
      });
      nlaunch_factor_ += 3;
      for (int which = 0; which < 2; ++which) {
        push_op([this, lvi, nfl, max_s, which](cudaStream_t st) {
          launch_trinv_diag<T>(fronts_d_.template as<FrontDev<T>>(), flist(lvi), nfl, max_s, which, nullptr, st);
        });
        nlaunch_factor_++;
      }
      // recursive 2 x 2 block inversion of the lower triangles, block 64 -> 128 -> ...
      for (int h = 64; h < max_s; h *= 2) {
        std::vector<GemmDesc<T>> b1, b2;
        for (int32_t fid : L) {
          const FrontDev<T>& f = fr_[fid];
          int s = f.s;
          for (int a0 = 0; a0 + h < s; a0 += 2 * h) {
            int c0 = a0 + h, c1 = std::min(a0 + 2 * h, s);
            int mc = c1 - c0;
            for (int which = 0; which < 2; ++which) {
              T* Tm = which == 0 ? f.LU : f.UT;
              T* X = which == 0 ? f.Linv : f.UinvT;
              T* W = f.W + (which == 0 ? 0 : 2 * f.pl_ss);   // separate work matrix per triangle
              const int ls = f.ls;
              int64_t woff = (int64_t)c0 * ls + a0;
              PMat<T> tca{Tm + (int64_t)c0 * ls + a0, f.pl_ss, ls};
              PMat<T> xaa{X + (int64_t)a0 * ls + a0, f.pl_ss, ls};
              PMat<T> w{W + woff, f.pl_ss, ls};
              PMat<T> xcc{X + (int64_t)c0 * ls + c0, f.pl_ss, ls};
              PMat<T> xca{X + (int64_t)c0 * ls + a0, f.pl_ss, ls};
              b1.push_back(gd(mc, h, h, 0, 0, T(1), T(0), tca, xaa, w));
              b2.push_back(gd(mc, h, mc, 0, 0, T(-1), T(0), xcc, w, xca));
            }
          }
        }
        GemmRef g1 = add_gemm(D, Tl, b1);
        GemmRef g2 = add_gemm(D, Tl, b2);
        if (g1.nt) {
          push_op([this, g1](cudaStream_t st) {
            launch_gemm<T>(descs_d_.template as<GemmDesc<T>>() + g1.d0, tiles_d_.template as<GemmTile>() + g1.t0, g1.nt, st);
          }, ref_flops(D, g1));
          push_op([this, g2](cudaStream_t st) {
            launch_gemm<T>(descs_d_.template as<GemmDesc<T>>() + g2.d0, tiles_d_.template as<GemmTile>() + g2.t0, g2.nt, st);
          }, ref_flops(D, g2));
          nlaunch_factor_ += 2;
        }
      }
      // F12^T <- (P^T F12)^T L^-T  and  F21 <- F21 U^-1
      {
        std::vector<GemmDesc<T>> b;
        for (int32_t fid : L) {
          const FrontDev<T>& f = fr_[fid];
          if (f.u == 0) continue;
          b.push_back(gd(f.u, f.s, f.s, 0, 1, T(1), T(0), PMat<T>{f.F12p, f.pl_us, f.ls}, PMat<T>{f.Linv, f.pl_ss, f.ls},
                         PMat<T>{f.F12T, f.pl_us, f.ls}));
          b.push_back(gd(f.u, f.s, f.s, 0, 1, T(1), T(0), PMat<T>{f.F21w, f.pl_us, f.ls},
                         PMat<T>{f.UinvT, f.pl_ss, f.ls}, PMat<T>{f.F21f, f.pl_us, f.ls}));
        }
        push_gemm_nt(D, Tl, b);
      }
      // Schur complement C = F22 - F21 F12   (Sec. 2 step 4)
      {
        std::vector<GemmDesc<T>> b;
        for (int32_t fid : L) {
          const FrontDev<T>& f = fr_[fid];
          if (f.u == 0 || F[fid].parent < 0) continue;
          b.push_back(gd(f.u, f.u, f.s, 0, 1, T(-1), T(1), PMat<T>{f.F21f, f.pl_us, f.ls},
                         PMat<T>{f.F12T, f.pl_us, f.ls}, PMat<T>{f.C, f.pl_uu, f.lu}));
        }
        push_gemm_nt(D, Tl, b);
      }
    }
    lvl_begin_.push_back(fops_.size());
    upload(descs_d_, D, st_);
    upload(tiles_d_, Tl, st_);
    MF_CUDA(cudaStreamSynchronize(st_));
  }

  SolveProg& solve_prog(int nrhs) {
    auto it = sprog_.find(nrhs);
    if (it != sprog_.end()) return *it->second;
    auto sp = std::make_unique<SolveProg>();
    const auto& F = an_.fronts;
    const int64_t n = an_.n;
    sp->X.alloc(sizeof(T) * 2 * n * nrhs);
    MF_CUDA(cudaMemsetAsync(sp->X.p, 0, sizeof(T) * 2 * n * nrhs, st_));   // padding columns stay zero
    // per-front temps ta (s x nrhs), tb (s x nrhs), tu (u x nrhs)
    std::vector<size_t> ta(F.size()), tb(F.size()), tu(F.size());
    size_t off = 0;
    for (size_t i = 0; i < F.size(); ++i) {
      ta[i] = off; off = align_up(off + sizeof(T) * 2 * F[i].s() * nrhs, 256);
      tb[i] = off; off = align_up(off + sizeof(T) * 2 * F[i].s() * nrhs, 256);
      tu[i] = off; off = align_up(off + sizeof(T) * 2 * F[i].u() * nrhs, 256);
    }
    sp->tmp.alloc(off);
    char* tb0 = sp->tmp.template as<char>();
    auto P = [&](size_t o) { return reinterpret_cast<T*>(tb0 + o); };
    // pointer tables per level: ta, tb, tu in level order
    std::vector<T*> ptab;
    std::vector<size_t> poff_ta(levels_.size()), poff_tb(levels_.size()), poff_tu(levels_.size());
    for (size_t lv = 0; lv < levels_.size(); ++lv) {
      poff_ta[lv] = ptab.size();
      for (int32_t f : levels_[lv]) ptab.push_back(P(ta[f]));
      poff_tb[lv] = ptab.size();
      for (int32_t f : levels_[lv]) ptab.push_back(P(tb[f]));
      poff_tu[lv] = ptab.size();
      for (int32_t f : levels_[lv]) ptab.push_back(P(tu[f]));
    }
    upload(sp->ptrs, ptab, st_);
    T* const* pt = sp->ptrs.template as<T* const>();
    std::vector<GemmDesc<T>> D;
    std::vector<GemmTile> Tl;
    T* X = sp->X.template as<T>();
    const int64_t xpl = n * nrhs;
    SolveProg* spp = sp.get();
    // narrow products (n = nrhs): 32-row tiles of the streaming kernel, K split over a cluster when
    // a level has few row tiles; wider ones: the square-tile SIMT kernel
    const int nb = gemm_nrhs_width(nrhs, sizeof(T));
    auto gemm_op = [&](const std::vector<GemmDesc<T>>& b) {
      if (nb) {
        GemmRef g = add_gemm(D, Tl, b, GEMM_NRHS_ROWS, nb);
        if (!g.nt) return;
        int maxk = 1;
        for (auto& x : b) maxk = std::max(maxk, (int)x.k);
        const int ks = gemm_nrhs_split(g.nt, maxk);
        const double fl = ref_flops(D, g), by = ref_bytes(D, g);
        sp->ops.push_back([this, spp, g, nb, ks, maxk, fl, by](cudaStream_t st) {
          prof[0].time(st, fl, by, [&] {
            launch_gemm_nrhs<T>(spp->descs.template as<GemmDesc<T>>() + g.d0,
                                spp->tiles.template as<GemmTile>() + g.t0, g.nt, nb, ks, maxk, st);
          });
        });
        sp->nlaunch++;
        return;
      }
      GemmRef g = add_gemm(D, Tl, b);
      if (g.nt) {
        sp->ops.push_back([spp, g](cudaStream_t st) {
          launch_gemm<T>(spp->descs.template as<GemmDesc<T>>() + g.d0, spp->tiles.template as<GemmTile>() + g.t0, g.nt, st);
        });
        sp->nlaunch++;
      }
    };
    auto comp_op = [&](size_t lv, bool fwd) {
      if (comp_levels_[lv].empty()) return;
      std::vector<int> fids(comp_levels_[lv].begin(), comp_levels_[lv].end());
      sp->ops.push_back([this, fids, fwd, X, n, nrhs](cudaStream_t) {
        Blk<T> Xb;
        Xb.p = X; Xb.rows = (int)n; Xb.cols = nrhs; Xb.ld = nrhs; Xb.plane = n * nrhs;
        if (fwd) comp_->forward(fids, Xb);
        else comp_->backward(fids, Xb);
      });
    };
    // forward: leaves -> root
    for (size_t lv = 0; lv < levels_.size(); ++lv) {
      comp_op(lv, true);
      const auto& L = levels_[lv];
      int nfl = (int)L.size(), max_s = 0, max_u = 0;
      for (int32_t f : L) { max_s = std::max<int>(max_s, fr_[f].s); max_u = std::max<int>(max_u, fr_[f].u); }
      size_t lvi = lv;
      sp->ops.push_back([this, lvi, nfl, max_s, X, xpl, nrhs, pt, poff_ta](cudaStream_t st) {
        launch_fwd_gather<T>(fronts_d_.template as<FrontDev<T>>(), flist(lvi), nfl, max_s, X, xpl, nrhs, pt + poff_ta[lvi], st);
      });
      sp->nlaunch++;
      std::vector<GemmDesc<T>> b1, b2;
      for (int32_t f : L) {
        const FrontDev<T>& fd = fr_[f];
        int64_t spl = (int64_t)fd.s * nrhs, upl = (int64_t)fd.u * nrhs;
        b1.push_back(gd(fd.s, nrhs, fd.s, 0, 0, T(1), T(0), PMat<T>{fd.Linv, fd.pl_ss, fd.ls},
                        PMat<T>{P(ta[f]), spl, nrhs}, PMat<T>{P(tb[f]), spl, nrhs}));
        if (fd.u)
          b2.push_back(gd(fd.u, nrhs, fd.s, 0, 0, T(-1), T(0), PMat<T>{fd.F21f, fd.pl_us, fd.ls},
                          PMat<T>{P(tb[f]), spl, nrhs}, PMat<T>{P(tu[f]), upl, nrhs}));
      }
      gemm_op(b1);
      sp->ops.push_back([this, lvi, nfl, max_s, X, xpl, nrhs, pt, poff_tb](cudaStream_t st) {
        launch_scatter_sep<T>(fronts_d_.template as<FrontDev<T>>(), flist(lvi), nfl, max_s, X, xpl, nrhs, pt + poff_tb[lvi], st);
      });
      sp->nlaunch++;
      gemm_op(b2);
      if (max_u) {
        sp->ops.push_back([this, lvi, nfl, max_u, X, xpl, nrhs, pt, poff_tu](cudaStream_t st) {
          launch_scatter_add_upd<T>(fronts_d_.template as<FrontDev<T>>(), flist(lvi), nfl, max_u, X, xpl, nrhs,
                                    pt + poff_tu[lvi], st);
        });
        sp->nlaunch++;
      }
    }
    // backward: root -> leaves
    for (size_t lvr = levels_.size(); lvr-- > 0;) {
      comp_op(lvr, false);
      const auto& L = levels_[lvr];
      int nfl = (int)L.size(), max_s = 0, max_u = 0;
      for (int32_t f : L) { max_s = std::max<int>(max_s, fr_[f].s); max_u = std::max<int>(max_u, fr_[f].u); }
      size_t lvi = lvr;
      if (max_u) {
        sp->ops.push_back([this, lvi, nfl, max_u, X, xpl, nrhs, pt, poff_tu](cudaStream_t st) {
          launch_gather_upd<T>(fronts_d_.template as<FrontDev<T>>(), flist(lvi), nfl, max_u, X, xpl, nrhs, pt + poff_tu[lvi],
                               st);
        });
        sp->nlaunch++;
      }
      sp->ops.push_back([this, lvi, nfl, max_s, X, xpl, nrhs, pt, poff_tb](cudaStream_t st) {
        launch_gather_sep<T>(fronts_d_.template as<FrontDev<T>>(), flist(lvi), nfl, max_s, X, xpl, nrhs, pt + poff_tb[lvi], st);
      });
      sp->nlaunch++;
      std::vector<GemmDesc<T>> b1, b2;
      for (int32_t f : L) {
        const FrontDev<T>& fd = fr_[f];
        int64_t spl = (int64_t)fd.s * nrhs, upl = (int64_t)fd.u * nrhs;
        if (fd.u)
          b1.push_back(gd(fd.s, nrhs, fd.u, 1, 0, T(-1), T(1), PMat<T>{fd.F12T, fd.pl_us, fd.ls},
                          PMat<T>{P(tu[f]), upl, nrhs}, PMat<T>{P(tb[f]), spl, nrhs}));
        b2.push_back(gd(fd.s, nrhs, fd.s, 1, 0, T(1), T(0), PMat<T>{fd.UinvT, fd.pl_ss, fd.ls},
                        PMat<T>{P(tb[f]), spl, nrhs}, PMat<T>{P(ta[f]), spl, nrhs}));
      }
      gemm_op(b1);
      gemm_op(b2);
      sp->ops.push_back([this, lvi, nfl, max_s, X, xpl, nrhs, pt, poff_ta](cudaStream_t st) {
        launch_scatter_sep<T>(fronts_d_.template as<FrontDev<T>>(), flist(lvi), nfl, max_s, X, xpl, nrhs, pt + poff_ta[lvi], st);
      });
      sp->nlaunch++;
    }
    upload(sp->descs, D, st_);
    upload(sp->tiles, Tl, st_);
    MF_CUDA(cudaStreamSynchronize(st_));
    auto& ref = *sp;
    sprog_[nrhs] = std::move(sp);
    return ref;
  }

  DevMem rel_;
};

template <>
void DenseEngine<float>::launch_nt(const GemmRef& g, cudaStream_t st) {
  launch_gemm_tc(descs_d_.template as<GemmDesc<float>>() + g.d0, tiles_d_.template as<GemmTile>() + g.t0, g.nt,
                 status_.template as<int32_t>(), st);
}
template <>
void DenseEngine<double>::launch_nt(const GemmRef& g, cudaStream_t st) {
  launch_gemm<double>(descs_d_.template as<GemmDesc<double>>() + g.d0, tiles_d_.template as<GemmTile>() + g.t0, g.nt,
                      st);
}

}  // namespace

std::unique_ptr<EngineBase> make_engine_c64(const Analysis& an, const DeviceMatrix& A, cudaStream_t st,
                                            const EngineOptions& eo) {
  return std::make_unique<DenseEngine<float>>(an, A, st, eo);
}
std::unique_ptr<EngineBase> make_engine_c128(const Analysis& an, const DeviceMatrix& A, cudaStream_t st,
                                             const EngineOptions& eo) {
  return std::make_unique<DenseEngine<double>>(an, A, st, eo);
}

}  // namespace mf
