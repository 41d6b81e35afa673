// Compressed fronts (Alg. 5) on the GPU; see engine_comp.h.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <numeric>
#include <thread>

#include "engine_comp.h"

namespace mf {

namespace {

IdxVec iota_vec(int n) {
  IdxVec v(n);
  std::iota(v.begin(), v.end(), 0);
  return v;
}

}  // namespace

template <typename T>
void CompressedPart<T>::ensure_contexts(int n) {
  n = std::min(n, kMaxContexts);
  while (contexts() < n) {
    cudaStream_t s = nullptr;
    MF_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    extra_st_.push_back(s);
    extra_.push_back(std::make_unique<BFContext<T>>(s, &cx.persist, scratch_bytes_));
    extra_.back()->prof = cx.prof;
  }
}

namespace {

// position of a global index in front f: I^s -> [0, s), I^u -> s + index, else -1
int32_t front_position(const FrontInfo& f, int64_t g) {
  if (g >= f.sep_begin && g < f.sep_end) return (int32_t)(g - f.sep_begin);
  auto it = std::lower_bound(f.upd.begin(), f.upd.end(), g);
  if (it == f.upd.end() || *it != g) return -1;
  return (int32_t)(f.s() + (it - f.upd.begin()));
}

template <typename Neigh>
void compute_neighbours(const Analysis& an, const FrontInfo& f, int knn, Neigh& out) {
  FrontNeighbours nb;
  front_neighbours(an, f, knn, nb);
  const int s = (int)f.s(), u = (int)f.u();
  auto to_local = [&](const std::vector<int64_t>& ptr, const std::vector<int64_t>& idx, int rows, int base) {
    std::vector<IdxVec> o(rows);
    for (int r = 0; r < rows; ++r)
      for (int64_t k = ptr[r]; k < ptr[r + 1]; ++k) {
        int32_t p = front_position(f, idx[k]);
        if (p >= 0) o[r].push_back(p - base);
      }
    return o;
  };
  out.nn11 = to_local(nb.nn11_ptr, nb.nn11, s, 0);
  out.nn12 = to_local(nb.nn12_ptr, nb.nn12, s, s);   // I^s row -> I^u local
  out.nn21 = to_local(nb.nn21_ptr, nb.nn21, u, 0);   // I^u row -> I^s local
  out.nn22 = to_local(nb.nn22_ptr, nb.nn22, u, s);
}

}  // namespace

template <typename T>
void CompressedPart<T>::prepare_neighbours(int knn) {
  std::vector<int> fids;
  for (const auto& f : an_.fronts)
    if (f.compressed) fids.push_back((int)f.id);
  std::vector<std::unique_ptr<Neigh>> res(fids.size());
  std::atomic<size_t> next{0};
  auto work = [&] {
    for (size_t i; (i = next.fetch_add(1)) < fids.size();) {
      res[i] = std::make_unique<Neigh>();
      compute_neighbours(an_, an_.fronts[fids[i]], knn, *res[i]);
    }
  };
  const size_t nt = std::min<size_t>(fids.size(), std::max(1u, std::min(8u, std::thread::hardware_concurrency())));
  std::vector<std::thread> th;
  for (size_t t = 1; t < nt; ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  std::lock_guard<std::mutex> lk(neigh_mu_);
  neigh_.clear();
  for (size_t i = 0; i < fids.size(); ++i) neigh_[fids[i]] = std::move(res[i]);
  neigh_knn_ = knn;
}

template <typename T>
const typename CompressedPart<T>::Neigh& CompressedPart<T>::neighbours(int fid, int knn) {
  {
    std::lock_guard<std::mutex> lk(neigh_mu_);
    if (neigh_knn_ != knn) {
      neigh_.clear();
      neigh_knn_ = knn;
    }
    auto it = neigh_.find(fid);
    if (it != neigh_.end()) return *it->second;
  }
  auto n = std::make_unique<Neigh>();
  compute_neighbours(an_, an_.fronts[fid], knn, *n);
  std::lock_guard<std::mutex> lk(neigh_mu_);
  auto& slot = neigh_[fid];
  if (!slot) slot = std::move(n);
  return *slot;
}

template <typename T>
void CompressedPart<T>::factor_front(int fid, const std::vector<FrontDev<T>>& fr, const BFParams& P, uint64_t seed,
                                     int w, int helper) {
  BFContext<T>& cx = ctx(w);          // this front's execution context and stream
  const cudaStream_t st_ = stream(w);
  const size_t scratch_mark = cx.scratch.mark();   // this front's work is released when it is built
  auto t0 = std::chrono::steady_clock::now();
  const FrontInfo& f = an_.fronts[fid];
  const int s = (int)f.s(), u = (int)f.u();
  auto cfp = std::make_unique<CompFront<T>>();
  CompFront<T>& cf = *cfp;
  cf.fid = fid;
  cf.s = s;
  cf.u = u;
  cf.sep_begin = f.sep_begin;
  // position of each global index in this front: I^s -> [0, s), I^u -> s + index
  auto front_pos = [&](int64_t g) -> int32_t { return front_position(f, g); };
  // children: inverse relative maps (front position -> child position, -1 if absent)
  struct Kid {
    int id;
    bool compressed;
    const CompFront<T>* cf = nullptr;   // a compressed child's factors (built at a lower level)
    std::vector<int32_t> inv;
    DevMem d_inv;
  };
  std::vector<Kid> kids;
  for (int64_t c : f.children) {
    Kid k;
    k.id = (int)c;
    k.compressed = an_.fronts[c].compressed;
    if (k.compressed) {
      std::lock_guard<std::mutex> lk(fronts_mu_);
      k.cf = fronts.at(k.id).get();
    }
    k.inv.assign(s + u, -1);
    const auto& cu = an_.fronts[c].upd;
    for (size_t i = 0; i < cu.size(); ++i) {
      int32_t p = front_pos(cu[i]);
      if (p < 0) throw std::runtime_error("child update set not in the parent front");
      k.inv[p] = (int32_t)i;
    }
    upload(k.d_inv, k.inv, st_);
    kids.push_back(std::move(k));
  }
  // device context of the gathers: A entries and dense children
  FrontCtx<T> ctx{};
  ctx.sep_begin = f.sep_begin;
  ctx.s = s;
  ctx.u = u;
  ctx.upd = fr[fid].upd;
  ctx.nkids = 0;
  for (auto& k : kids)
    if (!k.compressed) {
      DenseKid<T> dk;
      dk.C = fr[k.id].C;
      dk.plane = fr[k.id].pl_uu;
      dk.ld = fr[k.id].lu;
      dk.inv = k.d_inv.template as<int32_t>();
      ctx.kids[ctx.nkids++] = dk;
    }
  DevMem d_ctx;
  upload(d_ctx, std::vector<FrontCtx<T>>{ctx}, st_);
  const FrontCtx<T>* dctx = d_ctx.template as<FrontCtx<T>>();
  const DBF<T>* Sptr = nullptr;
  // extraction over front positions; shifts map the caller's local indices to front positions
  // (on: the context that issues the extraction's work, this front's own by default)
  auto make_ext = [&, dctx](int rs, int cs, bool with_A, bool minus_S, BFContext<T>* on = nullptr) -> DExtract<T> {
    BFContext<T>* ec = on ? on : &cx;
    return [&, dctx, rs, cs, with_A, minus_S, ec](const std::vector<std::pair<IdxVec, IdxVec>>& lst,
                                                  std::vector<Blk<T>>& dst) {
      std::vector<FrontEntryJob<T>> jobs;
      int64_t mx = 0;
      std::vector<std::pair<IdxVec, IdxVec>> g(lst);
      for (auto& pr : g) {
        for (auto& x : pr.first) x += rs;
        for (auto& y : pr.second) y += cs;
      }
      for (size_t q = 0; q < g.size(); ++q) {
        if (g[q].first.empty() || g[q].second.empty()) continue;
        FrontEntryJob<T> j;
        j.ctx = 0;
        j.X = static_cast<const int32_t*>(ec->upload(g[q].first.data(), g[q].first.size() * 4));
        j.Y = static_cast<const int32_t*>(ec->upload(g[q].second.data(), g[q].second.size() * 4));
        j.nx = (int)g[q].first.size(); j.ny = (int)g[q].second.size();
        j.dst = dst[q].p; j.dplane = dst[q].plane; j.dld = dst[q].ld;
        j.with_A = with_A ? 1 : 0;
        j.accumulate = 0;
        jobs.push_back(j);
        mx = std::max<int64_t>(mx, (int64_t)j.nx * j.ny);
      }
      if (!jobs.empty()) {
        const FrontEntryJob<T>* dj = ec->stage(jobs.data(), jobs.size());
        launch_front_entries<T>(dj, (int)jobs.size(), mx, dctx, A_.rowptr.template as<int64_t>(),
                                A_.col32.template as<int32_t>(), A_.vals.template as<double>(), ec->st);
      }
      for (auto& k : kids) {
        if (!k.compressed) continue;
        std::vector<std::pair<IdxVec, IdxVec>> m(g.size());
        bool any = false;
        for (size_t q = 0; q < g.size(); ++q) {
          for (int32_t x : g[q].first) m[q].first.push_back(x >= 0 && x < s + u ? k.inv[x] : -1);
          for (int32_t y : g[q].second) m[q].second.push_back(y >= 0 && y < s + u ? k.inv[y] : -1);
          any = true;
        }
        if (any) ec->hodbf_extract(*k.cf->C, m, dst, T(1));
      }
      if (minus_S && Sptr) {
        std::vector<std::pair<IdxVec, IdxVec>> m(g);
        for (auto& pr : m) {
          for (auto& x : pr.first) x -= s;
          for (auto& y : pr.second) y -= s;
        }
        ec->extract_bf(*Sptr, m, dst, T(-1));
      }
    };
  };
  // neighbour lists in front positions (symbolic: computed once per analysis)
  const Neigh& ng = neighbours(fid, P.knn);
  const std::vector<IdxVec>& nn11 = ng.nn11;
  const std::vector<IdxVec>& nn12 = ng.nn12;
  const std::vector<IdxVec>& nn21 = ng.nn21;
  const std::vector<IdxVec>& nn22 = ng.nn22;
  Tree th = f.th_tree, t22 = f.f22_tree;
  // optional phase trace (MF_TRACE=1): wall time and kernel launches per phase on stderr
  const bool trace = getenv("MF_TRACE") && getenv("MF_TRACE")[0] == '1';
  auto tp = std::chrono::steady_clock::now();
  int64_t lp = launch_count();
  int64_t idp = cx.n_id, cpp = cx.n_copies;
  double wp = cx.t_wait;
  std::vector<double> hp(cx.t_host, cx.t_host + BFContext<T>::H_N);
  auto phase = [&](const char* name) {
    if (!trace) return;
    cx.sync();
    auto tn = std::chrono::steady_clock::now();
    static const char* hn[] = {"gemm", "rowid", "apply", "extract", "proxy", "rmv", "blk2", "sketch", "upload",
                               "hextract", "ext"};
    char hb[512];
    int o = 0;
    for (int c = 0; c < BFContext<T>::H_N; ++c)
      o += snprintf(hb + o, sizeof(hb) - o, " %s %.3f", hn[c], cx.t_host[c] - hp[c]);
    fprintf(stderr, "[mf] front %d (s=%d u=%d) %-10s %8.3f s (waiting %6.3f s) %7lld launches %6lld IDs %7lld copies |%s\n",
            fid, s, u, name, std::chrono::duration<double>(tn - tp).count(), cx.t_wait - wp,
            (long long)(launch_count() - lp), (long long)(cx.n_id - idp), (long long)(cx.n_copies - cpp), hb);
    tp = tn;
    lp = launch_count();
    idp = cx.n_id;
    cpp = cx.n_copies;
    wp = cx.t_wait;
    hp.assign(cx.t_host, cx.t_host + BFContext<T>::H_N);
  };
  const int LH = (int)th.size() - 1, L22 = (int)t22.size() - 1, L = std::min(LH, L22);
  // F12 and F21 do not depend on F11 or its inverse: with a helper context they are built by a
  // second host thread on its own stream while this thread builds F11 and F11^-1 (the phase trace
  // keeps them sequential)
  std::thread helper_th;
  std::exception_ptr helper_err;
  cudaEvent_t setup_ev = nullptr;
  struct Join {
    std::thread& t;
    cudaEvent_t& e;
    ~Join() {
      if (t.joinable()) t.join();
      if (e) cudaEventDestroy(e);
    }
  } join_guard{helper_th, setup_ev};
  if (helper >= 0 && u > 0 && !trace) {
    MF_CUDA(cudaEventCreateWithFlags(&setup_ev, cudaEventDisableTiming));
    MF_CUDA(cudaEventRecord(setup_ev, st_));   // the front's uploads (relative maps, gather context)
    int dev = 0;
    MF_CUDA(cudaGetDevice(&dev));
    helper_th = std::thread([&, dev] {
      try {
        MF_CUDA(cudaSetDevice(dev));
        BFContext<T>& hc = this->ctx(helper);
        MF_CUDA(cudaStreamWaitEvent(hc.st, setup_ev, 0));
        const size_t hm = hc.scratch.mark();
        cf.F12 = hc.entry_eval(make_ext(0, s, true, false, &hc), s, u, th, t22, L, nn12, nn21, P);
        cf.F21 = hc.entry_eval(make_ext(s, 0, true, false, &hc), u, s, t22, th, L, nn21, nn12, P);
        hc.flush();
        MF_CUDA(cudaStreamSynchronize(hc.st));
        hc.scratch.release(hm);
      } catch (...) {
        helper_err = std::current_exception();
      }
    });
  }
  cf.F11 = cx.hodbf_entry_eval(make_ext(0, 0, true, false), s, th, nn11, P);
  phase("F11");
  cf.F11inv = cx.hodbf_invert(*cf.F11, P, (uint32_t)((seed * 7 + fid) & 0xFFFFF));
  phase("F11inv");
  if (u > 0) {
    if (helper_th.joinable()) {
      helper_th.join();
      if (helper_err) std::rethrow_exception(helper_err);
    } else {
      cf.F12 = cx.entry_eval(make_ext(0, s, true, false), s, u, th, t22, L, nn12, nn21, P);
      cf.F21 = cx.entry_eval(make_ext(s, 0, true, false), u, s, t22, th, L, nn21, nn12, P);
    }
    phase("F12,F21");
    const DBF<T>* F12p = cf.F12.get();
    const DBF<T>* F21p = cf.F21.get();
    const DHODBFInv<T>* Ip = cf.F11inv.get();
    DOp<T> op;
    op.rows = u;
    op.cols = u;
    BFContext<T>* cxp = &cx;
    op.apply = [cxp, F12p, F21p, Ip, s](const Blk<T>& X, Blk<T>& Y, bool tr) {
      BFContext<T>& cx = *cxp;
      const int k = X.cols;
      Blk<T> a = new_blk<T>(cx.scratch, s, k), b = new_blk<T>(cx.scratch, s, k);
      std::vector<Blk<T>> xs{X}, as{a};
      std::vector<const DBF<T>*> one{tr ? F21p : F12p};
      cx.apply(one, xs, as, tr, false);                 // F12 x   (or F21^T x)
      cx.inv_apply(*Ip, a, b, tr, 0, 0);                // F11^-1 . (or F11^-T .)
      std::vector<Blk<T>> bs{b}, ys{Y};
      std::vector<const DBF<T>*> two{tr ? F12p : F21p};
      cx.apply(two, bs, ys, tr, false);                 // F21 .   (or F12^T .)
    };
    auto S = cx.random_matvec(op, t22, t22, L22, P, (uint32_t)((seed * 13 + fid) & 0xFFFFF));
    Sptr = S.get();
    phase("S");
    if (f.parent >= 0) cf.C = cx.hodbf_entry_eval(make_ext(s, s, false, true), u, t22, nn22, P);
    phase("C");
    Sptr = nullptr;
    cf.max_rank = std::max({cf.F11->max_rank(), cf.F12->max_rank(), cf.F21->max_rank(), S->max_rank(),
                            cf.C ? cf.C->max_rank() : 0});
  } else {
    cf.max_rank = cf.F11->max_rank();
  }
  cf.upd32.resize(u);
  for (int i = 0; i < u; ++i) cf.upd32[i] = (int32_t)f.upd[i];
  upload(cf.d_upd32, cf.upd32, st_);
  MF_CUDA(cudaStreamSynchronize(st_));
  cx.check_status();
  cx.scratch.release(scratch_mark);   // the stream is idle: the work buffers can be reused
  cf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  std::lock_guard<std::mutex> lk(fronts_mu_);
  fronts[fid] = std::move(cfp);
}

template <typename T>
void CompressedPart<T>::densify_C(int fid, const FrontDev<T>& fd, int w) {
  BFContext<T>& cx = ctx(w);
  const cudaStream_t st_ = stream(w);
  CompFront<T>* cfp;
  {
    std::lock_guard<std::mutex> lk(fronts_mu_);
    cfp = fronts.at(fid).get();
  }
  CompFront<T>& cf = *cfp;
  if (!cf.C || cf.u == 0) return;
  const int u = cf.u;
  const size_t mk = cx.scratch.mark();
  Blk<T> I = new_blk<T>(cx.scratch, u, u);
  cx.zero(I);
  {
    std::vector<T> ones(u, T(1));
    // identity: set the diagonal of the real plane through strided copies
    MF_CUDA(cudaMemcpy2DAsync(I.p, (I.ld + 1) * sizeof(T), ones.data(), sizeof(T), sizeof(T), u,
                              cudaMemcpyHostToDevice, st_));
    MF_CUDA(cudaStreamSynchronize(st_));
  }
  Blk<T> Cd;
  Cd.p = fd.C; Cd.rows = u; Cd.cols = u; Cd.ld = fd.lu; Cd.plane = fd.pl_uu;
  cx.hodbf_apply(*cf.C, I, Cd, false);
  cx.scratch.release(mk);   // stream order makes later reuse of the scratch safe
}

template <typename T>
void CompressedPart<T>::forward(const std::vector<int>& fids, Blk<T>& X) {
  // all compressed fronts of one level at once: w_f = F11_f^-1 x_s(f), x_s(f) = w_f, x_u(f) -= F21_f w_f
  const int k = X.cols;
  const size_t mk = cx.scratch.mark();
  std::vector<const DHODBFInv<T>*> inv;
  std::vector<Blk<T>> xs, ws;
  std::vector<CompFront<T>*> cfs;
  for (int fid : fids) {
    CompFront<T>& cf = *fronts.at(fid);
    cfs.push_back(&cf);
    inv.push_back(cf.F11inv.get());
    xs.push_back(X.sub((int)cf.sep_begin, 0, cf.s, k));
    ws.push_back(new_blk<T>(cx.scratch, cf.s, k));
  }
  cx.inv_apply_multi(inv, xs, ws, false);
  std::vector<Blk2Job<T>> cp;
  for (size_t q = 0; q < cfs.size(); ++q) {
    Blk2Job<T> j{};
    j.src = ws[q].p; j.splane = ws[q].plane; j.sld = ws[q].ld; j.dst = xs[q].p; j.dplane = xs[q].plane;
    j.dld = xs[q].ld; j.rows = cfs[q]->s; j.cols = k; j.alpha = T(1); j.mode = 3;
    cp.push_back(j);
  }
  int64_t mx = 0;
  for (auto& j : cp) mx = std::max<int64_t>(mx, (int64_t)j.rows * j.cols);
  launch_blk2<T>(cx.stage(cp.data(), cp.size()), (int)cp.size(), mx, st_);
  std::vector<const DBF<T>*> b;
  std::vector<Blk<T>> wu, ts;
  std::vector<size_t> which;
  for (size_t q = 0; q < cfs.size(); ++q) {
    if (cfs[q]->u == 0) continue;
    b.push_back(cfs[q]->F21.get());
    wu.push_back(ws[q]);
    ts.push_back(new_blk<T>(cx.scratch, cfs[q]->u, k));
    which.push_back(q);
  }
  if (!b.empty()) {
    cx.apply(b, wu, ts, false, false);
    IdxVec cols = iota_vec(k);
    const int32_t* dc = static_cast<const int32_t*>(cx.upload(cols.data(), (size_t)k * 4));
    std::vector<PlaceJob<T>> pls;
    int64_t mxp = 0;
    for (size_t t = 0; t < b.size(); ++t) {
      const CompFront<T>& cf = *cfs[which[t]];
      PlaceJob<T> pl{};
      pl.src = ts[t].p; pl.splane = ts[t].plane; pl.sld = ts[t].ld;
      pl.rows = cf.d_upd32.template as<int32_t>(); pl.cols = dc; pl.nr = cf.u; pl.nc = k;
      pl.dst = X.p; pl.dplane = X.plane; pl.dld = X.ld; pl.sign = T(-1);
      pl.atomic = b.size() > 1 ? 1 : 0;   // sibling fronts share update rows
      pls.push_back(pl);
      mxp = std::max<int64_t>(mxp, (int64_t)cf.u * k);
    }
    launch_place<T>(cx.stage(pls.data(), pls.size()), (int)pls.size(), mxp, st_);
  }
  cx.scratch.release(mk);   // stream order makes later reuse of the scratch safe
}

template <typename T>
void CompressedPart<T>::backward(const std::vector<int>& fids, Blk<T>& X) {
  // all compressed fronts of one level at once: x_s(f) -= F11_f^-1 F12_f x_u(f)
  const int k = X.cols;
  const size_t mk = cx.scratch.mark();
  std::vector<CompFront<T>*> cfs;
  for (int fid : fids) {
    CompFront<T>& cf = *fronts.at(fid);
    if (cf.u > 0) cfs.push_back(&cf);
  }
  if (cfs.empty()) return;
  std::vector<Blk<T>> gs, vs, zs, xs;
  std::vector<Blk2Job<T>> gj;
  std::vector<const DBF<T>*> b;
  std::vector<const DHODBFInv<T>*> inv;
  int64_t mx = 0;
  for (CompFront<T>* cf : cfs) {
    Blk<T> g = new_blk<T>(cx.scratch, cf->u, k);
    Blk2Job<T> j{};
    j.src = X.p; j.splane = X.plane; j.sld = X.ld; j.dst = g.p; j.dplane = g.plane; j.dld = g.ld;
    j.rows = cf->u; j.cols = k; j.alpha = T(1); j.mode = 4;
    j.ridx = cf->d_upd32.template as<int32_t>(); j.cidx = nullptr;
    gj.push_back(j);
    mx = std::max<int64_t>(mx, (int64_t)cf->u * k);
    gs.push_back(g);
    vs.push_back(new_blk<T>(cx.scratch, cf->s, k));
    zs.push_back(new_blk<T>(cx.scratch, cf->s, k));
    xs.push_back(X.sub((int)cf->sep_begin, 0, cf->s, k));
    b.push_back(cf->F12.get());
    inv.push_back(cf->F11inv.get());
  }
  launch_blk2<T>(cx.stage(gj.data(), gj.size()), (int)gj.size(), mx, st_);
  cx.apply(b, gs, vs, false, false);
  cx.inv_apply_multi(inv, vs, zs, false);
  std::vector<Blk2Job<T>> aj;
  int64_t mxa = 0;
  for (size_t q = 0; q < cfs.size(); ++q) {
    Blk2Job<T> a{};
    a.src = zs[q].p; a.splane = zs[q].plane; a.sld = zs[q].ld; a.dst = xs[q].p; a.dplane = xs[q].plane;
    a.dld = xs[q].ld; a.rows = cfs[q]->s; a.cols = k; a.alpha = T(-1); a.mode = 2;
    aj.push_back(a);
    mxa = std::max<int64_t>(mxa, (int64_t)cfs[q]->s * k);
  }
  launch_blk2<T>(cx.stage(aj.data(), aj.size()), (int)aj.size(), mxa, st_);
  cx.scratch.release(mk);   // stream order makes later reuse of the scratch safe
}

template class CompressedPart<float>;
template class CompressedPart<double>;

}  // namespace mf
