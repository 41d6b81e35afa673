// Butterfly and HOD-BF algorithms on the GPU (Sec. 3-4; Alg. 2, 3, 4), host-driven:
// index sets, ranks and skeletons are host data; every product, ID, gather
// and solve is a batched device launch on the context's stream.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <chrono>
#include <climits>
#include <cstring>
#include <map>
#include <numeric>
#include <type_traits>

#include "bf_engine.h"

namespace mf {

namespace {

// splitmix64 (Steele, Lea, Flood 2014) for reproducible uniform sampling of proxies
inline uint64_t splitmix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  uint64_t z = x;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// cnt indices of [a, b) uniformly without replacement: the cnt smallest hashes
// h(c) = splitmix64(salt ^ (c * golden)), salt = (a << 32) | b, returned sorted.
// The order of [a, b) by hash depends on (a, b) only; it is kept per thread (ranges recur for every
// row block of a cluster-tree level) and every sample is a prefix of it.
IdxVec uniform_sample(int64_t a, int64_t b, int64_t cnt) {
  thread_local std::map<std::pair<int64_t, int64_t>, IdxVec> order_of;
  thread_local size_t cached = 0;
  auto it = order_of.find({a, b});
  if (it == order_of.end()) {
    const uint64_t salt = ((uint64_t)(a & 0xFFFFFFFF) << 32) | (uint64_t)(b & 0xFFFFFFFF);
    std::vector<std::pair<uint64_t, int32_t>> h;
    h.reserve(b - a);
    for (int64_t c = a; c < b; ++c) h.push_back({splitmix(salt ^ ((uint64_t)c * 0x9E3779B97F4A7C15ull)), (int32_t)c});
    std::sort(h.begin(), h.end());
    if (cached > (size_t(1) << 24)) {   // bound the cache (entries of all kept ranges)
      order_of.clear();
      cached = 0;
    }
    IdxVec ord(h.size());
    for (size_t k = 0; k < h.size(); ++k) ord[k] = h[k].second;
    cached += ord.size();
    it = order_of.emplace(std::make_pair(a, b), std::move(ord)).first;
  }
  const IdxVec& ord = it->second;
  const size_t n = (size_t)std::min<int64_t>(cnt, (int64_t)ord.size());
  IdxVec out(ord.begin(), ord.begin() + n);
  std::sort(out.begin(), out.end());
  return out;
}

// Proxy columns for rows X inside [a, b): alpha |X| uniform samples plus the
// knn nearest neighbours of each row that fall in [a, b); all of [a, b) when
// (alpha + knn) |X| >= b - a.
IdxVec proxies(const IdxVec& X, int64_t a, int64_t b, const std::vector<IdxVec>& nn, int alpha, int knn) {
  const int64_t size = b - a;
  IdxVec out;
  if ((int64_t)(alpha + knn) * (int64_t)X.size() >= size) {
    out.resize(size);
    std::iota(out.begin(), out.end(), (int32_t)a);
    return out;
  }
  out = uniform_sample(a, b, (int64_t)alpha * X.size());
  out.reserve(out.size() + (size_t)knn * X.size());
  for (int32_t x : X) {
    if (x < 0 || x >= (int32_t)nn.size()) continue;
    int k = 0;
    for (int32_t c : nn[x]) {
      if (k++ >= knn) break;
      if (c >= a && c < b) out.push_back(c);
    }
  }
  std::sort(out.begin(), out.end());
  out.erase(std::unique(out.begin(), out.end()), out.end());
  return out;
}

IdxVec cat(const IdxVec& a, const IdxVec& b) {
  IdxVec o(a);
  o.insert(o.end(), b.begin(), b.end());
  return o;
}

IdxVec range_vec(int64_t a, int64_t b) {
  IdxVec o(b - a);
  std::iota(o.begin(), o.end(), (int32_t)a);
  return o;
}

template <typename T>
GemmDesc<T> gdesc(int m, int n, int k, int ta, int tb, T alpha, T beta, const Blk<T>& A, const Blk<T>& B,
                  const Blk<T>& C) {
  GemmDesc<T> d;
  d.m = m; d.n = n; d.k = k; d.transA = ta; d.transB = tb; d.alpha = alpha; d.beta = beta;
  d.A = A.pm(); d.B = B.pm(); d.C = C.pm();
  return d;
}

// C = alpha (op(A1) op(B1) + op(A2) op(B2)) + beta C as one two-term product (k1 + k2 reduction
// indices; narrow kernel only)
template <typename T>
GemmDesc<T> gdesc2(int m, int n, int k1, int k2, int ta, int tb, T alpha, T beta, const Blk<T>& A1, const Blk<T>& B1,
                   const Blk<T>& A2, const Blk<T>& B2, const Blk<T>& C) {
  if (k1 == 0) return gdesc<T>(m, n, k2, ta, tb, alpha, beta, A2, B2, C);
  GemmDesc<T> d = gdesc<T>(m, n, k1 + k2, ta, tb, alpha, beta, A1, B1, C);
  if (k2 > 0) {
    d.k1 = k1;
    d.A2 = A2.pm();
    d.B2 = B2.pm();
  }
  return d;
}

}  // namespace

Tree subtree(const Tree& t, int l0, int i0, int depth);
Tree extend_tree(const Tree& t, int depth);

Tree subtree(const Tree& t, int l0, int i0, int depth) {
  const int64_t a0 = t[l0][i0].a;
  Tree out;
  for (int d = 0; d <= depth; ++d) {
    std::vector<Range> lv;
    for (int k = i0 * (1 << d); k < (i0 + 1) * (1 << d); ++k) lv.push_back({t[l0 + d][k].a - a0, t[l0 + d][k].b - a0});
    out.push_back(std::move(lv));
  }
  return out;
}

Tree extend_tree(const Tree& t, int depth) {
  Tree out(t.begin(), t.begin() + std::min<size_t>(t.size(), depth + 1));
  while ((int)out.size() < depth + 1) {
    std::vector<Range> nw;
    for (auto& r : out.back()) {
      int64_t m = r.a + (r.b - r.a + 1) / 2;
      nw.push_back({r.a, m});
      nw.push_back({m, r.b});
    }
    out.push_back(std::move(nw));
  }
  return out;
}

template <typename T>
int DBF<T>::max_rank() const {
  int r = 0;
  for (auto& lv : Osk)
    for (auto& s : lv) r = std::max(r, (int)s.size());
  for (auto& lv : Ssk)
    for (auto& s : lv) r = std::max(r, (int)s.size());
  return r;
}

template <typename T>
double DBF<T>::storage() const {
  double s = 0;
  for (auto& lv : U)
    for (auto& b : lv) s += (double)b.rows * b.cols;
  for (auto& lv : V)
    for (auto& b : lv) s += (double)b.rows * b.cols;
  for (auto& b : B) s += (double)b.rows * b.cols;
  return s;
}

template <typename T>
int DHODBF<T>::max_rank() const {
  int r = 0;
  for (auto& lv : off)
    for (auto& b : lv)
      if (b) r = std::max(r, b->max_rank());
  return r;
}

template <typename T>
double DHODBF<T>::storage() const {
  double s = 0;
  for (auto& d : D) s += (double)d.rows * d.cols;
  for (auto& lv : off)
    for (auto& b : lv)
      if (b) s += b->storage();
  return s;
}

template <typename T>
double DHODBFInv<T>::storage() const {
  double s = 0;
  for (auto& d : Dinv) s += (double)d.rows * d.cols;
  for (auto& lv : M)
    for (auto& b : lv)
      if (b) s += b->storage();
  return s;
}

// ---------------------------------------------------------------------------
// context and primitives
// ---------------------------------------------------------------------------
template <typename T>
BFContext<T>::BFContext(cudaStream_t s, size_t pb, size_t sb) : st(s) {
  persist.init(pb);
  scratch.init(sb);
  status.alloc(sizeof(int32_t));
  MF_CUDA(cudaMemsetAsync(status.p, 0, sizeof(int32_t), st));
}

template <typename T>
BFContext<T>::BFContext(cudaStream_t s, Arena* shared_persist, size_t sb) : st(s) {
  persist.share(shared_persist);
  scratch.init(sb);
  status.alloc(sizeof(int32_t));
  MF_CUDA(cudaMemsetAsync(status.p, 0, sizeof(int32_t), st));
}

template <typename T>
BFContext<T>::~BFContext() {
  if (ring) cudaFreeHost(ring);
  for (int i = 0; i < 2; ++i) {
    if (side[i]) cudaStreamDestroy(side[i]);
    if (ev_join[i]) cudaEventDestroy(ev_join[i]);
  }
  if (ev_fork) cudaEventDestroy(ev_fork);
}

namespace {
constexpr size_t kRingBytes = size_t(128) << 20;
}

template <typename T>
void BFContext<T>::sync() {
  if (cap_mode == 2) {   // not allowed while capturing
    cap_bad = true;
    return;
  }
  auto t0 = std::chrono::steady_clock::now();
  MF_CUDA(cudaStreamSynchronize(st));
  t_wait += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

template <typename T>
void BFContext<T>::flush() {
  if (!pend || cap_mode == 2) return;
  if (ring_dev) {   // mapped ring: the kernels read the staged bytes in place
    pend = false;
    return;
  }
  MF_CUDA(cudaMemcpyAsync(dring.as<char>() + pend_begin, ring + pend_begin, ring_off - pend_begin,
                          cudaMemcpyHostToDevice, st));
  ++n_copies;
  pend = false;
}

template <typename T>
const void* BFContext<T>::upload(const void* src, size_t bytes) {
  HostTimer ht_(t_host + H_UPLOAD);
  if (cap_mode == 2) {
    const size_t o = (cap_off + 15) & ~size_t(15);
    if (o + bytes > cap_cap) {
      cap_bad = true;
      return cap_dev;
    }
    if (bytes) std::memcpy(cap_host + o, src, bytes);
    cap_off = o + bytes;
    return cap_dev + o;
  }
  if (cap_mode == 1) cap_off = ((cap_off + 15) & ~size_t(15)) + bytes;
  if (!ring) {
    // Mapped pinned memory: a launch's descriptors are written on the host and read by the kernel
    // in place (coherent host memory on the GPU's side), which saves one copy per launch; host
    // writes before a launch are visible to it, and the ring is reused only after the stream has
    // drained.  Without mapping, a device mirror receives one copy before each launch.
    if (cudaHostAlloc(reinterpret_cast<void**>(&ring), kRingBytes, cudaHostAllocMapped) == cudaSuccess) {
      void* d = nullptr;
      if (cudaHostGetDevicePointer(&d, ring, 0) == cudaSuccess && d) ring_dev = static_cast<char*>(d);
    } else {
      cudaGetLastError();
      ring = nullptr;
      if (cudaHostAlloc(reinterpret_cast<void**>(&ring), kRingBytes, cudaHostAllocDefault) != cudaSuccess)
        throw CudaError("cudaHostAlloc of the staging ring failed");
    }
    if (!ring_dev) dring.alloc(kRingBytes);
    ring_cap = kRingBytes;
  }
  if (bytes == 0) return ring_dev ? static_cast<const void*>(ring_dev) : dring.p;
  if (bytes > ring_cap / 4) {   // large: a scratch copy of its own
    void* d = scratch.take(bytes);
    flush();
    MF_CUDA(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, st));
    sync();
    ++n_copies;
    return d;
  }
  size_t o = (ring_off + 15) & ~size_t(15);
  if (o + bytes > ring_cap) {   // wrap: once the stream drains, nothing reads the ring any more
    flush();
    sync();
    o = 0;
  }
  std::memcpy(ring + o, src, bytes);
  if (!pend) {
    pend_begin = o;
    pend = true;
  }
  ring_off = o + bytes;
  return (ring_dev ? ring_dev : dring.as<char>()) + o;
}

template <typename T>
bool BFContext<T>::capture_end() {
  cap_mode = 0;
  if (cap_bad) return false;
  MF_CUDA(cudaMemcpyAsync(cap_dev, cap_host, cap_off, cudaMemcpyHostToDevice, st));
  MF_CUDA(cudaStreamSynchronize(st));
  return true;
}

template <typename T>
void BFContext<T>::h2d(void* dst, const void* src, size_t bytes) {
  flush();
  if (bytes == 0) return;
  if (cap_mode == 2) {   // a memcpy node from the persistent blob
    const size_t o = (cap_off + 15) & ~size_t(15);
    if (o + bytes > cap_cap) {
      cap_bad = true;
      return;
    }
    std::memcpy(cap_host + o, src, bytes);
    cap_off = o + bytes;
    MF_CUDA(cudaMemcpyAsync(dst, cap_host + o, bytes, cudaMemcpyHostToDevice, st));
    return;
  }
  if (cap_mode == 1) cap_off = ((cap_off + 15) & ~size_t(15)) + bytes;
  if (!ring) upload(nullptr, 0);
  if (bytes > ring_cap / 4) {
    MF_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
    sync();
    ++n_copies;
    return;
  }
  size_t o = (ring_off + 255) & ~size_t(255);
  if (o + bytes > ring_cap) {          // wrap: every earlier copy out of the ring has completed after this
    sync();
    o = 0;
  }
  std::memcpy(ring + o, src, bytes);
  MF_CUDA(cudaMemcpyAsync(dst, ring + o, bytes, cudaMemcpyHostToDevice, st));
  ++n_copies;
  ring_off = o + bytes;
}

template <typename T>
void BFContext<T>::gemm_stages(std::map<int, std::vector<GemmDesc<T>>>& stages) {
  if constexpr (std::is_same<T, float>::value) {
    std::vector<GemmDesc<T>> D;
    std::vector<GemmTile> tl;
    std::vector<std::pair<size_t, size_t>> span;   // tiles of each launch: [first, last)
    bool tc = true;
    for (auto& kv : stages) {
      int maxn = 0;
      const size_t t0 = tl.size();
      for (auto& d : kv.second) {
        if (d.m <= 0 || d.n <= 0) continue;
        tc = tc && gemm_nrhs_tc_ok(d);
        maxn = std::max(maxn, (int)d.n);
        for (int i = 0; i < (d.m + gemm_nrhs_tc_rows() - 1) / gemm_nrhs_tc_rows(); ++i)
          tl.push_back({(int)D.size(), i, 0, 0});
        D.push_back(d);
      }
      tc = tc && (maxn == 0 || maxn >= 48);
      if (!tc) break;
      if (tl.size() > t0) span.push_back({t0, tl.size()});
    }
    if (tc) {
      if (D.empty()) return;
      HostTimer ht_(t_host + H_GEMM);
      double fl = 0, by = 0;
      for (auto& d : D) {
        fl += 8.0 * d.m * d.n * d.k;
        by += gemm_bytes(d);
      }
      flops += fl;
      bytes += by;
      const GemmDesc<T>* dd = static_cast<const GemmDesc<T>*>(upload(D.data(), D.size() * sizeof(GemmDesc<T>)));
      const GemmTile* dt = stage(tl.data(), tl.size());
      for (auto& sp : span) {
        auto go = [&] {
          launch_gemm_nrhs_tc(dd, dt + sp.first, (int)(sp.second - sp.first), status.template as<int32_t>(), st);
        };
        if (prof && prof->on) {
          double f1 = 0, b1 = 0;
          for (size_t t = sp.first; t < sp.second; ++t)
            if (tl[t].tm == 0) {
              f1 += 8.0 * D[tl[t].desc].m * D[tl[t].desc].n * D[tl[t].desc].k;
              b1 += gemm_bytes(D[tl[t].desc]);
            }
          prof->time(st, f1, b1, go);
        } else {
          go();
        }
      }
      return;
    }
  }
  for (auto& kv : stages) gemm(kv.second);
}

template <typename T>
void BFContext<T>::check_status() {
  int32_t v = 0;
  MF_CUDA(cudaMemcpyAsync(&v, status.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  sync();
  if (v == 2) throw TimeoutError("a bounded wait in a tensor-core kernel expired");
  if (v != 0) throw SingularError("singular block in a compressed front (zero pivot or indefinite normal equations)");
}

template <typename T>
void BFContext<T>::gemm(std::vector<GemmDesc<T>>& descs) {
  HostTimer ht_(t_host + H_GEMM);
  std::vector<GemmDesc<T>> D;
  D.reserve(descs.size());
  int maxn = 0, maxk = 1;
  bool two = false;
  for (auto& d : descs) {
    if (d.m <= 0 || d.n <= 0) continue;
    two = two || d.k1 > 0;
    D.push_back(d);
    flops += 8.0 * d.m * d.n * d.k;
    bytes += gemm_bytes(d);
    maxn = std::max(maxn, (int)d.n);
    maxk = std::max(maxk, (int)d.k);
  }
  if (D.empty()) return;
  if constexpr (std::is_same<T, float>::value) {
    // complex64 products of 48 to 64 vectors: the tensor-core kernel (the 64 vectors fill its
    // M = 128 rows with both planes; narrower blocks run faster on the SIMT kernel's 16- and
    // 32-column tiles, measured on the solve's 16 right-hand sides)
    bool tc = maxn >= 48;
    for (auto& d : D) tc = tc && gemm_nrhs_tc_ok(d);
    if (tc) {
      std::vector<GemmTile> tl;
      for (size_t idx = 0; idx < D.size(); ++idx)
        for (int i = 0; i < (D[idx].m + gemm_nrhs_tc_rows() - 1) / gemm_nrhs_tc_rows(); ++i)
        tl.push_back({(int)idx, i, 0, 0});
      const GemmDesc<T>* dd = static_cast<const GemmDesc<T>*>(upload(D.data(), D.size() * sizeof(GemmDesc<T>)));
      const GemmTile* dt = stage(tl.data(), tl.size());
      auto go = [&] { launch_gemm_nrhs_tc(dd, dt, (int)tl.size(), status.template as<int32_t>(), st); };
      if (prof && prof->on) {
        double fl = 0, by = 0;
        for (auto& d : D) {
          fl += 8.0 * d.m * d.n * d.k;
          by += gemm_bytes(d);
        }
        prof->time(st, fl, by, go);
      } else {
        go();
      }
      return;
    }
  }
  // narrow products (blocks of vectors, n <= 128): 32-row tiles of the streaming kernel; else 64 x 64 tiles
  const int nb = gemm_nrhs_width(maxn, sizeof(T));
  const int tr = nb ? GEMM_NRHS_ROWS : GEMM_TILE;
  std::vector<GemmTile> tl;
  for (size_t idx = 0; idx < D.size(); ++idx) {
    const auto& d = D[idx];
    const int tn = (d.n + (nb ? nb : GEMM_TILE) - 1) / (nb ? nb : GEMM_TILE);
    for (int i = 0; i < (d.m + tr - 1) / tr; ++i)
      for (int j = 0; j < tn; ++j) tl.push_back({(int)idx, i, j, 0});
  }
  const GemmDesc<T>* dd = static_cast<const GemmDesc<T>*>(upload(D.data(), D.size() * sizeof(GemmDesc<T>)));
  const GemmTile* dt = stage(tl.data(), tl.size());
  if (nb) {
    auto go = [&] { launch_gemm_nrhs<T>(dd, dt, (int)tl.size(), nb, gemm_nrhs_split((int)tl.size(), maxk), maxk, st, two); };
    if (prof && prof->on) {
      double fl = 0, by = 0;
      for (auto& d : D) {
        fl += 8.0 * d.m * d.n * d.k;
        by += gemm_bytes(d);
      }
      prof->time(st, fl, by, go);
    } else {
      go();
    }
  } else {
    launch_gemm<T>(dd, dt, (int)tl.size(), st);
  }
}

template <typename T>
void BFContext<T>::zero(Blk<T>& b) {
  if (b.rows <= 0 || b.cols <= 0) return;
  if ((int64_t)b.rows * b.ld == b.plane) {   // the two planes are adjacent
    MF_CUDA(cudaMemsetAsync(b.p, 0, sizeof(T) * 2 * (size_t)b.plane, st));
    return;
  }
  MF_CUDA(cudaMemsetAsync(b.p, 0, sizeof(T) * (size_t)b.rows * b.ld, st));
  MF_CUDA(cudaMemsetAsync(b.p + b.plane, 0, sizeof(T) * (size_t)b.rows * b.ld, st));
}

template <typename T>
static void run_blk2(BFContext<T>& cx, std::vector<Blk2Job<T>>& jobs) {
  typename BFContext<T>::HostTimer ht_(cx.t_host + BFContext<T>::H_BLK2);
  if (jobs.empty()) return;
  int64_t mx = 0;
  for (auto& j : jobs) mx = std::max<int64_t>(mx, (int64_t)j.rows * j.cols);
  const Blk2Job<T>* dj = cx.stage(jobs.data(), jobs.size());
  launch_blk2<T>(dj, (int)jobs.size(), mx, cx.st);
}

template <typename T>
static const int32_t* dev_idx(BFContext<T>& cx, const IdxVec& v) {
  return static_cast<const int32_t*>(cx.upload(v.data(), v.size() * 4));
}

template <typename T>
void BFContext<T>::row_ids(const std::vector<Blk<T>>& Ms, double tol, int max_rank, std::vector<IdxVec>& sk,
                           std::vector<Blk<T>>& Us) {
  HostTimer ht_(t_host + H_ROWID);
  const size_t nj = Ms.size();
  sk.assign(nj, {});
  Us.assign(nj, Blk<T>());
  if (!nj) return;
  std::vector<IdJob<T>> jobs, sjobs, rjobs;
  std::vector<size_t> which;
  int smax_m = 1, smax_n = 1, rmax_m = 1, rmax_n = 1;
  size_t sbytes = 0;
  int32_t* dsk = nullptr;
  int32_t* drk = scratch.takeT<int32_t>(nj);
  std::vector<int> kmaxv(nj, 0);
  size_t sktot = 0;
  for (size_t q = 0; q < nj; ++q) {
    int m = Ms[q].rows, n = Ms[q].cols;
    int kmax = std::min(m, n);
    if (max_rank > 0) kmax = std::min(kmax, max_rank);
    kmaxv[q] = kmax;
    sktot += std::max(kmax, 1);
  }
  dsk = scratch.takeT<int32_t>(sktot);
  size_t skoff = 0;
  int max_m = 1, max_n = 1;
  std::vector<size_t> skoffv(nj);
  for (size_t q = 0; q < nj; ++q) {
    skoffv[q] = skoff;
    int m = Ms[q].rows, n = Ms[q].cols, kmax = kmaxv[q];
    skoff += std::max(kmax, 1);
    Blk<T> U;
    U.rows = m;
    U.cols = 0;
    U.ld = std::max(1, (kmax + 3) & ~3);
    U.plane = (int64_t)std::max(m, 1) * U.ld;
    U.p = persist.takeT<T>(2 * (size_t)U.plane);
    Us[q] = U;
    if (m == 0 || n == 0 || kmax == 0) continue;
    IdJob<T> j;
    j.M = Ms[q].p;
    j.plane = Ms[q].plane;
    j.ld = Ms[q].ld;
    j.m = m;
    j.n = n;
    j.U = U.p;
    j.uplane = U.plane;
    j.ldu = (int32_t)U.ld;
    j.sk = dsk + skoffv[q];
    j.rank = drk + q;
    j.wplane = (int64_t)m * n;
    const size_t sb = row_id_smem_bytes(m, n, sizeof(T), true);
    if (sizeof(T) == 4 && m <= 128 && n <= 128) {   // rows in registers
      j.work = nullptr;
      rjobs.push_back(j);
      rmax_m = std::max(rmax_m, m);
      rmax_n = std::max(rmax_n, n);
    } else if (sb <= kRowIdSmemCap) {   // QR work in shared memory
      j.work = nullptr;
      sjobs.push_back(j);
      smax_m = std::max(smax_m, m);
      smax_n = std::max(smax_n, n);
      sbytes = std::max(sbytes, sb);
    } else {
      j.work = scratch.takeT<T>(2 * (size_t)m * n);
      jobs.push_back(j);
      max_m = std::max(max_m, m);
      max_n = std::max(max_n, n);
    }
    which.push_back(q);
  }
  MF_CUDA(cudaMemsetAsync(drk, 0, nj * 4, st));
  // MF_TRACE=2: one line per call with the three kernels' job counts, largest shapes and GPU time
  static const bool id_trace = getenv("MF_TRACE") && getenv("MF_TRACE")[0] == '2';
  cudaEvent_t ie0 = nullptr, ie1 = nullptr;
  if (id_trace && cap_mode != 2) {
    MF_CUDA(cudaEventCreate(&ie0));
    MF_CUDA(cudaEventCreate(&ie1));
    MF_CUDA(cudaEventRecord(ie0, st));
  }
  // small matrices with their rows in registers, matrices whose QR work fits in shared memory,
  // and the others (work in global memory, a thread-block cluster each): three independent
  // kernels, run side by side on forked streams when more than one kind is present
  auto up = [&](const std::vector<IdJob<T>>& v) {
    return v.empty() ? nullptr : static_cast<const IdJob<T>*>(upload(v.data(), v.size() * sizeof(IdJob<T>)));
  };
  const IdJob<T>* drj = up(rjobs);
  const IdJob<T>* dsj = up(sjobs);
  const IdJob<T>* dgj = up(jobs);
  flush();   // one copy for the three job tables
  const int kinds = (drj ? 1 : 0) + (dsj ? 1 : 0) + (dgj ? 1 : 0);
  const bool fork = kinds > 1 && cap_mode != 2;
  if (fork) {
    if (!ev_fork) {
      MF_CUDA(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
      for (int i = 0; i < 2; ++i) {
        MF_CUDA(cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking));
        MF_CUDA(cudaEventCreateWithFlags(&ev_join[i], cudaEventDisableTiming));
      }
    }
    MF_CUDA(cudaEventRecord(ev_fork, st));
    for (int i = 0; i < 2; ++i) MF_CUDA(cudaStreamWaitEvent(side[i], ev_fork, 0));
  }
  if (drj) {
    if (launch_row_id_reg<T>(drj, (int)rjobs.size(), rmax_m, rmax_n, (T)tol, max_rank, fork ? side[0] : st) != 0)
      throw std::runtime_error("ID block too large for the register row-ID kernel");
    n_id += (int64_t)rjobs.size();
  }
  if (dgj) {
    if (launch_row_id<T>(dgj, (int)jobs.size(), max_m, max_n, (T)tol, max_rank, fork ? side[1] : st) != 0)
      throw std::runtime_error("ID block too large for the row-ID kernel (" + std::to_string(max_m) + " x " +
                               std::to_string(max_n) + ")");
    n_id += (int64_t)jobs.size();
  }
  if (dsj) {
    if (launch_row_id<T>(dsj, (int)sjobs.size(), smax_m, smax_n, (T)tol, max_rank, st, true, sbytes) != 0)
      throw std::runtime_error("ID block too large for the shared-memory row-ID kernel");
    n_id += (int64_t)sjobs.size();
  }
  if (fork)
    for (int i = 0; i < 2; ++i) {
      MF_CUDA(cudaEventRecord(ev_join[i], side[i]));
      MF_CUDA(cudaStreamWaitEvent(st, ev_join[i], 0));
    }
  std::vector<int32_t> hr(nj), hs(sktot);
  if (ie0) MF_CUDA(cudaEventRecord(ie1, st));
  MF_CUDA(cudaMemcpyAsync(hr.data(), drk, nj * 4, cudaMemcpyDeviceToHost, st));
  MF_CUDA(cudaMemcpyAsync(hs.data(), dsk, sktot * 4, cudaMemcpyDeviceToHost, st));
  sync();
  if (ie0) {
    float ms = 0;
    MF_CUDA(cudaEventElapsedTime(&ms, ie0, ie1));
    fprintf(stderr, "[id] reg %zu (%dx%d) smem %zu (%dx%d) global %zu (%dx%d) max_rank %d  %.3f ms\n", rjobs.size(),
            rmax_m, rmax_n, sjobs.size(), smax_m, smax_n, jobs.size(), max_m, max_n, max_rank, ms);
    cudaEventDestroy(ie0);
    cudaEventDestroy(ie1);
  }
  for (size_t q = 0; q < nj; ++q) {
    int r = hr[q];
    Us[q].cols = r;
    sk[q].assign(hs.begin() + skoffv[q], hs.begin() + skoffv[q] + r);
    max_rank_seen = std::max(max_rank_seen, r);
    flops += 8.0 * 2.0 * Ms[q].rows * (double)Ms[q].cols * r;
  }
}

// ---------------------------------------------------------------------------
// apply: Y (=|+=) K X for several butterflies at once (stage-merged launches)
// ---------------------------------------------------------------------------
template <typename T>
void BFContext<T>::apply(const std::vector<const DBF<T>*>& bfs, const std::vector<Blk<T>>& X, std::vector<Blk<T>>& Y,
                         bool transpose, bool accumulate) {
  HostTimer ht_(t_host + H_APPLY);
  const size_t nb = bfs.size();
  if (!nb) return;
  std::map<int, std::vector<GemmDesc<T>>> stages;   // stage index -> descs
  // narrow products (n <= 128): the two halves of a pulled level go into one two-term product
  int maxcols = 0;
  for (size_t q = 0; q < nb; ++q) maxcols = std::max(maxcols, (int)X[q].cols);
  const bool two = gemm_nrhs_width(maxcols, sizeof(T)) != 0;
  const T one = T(1), zero = T(0), beta_out = accumulate ? T(1) : T(0);
  for (size_t q = 0; q < nb; ++q) {
    const DBF<T>& bf = *bfs[q];
    const int k = X[q].cols;   // block widths may differ between butterflies
    const int L = bf.L, lc = bf.lc;
    auto vec_buf = [&](const std::vector<int>& ranks, std::vector<Blk<T>>& out) {
      size_t tot = 0;
      for (int r : ranks) tot += (size_t)r;
      Blk<T> all;
      all.rows = (int)tot;
      all.cols = k;
      all.ld = k;
      all.plane = (int64_t)std::max<size_t>(tot, 1) * k;
      all.p = scratch.takeT<T>(2 * (size_t)all.plane);
      out.resize(ranks.size());
      size_t o = 0;
      for (size_t p = 0; p < ranks.size(); ++p) {
        out[p] = all.sub((int)o, 0, ranks[p], k);
        o += ranks[p];
      }
    };
    // the same with the blocks laid out in the order `order` (a permutation of the block indices)
    auto vec_buf_ordered = [&](const std::vector<int>& ranks, const std::vector<int>& order,
                               std::vector<Blk<T>>& out) {
      size_t tot = 0;
      for (int r : ranks) tot += (size_t)r;
      Blk<T> all;
      all.rows = (int)tot;
      all.cols = k;
      all.ld = k;
      all.plane = (int64_t)std::max<size_t>(tot, 1) * k;
      all.p = scratch.takeT<T>(2 * (size_t)all.plane);
      out.resize(ranks.size());
      size_t o = 0;
      for (int p : order) {
        out[p] = all.sub((int)o, 0, ranks[p], k);
        o += ranks[p];
      }
    };
    int stg = 0;
    if (!transpose) {
      // right half: level 0 (V), levels 1..lc (W)
      std::vector<Blk<T>> prev, cur;
      {
        std::vector<int> rk;
        for (int j = 0; j < (1 << L); ++j) rk.push_back(bf.rc(0, 0, j));
        vec_buf(rk, cur);
        for (int j = 0; j < (1 << L); ++j) {
          const Range r = bf.ct[L][j];
          const Blk<T>& V = bf.V[0][j];
          stages[stg].push_back(gdesc<T>(bf.rc(0, 0, j), k, (int)(r.b - r.a), 1, 0, one, zero, V,
                                         X[q].sub((int)r.a, 0, (int)(r.b - r.a), k), cur[j]));
        }
        ++stg;
      }
      for (int l = 1; l <= lc; ++l) {
        prev.swap(cur);
        std::vector<int> rk;
        for (int i = 0; i < (1 << l); ++i)
          for (int j = 0; j < (1 << (L - l)); ++j) rk.push_back(bf.rc(l, i, j));
        vec_buf(rk, cur);
        for (int i = 0; i < (1 << l); ++i)
          for (int j = 0; j < (1 << (L - l)); ++j) {
            const int p = bf.pidx(l, i, j);
            const int p1 = bf.pidx(l - 1, i / 2, 2 * j);
            const int c1 = bf.rc(l - 1, i / 2, 2 * j), c2 = bf.rc(l - 1, i / 2, 2 * j + 1);
            Blk<T> in = prev[p1];
            in.rows = c1 + c2;   // (i/2, 2j) and (i/2, 2j+1) are adjacent in the level buffer
            stages[stg].push_back(gdesc<T>(bf.rc(l, i, j), k, c1 + c2, 1, 0, one, zero, bf.V[l][p], in, cur[p]));
          }
        ++stg;
      }
      // centre
      std::vector<Blk<T>> ys;
      {
        std::vector<int> rk;
        for (int i = 0; i < (1 << lc); ++i)
          for (int j = 0; j < (1 << (L - lc)); ++j) rk.push_back(bf.rr(lc, i, j));
        vec_buf(rk, ys);
        for (int i = 0; i < (1 << lc); ++i)
          for (int j = 0; j < (1 << (L - lc)); ++j) {
            const int p = bf.pidx(lc, i, j);
            stages[stg].push_back(gdesc<T>(bf.rr(lc, i, j), k, bf.rc(lc, i, j), 0, 0, one, zero, bf.B[p], cur[p], ys[p]));
          }
        ++stg;
      }
      // left half: levels lc .. L-1 -> l+1, pulled per output pair, two accumulation stages
      for (int l = lc; l < L; ++l) {
        std::vector<Blk<T>> nxt;
        std::vector<int> rk;
        for (int i = 0; i < (1 << (l + 1)); ++i)
          for (int j = 0; j < (1 << (L - l - 1)); ++j) rk.push_back(bf.rr(l + 1, i, j));
        if (two) {
          // both output halves (2i, j2) and (2i+1, j2) read the same two inputs (i, 2j2), (i, 2j2+1),
          // and the stored R blocks hold the rows of both halves: one two-term product computes
          // the pair, into a level buffer laid out so that the pair's blocks are adjacent
          std::vector<int> order;
          for (int i = 0; i < (1 << l); ++i)
            for (int j2 = 0; j2 < (1 << (L - l - 1)); ++j2)
              for (int h = 0; h < 2; ++h) order.push_back(bf.pidx(l + 1, 2 * i + h, j2));
          vec_buf_ordered(rk, order, nxt);
          for (int i = 0; i < (1 << l); ++i)
            for (int j2 = 0; j2 < (1 << (L - l - 1)); ++j2) {
              const int p0 = bf.pidx(l, i, 2 * j2), p1 = bf.pidx(l, i, 2 * j2 + 1);
              const int nrow = bf.rr(l + 1, 2 * i, j2) + bf.rr(l + 1, 2 * i + 1, j2);
              const Blk<T>& R0 = bf.U[l][p0];
              const Blk<T>& R1 = bf.U[l][p1];
              Blk<T> out = nxt[bf.pidx(l + 1, 2 * i, j2)];
              out.rows = nrow;
              stages[stg].push_back(gdesc2<T>(nrow, k, bf.rr(l, i, 2 * j2), bf.rr(l, i, 2 * j2 + 1), 0, 0, one, zero,
                                              R0.sub(0, 0, nrow, R0.cols), ys[p0], R1.sub(0, 0, nrow, R1.cols),
                                              ys[p1], out));
            }
          stg += 1;
        } else {
          vec_buf(rk, nxt);
          for (int t = 0; t < 2; ++t) {
            for (int i2 = 0; i2 < (1 << (l + 1)); ++i2)
              for (int j2 = 0; j2 < (1 << (L - l - 1)); ++j2) {
                const int i = i2 / 2, nu = 2 * j2 + t;
                const int p = bf.pidx(l, i, nu);
                const int r1 = bf.rr(l + 1, 2 * i, j2);
                const int rows0 = (i2 % 2 == 0) ? 0 : r1;
                const int nrow = bf.rr(l + 1, i2, j2);
                const Blk<T>& R = bf.U[l][p];
                stages[stg + t].push_back(gdesc<T>(nrow, k, bf.rr(l, i, nu), 0, 0, one, t == 0 ? zero : one,
                                                   R.sub(rows0, 0, nrow, R.cols), ys[p], nxt[bf.pidx(l + 1, i2, j2)]));
              }
          }
          stg += 2;
        }
        ys.swap(nxt);
      }
      for (int i = 0; i < (1 << L); ++i) {
        const Range r = bf.rt[L][i];
        const Blk<T>& U = bf.U[L][i];
        stages[stg].push_back(gdesc<T>((int)(r.b - r.a), k, bf.rr(L, i, 0), 0, 0, one, beta_out, U, ys[i],
                                       Y[q].sub((int)r.a, 0, (int)(r.b - r.a), k)));
      }
    } else {
      // transpose: U^T, R^T (two stages), B^T, W (pulled, two stages), V
      std::vector<Blk<T>> cur;
      {
        std::vector<int> rk;
        for (int i = 0; i < (1 << L); ++i) rk.push_back(bf.rr(L, i, 0));
        vec_buf(rk, cur);
        for (int i = 0; i < (1 << L); ++i) {
          const Range r = bf.rt[L][i];
          stages[stg].push_back(gdesc<T>(bf.rr(L, i, 0), k, (int)(r.b - r.a), 1, 0, one, zero, bf.U[L][i],
                                         X[q].sub((int)r.a, 0, (int)(r.b - r.a), k), cur[i]));
        }
        ++stg;
      }
      for (int l = L - 1; l >= lc; --l) {
        std::vector<Blk<T>> nxt;
        std::vector<int> rk;
        for (int i = 0; i < (1 << l); ++i)
          for (int j = 0; j < (1 << (L - l)); ++j) rk.push_back(bf.rr(l, i, j));
        vec_buf(rk, nxt);
        if (two) {
          for (int i = 0; i < (1 << l); ++i)
            for (int j = 0; j < (1 << (L - l)); ++j) {
              const int p = bf.pidx(l, i, j);
              const int r1 = bf.rr(l + 1, 2 * i, j / 2), r2 = bf.rr(l + 1, 2 * i + 1, j / 2);
              const Blk<T>& R = bf.U[l][p];
              stages[stg].push_back(gdesc2<T>(bf.rr(l, i, j), k, r1, r2, 1, 0, one, zero, R.sub(0, 0, r1, R.cols),
                                              cur[bf.pidx(l + 1, 2 * i, j / 2)], R.sub(r1, 0, r2, R.cols),
                                              cur[bf.pidx(l + 1, 2 * i + 1, j / 2)], nxt[p]));
            }
          stg += 1;
        } else {
          for (int t = 0; t < 2; ++t) {
            for (int i = 0; i < (1 << l); ++i)
              for (int j = 0; j < (1 << (L - l)); ++j) {
                const int p = bf.pidx(l, i, j);
                const int r1 = bf.rr(l + 1, 2 * i, j / 2);
                const int rows0 = t == 0 ? 0 : r1;
                const int nrow = bf.rr(l + 1, 2 * i + t, j / 2);
                const Blk<T>& R = bf.U[l][p];
                stages[stg + t].push_back(gdesc<T>(bf.rr(l, i, j), k, nrow, 1, 0, one, t == 0 ? zero : one,
                                                   R.sub(rows0, 0, nrow, R.cols), cur[bf.pidx(l + 1, 2 * i + t, j / 2)],
                                                   nxt[p]));
              }
          }
          stg += 2;
        }
        cur.swap(nxt);
      }
      std::vector<Blk<T>> ys;
      {
        std::vector<int> rk;
        for (int i = 0; i < (1 << lc); ++i)
          for (int j = 0; j < (1 << (L - lc)); ++j) rk.push_back(bf.rc(lc, i, j));
        vec_buf(rk, ys);
        for (int i = 0; i < (1 << lc); ++i)
          for (int j = 0; j < (1 << (L - lc)); ++j) {
            const int p = bf.pidx(lc, i, j);
            stages[stg].push_back(gdesc<T>(bf.rc(lc, i, j), k, bf.rr(lc, i, j), 1, 0, one, zero, bf.B[p], cur[p], ys[p]));
          }
        ++stg;
      }
      for (int l = lc; l >= 1; --l) {
        std::vector<Blk<T>> nxt;
        std::vector<int> rk;
        for (int i = 0; i < (1 << (l - 1)); ++i)
          for (int j = 0; j < (1 << (L - l + 1)); ++j) rk.push_back(bf.rc(l - 1, i, j));
        vec_buf(rk, nxt);
        if (two) {
          for (int i2 = 0; i2 < (1 << (l - 1)); ++i2)
            for (int j2 = 0; j2 < (1 << (L - l + 1)); ++j2) {
              const int j = j2 / 2, p0 = bf.pidx(l, 2 * i2, j), p1 = bf.pidx(l, 2 * i2 + 1, j);
              const int c1 = bf.rc(l - 1, i2, 2 * j);
              const int rows0 = (j2 % 2 == 0) ? 0 : c1;
              const int nrow = bf.rc(l - 1, i2, j2);
              const Blk<T>& W0 = bf.V[l][p0];
              const Blk<T>& W1 = bf.V[l][p1];
              stages[stg].push_back(gdesc2<T>(nrow, k, bf.rc(l, 2 * i2, j), bf.rc(l, 2 * i2 + 1, j), 0, 0, one, zero,
                                              W0.sub(rows0, 0, nrow, W0.cols), ys[p0], W1.sub(rows0, 0, nrow, W1.cols),
                                              ys[p1], nxt[bf.pidx(l - 1, i2, j2)]));
            }
          stg += 1;
        } else {
          for (int t = 0; t < 2; ++t) {
            for (int i2 = 0; i2 < (1 << (l - 1)); ++i2)
              for (int j2 = 0; j2 < (1 << (L - l + 1)); ++j2) {
                const int i = 2 * i2 + t, j = j2 / 2;
                const int p = bf.pidx(l, i, j);
                const int c1 = bf.rc(l - 1, i2, 2 * j);
                const int rows0 = (j2 % 2 == 0) ? 0 : c1;
                const int nrow = bf.rc(l - 1, i2, j2);
                const Blk<T>& W = bf.V[l][p];
                stages[stg + t].push_back(gdesc<T>(nrow, k, bf.rc(l, i, j), 0, 0, one, t == 0 ? zero : one,
                                                   W.sub(rows0, 0, nrow, W.cols), ys[p], nxt[bf.pidx(l - 1, i2, j2)]));
              }
          }
          stg += 2;
        }
        ys.swap(nxt);
      }
      for (int j = 0; j < (1 << L); ++j) {
        const Range r = bf.ct[L][j];
        stages[stg].push_back(gdesc<T>((int)(r.b - r.a), k, bf.rc(0, 0, j), 0, 0, one, beta_out, bf.V[0][j], ys[j],
                                       Y[q].sub((int)r.a, 0, (int)(r.b - r.a), k)));
      }
    }
  }
  // The final stage of each butterfly writes its output; butterflies with fewer stages finish earlier,
  // which is fine because outputs of different butterflies in one call are disjoint or accumulated in
  // separate calls by the callers.
  gemm_stages(stages);
}

template <typename T>
void BFContext<T>::right_transform(const DBF<T>& bf, const Blk<T>& X, std::vector<Blk<T>>& xs) {
  const int L = bf.L, lc = bf.lc, k = X.cols;
  std::vector<Blk<T>> prev, cur;
  auto buf = [&](std::vector<Blk<T>>& out, int l) {
    out.assign((size_t)1 << L, Blk<T>());
    size_t tot = 0;
    for (int p = 0; p < (1 << L); ++p) tot += (size_t)bf.Ssk[l][p].size();
    Blk<T> all;
    all.rows = (int)tot; all.cols = k; all.ld = k; all.plane = (int64_t)std::max<size_t>(tot, 1) * k;
    all.p = scratch.takeT<T>(2 * (size_t)all.plane);
    size_t o = 0;
    for (int p = 0; p < (1 << L); ++p) {
      out[p] = all.sub((int)o, 0, (int)bf.Ssk[l][p].size(), k);
      o += bf.Ssk[l][p].size();
    }
  };
  buf(cur, 0);
  std::vector<GemmDesc<T>> g;
  for (int j = 0; j < (1 << L); ++j) {
    const Range r = bf.ct[L][j];
    g.push_back(gdesc<T>(bf.rc(0, 0, j), k, (int)(r.b - r.a), 1, 0, T(1), T(0), bf.V[0][j],
                         X.sub((int)r.a, 0, (int)(r.b - r.a), k), cur[j]));
  }
  gemm(g);
  for (int l = 1; l <= lc; ++l) {
    prev.swap(cur);
    buf(cur, l);
    g.clear();
    for (int i = 0; i < (1 << l); ++i)
      for (int j = 0; j < (1 << (L - l)); ++j) {
        const int p = bf.pidx(l, i, j);
        const int p1 = bf.pidx(l - 1, i / 2, 2 * j);
        const int c1 = bf.rc(l - 1, i / 2, 2 * j), c2 = bf.rc(l - 1, i / 2, 2 * j + 1);
        Blk<T> in = prev[p1];
        in.rows = c1 + c2;
        g.push_back(gdesc<T>(bf.rc(l, i, j), k, c1 + c2, 1, 0, T(1), T(0), bf.V[l][p], in, cur[p]));
      }
    gemm(g);
  }
  xs.swap(cur);
}

// ---------------------------------------------------------------------------
// construction from entry extraction (Alg. 2), many butterflies with the same
// number of levels in lockstep: per level one extraction call (all blocks of
// all problems) and one batched ID launch.  Problem q's local indices are
// shifted by (row_off, col_off) into the index space of the extractor.
// ---------------------------------------------------------------------------
template <typename T>
void BFContext<T>::entry_eval_batch(const DExtract<T>& ext, std::vector<BFProblem<T>>& probs, const BFParams& P) {
  if (probs.empty()) return;
  const int L = probs[0].L, lc = L / 2;
  for (auto& pb : probs) {
    if (pb.L != L) throw std::runtime_error("entry_eval_batch: problems must share the level count");
    pb.out = std::make_unique<DBF<T>>();
    pb.out->init(pb.m, pb.n, pb.rt, pb.ct, L);
  }
  const size_t mk = scratch.mark();
  auto shifted = [&](const std::vector<std::pair<IdxVec, IdxVec>>& lst, const BFProblem<T>& pb,
                     std::vector<std::pair<IdxVec, IdxVec>>& g) {
    for (auto pr : lst) {
      for (auto& x : pr.first) x += (int32_t)pb.row_off;
      for (auto& y : pr.second) y += (int32_t)pb.col_off;
      g.push_back(std::move(pr));
    }
  };
  for (int l = L; l >= lc; --l) {                         // left to middle
    std::vector<std::pair<IdxVec, IdxVec>> all;
    std::vector<std::vector<std::pair<IdxVec, IdxVec>>> loc(probs.size());
    for (size_t q = 0; q < probs.size(); ++q) {
      DBF<T>& bf = *probs[q].out;
      for (int i = 0; i < (1 << l); ++i)
        for (int j = 0; j < (1 << (L - l)); ++j) {
          IdxVec X = l == L ? range_vec(bf.rt[L][i].a, bf.rt[L][i].b)
                            : cat(bf.Osk[l + 1][bf.pidx(l + 1, 2 * i, j / 2)],
                                  bf.Osk[l + 1][bf.pidx(l + 1, 2 * i + 1, j / 2)]);
          const Range c = bf.ct[L - l][j];
          HostTimer tp_(t_host + H_PROXY);
          loc[q].push_back({X, proxies(X, c.a, c.b, probs[q].nn_r, P.alpha, P.knn)});
        }
      shifted(loc[q], probs[q], all);
    }
    std::vector<Blk<T>> blocks(all.size());
    for (size_t t = 0; t < all.size(); ++t) blocks[t] = new_blk<T>(scratch, (int)all[t].first.size(), (int)all[t].second.size());
    {
      HostTimer te_(t_host + H_EXT);
      ext(all, blocks);
    }
    std::vector<IdxVec> sk;
    std::vector<Blk<T>> Us;
    row_ids(blocks, P.tol, P.max_rank, sk, Us);
    size_t t = 0;
    for (size_t q = 0; q < probs.size(); ++q) {
      DBF<T>& bf = *probs[q].out;
      for (size_t p = 0; p < loc[q].size(); ++p, ++t) {
        bf.U[l][p] = Us[t];
        IdxVec o;
        for (int32_t x : sk[t]) o.push_back(loc[q][p].first[x]);
        bf.Osk[l][p] = o;
      }
    }
    scratch.release(mk);
  }
  for (int l = 0; l <= lc; ++l) {                         // right to middle (column IDs)
    std::vector<std::pair<IdxVec, IdxVec>> all;
    std::vector<std::vector<std::pair<IdxVec, IdxVec>>> loc(probs.size());
    for (size_t q = 0; q < probs.size(); ++q) {
      DBF<T>& bf = *probs[q].out;
      for (int i = 0; i < (1 << l); ++i)
        for (int j = 0; j < (1 << (L - l)); ++j) {
          IdxVec Y = l == 0 ? range_vec(bf.ct[L][j].a, bf.ct[L][j].b)
                            : cat(bf.Ssk[l - 1][bf.pidx(l - 1, i / 2, 2 * j)],
                                  bf.Ssk[l - 1][bf.pidx(l - 1, i / 2, 2 * j + 1)]);
          const Range r = bf.rt[l][i];
          HostTimer tp_(t_host + H_PROXY);
          loc[q].push_back({proxies(Y, r.a, r.b, probs[q].nn_c, P.alpha, P.knn), Y});
        }
      shifted(loc[q], probs[q], all);
    }
    std::vector<Blk<T>> blocks(all.size()), tblocks(all.size());
    for (size_t t = 0; t < all.size(); ++t) {
      blocks[t] = new_blk<T>(scratch, (int)all[t].first.size(), (int)all[t].second.size());
      tblocks[t] = new_blk<T>(scratch, (int)all[t].second.size(), (int)all[t].first.size());
    }
    {
      HostTimer te_(t_host + H_EXT);
      ext(all, blocks);
    }
    std::vector<Blk2Job<T>> tj;
    for (size_t t = 0; t < all.size(); ++t) {
      Blk2Job<T> jb{};
      jb.src = blocks[t].p; jb.splane = blocks[t].plane; jb.sld = blocks[t].ld;
      jb.dst = tblocks[t].p; jb.dplane = tblocks[t].plane; jb.dld = tblocks[t].ld;
      jb.rows = blocks[t].rows; jb.cols = blocks[t].cols; jb.mode = 0; jb.alpha = T(1);
      if (jb.rows && jb.cols) tj.push_back(jb);
    }
    run_blk2(*this, tj);
    std::vector<IdxVec> sk;
    std::vector<Blk<T>> Vs;
    row_ids(tblocks, P.tol, P.max_rank, sk, Vs);
    size_t t = 0;
    for (size_t q = 0; q < probs.size(); ++q) {
      DBF<T>& bf = *probs[q].out;
      for (size_t p = 0; p < loc[q].size(); ++p, ++t) {
        bf.V[l][p] = Vs[t];
        IdxVec o;
        for (int32_t y : sk[t]) o.push_back(loc[q][p].second[y]);
        bf.Ssk[l][p] = o;
      }
    }
    scratch.release(mk);
  }
  {                                                       // centre
    std::vector<std::pair<IdxVec, IdxVec>> all, loc;
    std::vector<Blk<T>> blocks;
    for (size_t q = 0; q < probs.size(); ++q) {
      DBF<T>& bf = *probs[q].out;
      loc.clear();
      for (int p = 0; p < (1 << L); ++p) loc.push_back({bf.Osk[lc][p], bf.Ssk[lc][p]});
      shifted(loc, probs[q], all);
      for (int p = 0; p < (1 << L); ++p) {
        bf.B[p] = new_blk<T>(persist, (int)bf.Osk[lc][p].size(), (int)bf.Ssk[lc][p].size());
        blocks.push_back(bf.B[p]);
      }
    }
    {
      HostTimer te_(t_host + H_EXT);
      ext(all, blocks);
    }
  }
  sync();
  scratch.release(mk);
}

template <typename T>
std::unique_ptr<DBF<T>> BFContext<T>::entry_eval(const DExtract<T>& ext, int m, int n, const Tree& rt, const Tree& ct,
                                                  int L, const std::vector<IdxVec>& nn_r,
                                                  const std::vector<IdxVec>& nn_c, const BFParams& P) {
  std::vector<BFProblem<T>> pr(1);
  pr[0].m = m; pr[0].n = n; pr[0].L = L; pr[0].rt = rt; pr[0].ct = ct; pr[0].nn_r = nn_r; pr[0].nn_c = nn_c;
  entry_eval_batch(ext, pr, P);
  return std::move(pr[0].out);
}

// ---------------------------------------------------------------------------
// construction from products (Sec. 3.2; reading: ID-based sketching variant of Alg. 2)
// ---------------------------------------------------------------------------
template <typename T>
std::unique_ptr<DBF<T>> BFContext<T>::random_matvec(const DOp<T>& op, const Tree& rt, const Tree& ct, int L,
                                                     const BFParams& P, uint32_t key) {
  std::vector<RMProblem<T>> pr(1);
  pr[0].m = op.rows;
  pr[0].n = op.cols;
  pr[0].rt = rt;
  pr[0].ct = ct;
  pr[0].key = key;
  DOpB<T> opb = [&op](const std::vector<Blk<T>>& X, std::vector<Blk<T>>& Y, bool tr) { op.apply(X[0], Y[0], tr); };
  random_matvec_batch(opb, pr, L, P);
  return std::move(pr[0].out);
}

// ---------------------------------------------------------------------------
// extraction of a list of sub-blocks (Alg. 3, loops reordered so each block
// of the butterfly is multiplied at most once per list item and level)
// dst[q] += sign * K(X_q, Y_q)
// ---------------------------------------------------------------------------
template <typename T>
struct ExtractPlan {
  std::vector<PlaceJob<T>> pj;
  std::map<int, std::vector<GemmDesc<T>>> Estage, Fstage;
  std::vector<Blk2Job<T>> gather0;
  std::vector<GemmDesc<T>> centre1, centre2;
};

template <typename T>
static void extract_collect(BFContext<T>& cx, const DBF<T>& bf, const std::vector<std::pair<IdxVec, IdxVec>>& lst,
                            std::vector<Blk<T>>& dst, T sign, ExtractPlan<T>& EP) {
  typename BFContext<T>::HostTimer ht_(cx.t_host + BFContext<T>::H_EXTRACT);
  const int L = bf.L, lc = bf.lc;
  struct Part {
    int p0, p1;   // positions [p0, p1) in the sorted list
  };
  auto& pj = EP.pj;
  auto& Estage = EP.Estage;
  auto& Fstage = EP.Fstage;
  auto& gather0 = EP.gather0;
  auto& centre1 = EP.centre1;
  auto& centre2 = EP.centre2;
  auto& scratch = cx.scratch;
  // E^l / F^l blocks of one list item, flat [l][p] (p < 2^L), reset after each item
  std::vector<Blk<T>> Ebuf(((size_t)L + 1) << L), Fbuf(((size_t)L + 1) << L);
  std::vector<size_t> touched;
  std::vector<int> xo, yo;
  IdxVec X, Y;
  for (size_t q = 0; q < lst.size(); ++q) {
    const IdxVec& X0 = lst[q].first;
    const IdxVec& Y0 = lst[q].second;
    if (X0.empty() || Y0.empty()) continue;
    // sorted copies and their original positions (lists that arrive sorted skip the sort)
    auto sort_pos = [](const IdxVec& v, std::vector<int>& o, IdxVec& sorted) {
      o.resize(v.size());
      std::iota(o.begin(), o.end(), 0);
      if (!std::is_sorted(v.begin(), v.end()))
        std::stable_sort(o.begin(), o.end(), [&](int a, int b) { return v[a] < v[b]; });
      sorted.resize(v.size());
      for (size_t t = 0; t < o.size(); ++t) sorted[t] = v[o[t]];
    };
    sort_pos(X0, xo, X);
    sort_pos(Y0, yo, Y);
    auto parts = [&](const Tree& tr, int l, const IdxVec& v) {
      std::vector<Part> out(tr[l].size());
      for (size_t k = 0; k < tr[l].size(); ++k) {
        out[k].p0 = (int)(std::lower_bound(v.begin(), v.end(), (int32_t)tr[l][k].a) - v.begin());
        out[k].p1 = (int)(std::lower_bound(v.begin(), v.end(), (int32_t)tr[l][k].b) - v.begin());
      }
      return out;
    };
    std::vector<std::vector<Part>> Xp(L + 1), Yp(L + 1);
    for (int l = 0; l <= L; ++l) { Xp[l] = parts(bf.rt, l, X); Yp[l] = parts(bf.ct, l, Y); }
    auto nonempty = [](const Part& p) { return p.p1 > p.p0; };
    // E^l blocks, l = L .. lc : rows = positions of X in O_i, cols = r(l,i,j)
    for (size_t t : touched) Ebuf[t] = Fbuf[t] = Blk<T>();   // p == nullptr: absent
    touched.clear();
    auto E = [&](int l, int p) -> Blk<T>& { return Ebuf[((size_t)l << L) + p]; };
    auto F = [&](int l, int p) -> Blk<T>& { return Fbuf[((size_t)l << L) + p]; };
    auto touch = [&](int l, int p) { touched.push_back(((size_t)l << L) + p); };
    const IdxVec* Xptr = &X;
    for (int i = 0; i < (1 << L); ++i) {
      if (!nonempty(Xp[L][i]) || !nonempty(Yp[0][0])) continue;
      const int r = bf.rr(L, i, 0);
      const int nr = Xp[L][i].p1 - Xp[L][i].p0;
      Blk<T> e = new_blk<T>(scratch, nr, std::max(r, 1));
      e.cols = r;
      E(L, i) = e;
      touch(L, i);
      if (r == 0) continue;
      IdxVec rows;
      for (int t = Xp[L][i].p0; t < Xp[L][i].p1; ++t) rows.push_back((*Xptr)[t] - (int32_t)bf.rt[L][i].a);
      Blk2Job<T> j{};
      j.src = bf.U[L][i].p; j.splane = bf.U[L][i].plane; j.sld = bf.U[L][i].ld;
      j.dst = e.p; j.dplane = e.plane; j.dld = e.ld; j.rows = nr; j.cols = r; j.alpha = T(1);
      j.ridx = dev_idx(cx, rows);
      j.cidx = nullptr;
      j.mode = 4;
      gather0.push_back(j);
    }
    for (int l = L - 1; l >= lc; --l)
      for (int i = 0; i < (1 << l); ++i)
        for (int jj = 0; jj < (1 << (L - l)); ++jj) {
          if (!nonempty(Xp[l][i]) || !nonempty(Yp[L - l][jj])) continue;
          const int p = bf.pidx(l, i, jj);
          const int r = bf.rr(l, i, jj);
          const int nr = Xp[l][i].p1 - Xp[l][i].p0;
          Blk<T> e = new_blk<T>(scratch, nr, std::max(r, 1));
          e.cols = r;
          E(l, p) = e;
          touch(l, p);
          const int r1 = bf.rr(l + 1, 2 * i, jj / 2);
          int roff = 0;
          for (int t = 0; t < 2; ++t) {
            const int ci = 2 * i + t;
            if (!nonempty(Xp[l + 1][ci])) continue;
            const int cp = bf.pidx(l + 1, ci, jj / 2);
            const Blk<T>& ec = E(l + 1, cp);
            const int nrc = Xp[l + 1][ci].p1 - Xp[l + 1][ci].p0;
            const int rc = bf.rr(l + 1, ci, jj / 2);
            const Blk<T>& R = bf.U[l][p];
            const int off = Xp[l + 1][ci].p0 - Xp[l][i].p0;
            if (!ec.p) continue;
            Estage[L - 1 - l].push_back(gdesc<T>(nrc, r, rc, 0, 0, T(1), T(0), ec,
                                         R.sub(t == 0 ? 0 : r1, 0, rc, R.cols), e.sub(off, 0, nrc, r)));
            (void)roff;
          }
        }
    // F^l blocks stored transposed: rows = positions of Y in S_j, cols = c(l,i,j)
    for (int jj = 0; jj < (1 << L); ++jj) {
      if (!nonempty(Yp[L][jj]) || !nonempty(Xp[0][0])) continue;
      const int c = bf.rc(0, 0, jj);
      const int nr = Yp[L][jj].p1 - Yp[L][jj].p0;
      Blk<T> f = new_blk<T>(scratch, nr, std::max(c, 1));
      f.cols = c;
      F(0, jj) = f;
      touch(0, jj);
      if (c == 0) continue;
      IdxVec rows;
      for (int t = Yp[L][jj].p0; t < Yp[L][jj].p1; ++t) rows.push_back(Y[t] - (int32_t)bf.ct[L][jj].a);
      Blk2Job<T> j{};
      j.src = bf.V[0][jj].p; j.splane = bf.V[0][jj].plane; j.sld = bf.V[0][jj].ld;
      j.dst = f.p; j.dplane = f.plane; j.dld = f.ld; j.rows = nr; j.cols = c; j.alpha = T(1);
      j.ridx = dev_idx(cx, rows);
      j.cidx = nullptr;
      j.mode = 4;
      gather0.push_back(j);
    }
    for (int l = 1; l <= lc; ++l)
      for (int i = 0; i < (1 << l); ++i)
        for (int jj = 0; jj < (1 << (L - l)); ++jj) {
          if (!nonempty(Xp[l][i]) || !nonempty(Yp[L - l][jj])) continue;
          const int p = bf.pidx(l, i, jj);
          const int c = bf.rc(l, i, jj);
          const int nr = Yp[L - l][jj].p1 - Yp[L - l][jj].p0;
          Blk<T> f = new_blk<T>(scratch, nr, std::max(c, 1));
          f.cols = c;
          F(l, p) = f;
          touch(l, p);
          const int c1 = bf.rc(l - 1, i / 2, 2 * jj);
          for (int t = 0; t < 2; ++t) {
            const int cj = 2 * jj + t;
            if (!nonempty(Yp[L - l + 1][cj])) continue;
            const int cp = bf.pidx(l - 1, i / 2, cj);
            const Blk<T>& fc = F(l - 1, cp);
            if (!fc.p) continue;
            const int nrc = Yp[L - l + 1][cj].p1 - Yp[L - l + 1][cj].p0;
            const int cc = bf.rc(l - 1, i / 2, cj);
            const Blk<T>& W = bf.V[l][p];
            const int off = Yp[L - l + 1][cj].p0 - Yp[L - l][jj].p0;
            Fstage[l - 1].push_back(gdesc<T>(nrc, c, cc, 0, 0, T(1), T(0), fc,
                                         W.sub(t == 0 ? 0 : c1, 0, cc, W.cols), f.sub(off, 0, nrc, c)));
          }
        }
    // centre: out(X in O_i, Y in S_j) = E B F = (E B) Ft^T
    for (int i = 0; i < (1 << lc); ++i)
      for (int jj = 0; jj < (1 << (L - lc)); ++jj) {
        if (!nonempty(Xp[lc][i]) || !nonempty(Yp[L - lc][jj])) continue;
        const int p = bf.pidx(lc, i, jj);
        const Blk<T>& ie = E(lc, p);
        const Blk<T>& iff = F(lc, p);
        if (!ie.p || !iff.p) continue;
        const int r = bf.rr(lc, i, jj), c = bf.rc(lc, i, jj);
        const int nx = Xp[lc][i].p1 - Xp[lc][i].p0, ny = Yp[L - lc][jj].p1 - Yp[L - lc][jj].p0;
        Blk<T> tmp = new_blk<T>(scratch, nx, std::max(c, 1));
        Blk<T> out = new_blk<T>(scratch, nx, ny);
        if (r == 0 || c == 0) continue;
        centre1.push_back(gdesc<T>(nx, c, r, 0, 0, T(1), T(0), ie, bf.B[p], tmp));
        centre2.push_back(gdesc<T>(nx, ny, c, 0, 1, T(1), T(0), tmp, iff, out));
        IdxVec rows, cols;
        for (int t = Xp[lc][i].p0; t < Xp[lc][i].p1; ++t) rows.push_back(xo[t]);
        for (int t = Yp[L - lc][jj].p0; t < Yp[L - lc][jj].p1; ++t) cols.push_back(yo[t]);
        PlaceJob<T> pl{};
        pl.src = out.p; pl.splane = out.plane; pl.sld = out.ld;
        pl.rows = dev_idx(cx, rows);
        pl.cols = dev_idx(cx, cols);
        pl.nr = nx; pl.nc = ny;
        pl.dst = dst[q].p; pl.dplane = dst[q].plane; pl.dld = dst[q].ld;
        pl.sign = sign;
        pj.push_back(pl);
      }
  }
}

template <typename T>
static void extract_run(BFContext<T>& cx, ExtractPlan<T>& EP) {
  run_blk2(cx, EP.gather0);
  for (auto& kv : EP.Estage) cx.gemm(kv.second);
  for (auto& kv : EP.Fstage) cx.gemm(kv.second);
  cx.gemm(EP.centre1);
  cx.gemm(EP.centre2);
  if (!EP.pj.empty()) {
    int64_t mx = 0;
    for (auto& p : EP.pj) mx = std::max<int64_t>(mx, (int64_t)p.nr * p.nc);
    const PlaceJob<T>* d = cx.stage(EP.pj.data(), EP.pj.size());
    launch_place<T>(d, (int)EP.pj.size(), mx, cx.st);
  }
}

template <typename T>
void BFContext<T>::extract_bf(const DBF<T>& bf, const std::vector<std::pair<IdxVec, IdxVec>>& lst,
                              std::vector<Blk<T>>& dst, T sign) {
  ExtractPlan<T> EP;
  extract_collect(*this, bf, lst, dst, sign, EP);
  extract_run(*this, EP);
}

template <typename T>
void BFContext<T>::extract_multi(const std::vector<const DBF<T>*>& bfs,
                                 const std::vector<const std::vector<std::pair<IdxVec, IdxVec>>*>& lsts,
                                 const std::vector<std::vector<Blk<T>>*>& dsts) {
  ExtractPlan<T> EP;
  for (size_t q = 0; q < bfs.size(); ++q) extract_collect(*this, *bfs[q], *lsts[q], *dsts[q], T(1), EP);
  extract_run(*this, EP);
}

// ---------------------------------------------------------------------------
// split of an L-level butterfly into the (L-2)-level child on quadrant (a, b) (Alg. 4, BF_SMW)
// ---------------------------------------------------------------------------
template <typename T>
std::unique_ptr<DBF<T>> BFContext<T>::split_child(const DBF<T>& bf, int a, int b) {
  const int L = bf.L, Lp = L - 2;
  const int64_t ra0 = bf.rt[1][a].a, cb0 = bf.ct[1][b].a;
  Tree rt = subtree(bf.rt, 1, a, Lp), ct = subtree(bf.ct, 1, b, Lp);
  auto ch = std::make_unique<DBF<T>>();
  ch->init((int)(rt[0][0].b), (int)(ct[0][0].b), rt, ct, Lp);
  std::vector<GemmDesc<T>> g;
  for (int lp = ch->lc; lp <= Lp; ++lp) {
    const int l = lp + 1;
    for (int ip = 0; ip < (1 << lp); ++ip)
      for (int jp = 0; jp < (1 << (Lp - lp)); ++jp) {
        const int i = a * (1 << lp) + ip, j = b * (1 << (Lp - lp)) + jp;
        const int p = bf.pidx(l, i, j), pp = ch->pidx(lp, ip, jp);
        const Blk<T>& R = bf.U[l][p];
        if (l == L - 1) {
          const int r1 = bf.rr(L, 2 * i, 0), r2 = bf.rr(L, 2 * i + 1, 0);
          const Blk<T>& U1 = bf.U[L][2 * i];
          const Blk<T>& U2 = bf.U[L][2 * i + 1];
          Blk<T> out = new_blk<T>(persist, U1.rows + U2.rows, std::max(R.cols, 1));
          out.cols = R.cols;
          if (R.cols > 0) {
            g.push_back(gdesc<T>(U1.rows, R.cols, r1, 0, 0, T(1), T(0), U1, R.sub(0, 0, r1, R.cols),
                                 out.sub(0, 0, U1.rows, R.cols)));
            g.push_back(gdesc<T>(U2.rows, R.cols, r2, 0, 0, T(1), T(0), U2, R.sub(r1, 0, r2, R.cols),
                                 out.sub(U1.rows, 0, U2.rows, R.cols)));
          }
          ch->U[lp][pp] = out;
        } else {
          ch->U[lp][pp] = R;
        }
        IdxVec o;
        for (int32_t x : bf.Osk[l][p]) o.push_back(x - (int32_t)ra0);
        ch->Osk[lp][pp] = o;
      }
  }
  for (int lp = 0; lp <= ch->lc; ++lp) {
    const int l = lp + 1;
    for (int ip = 0; ip < (1 << lp); ++ip)
      for (int jp = 0; jp < (1 << (Lp - lp)); ++jp) {
        const int i = a * (1 << lp) + ip, j = b * (1 << (Lp - lp)) + jp;
        const int p = bf.pidx(l, i, j), pp = ch->pidx(lp, ip, jp);
        const Blk<T>& W = bf.V[l][p];
        if (l == 1) {
          const int c1 = bf.rc(0, 0, 2 * j), c2 = bf.rc(0, 0, 2 * j + 1);
          const Blk<T>& V1 = bf.V[0][2 * j];
          const Blk<T>& V2 = bf.V[0][2 * j + 1];
          Blk<T> out = new_blk<T>(persist, V1.rows + V2.rows, std::max(W.cols, 1));
          out.cols = W.cols;
          if (W.cols > 0) {
            g.push_back(gdesc<T>(V1.rows, W.cols, c1, 0, 0, T(1), T(0), V1, W.sub(0, 0, c1, W.cols),
                                 out.sub(0, 0, V1.rows, W.cols)));
            g.push_back(gdesc<T>(V2.rows, W.cols, c2, 0, 0, T(1), T(0), V2, W.sub(c1, 0, c2, W.cols),
                                 out.sub(V1.rows, 0, V2.rows, W.cols)));
          }
          ch->V[lp][pp] = out;
        } else {
          ch->V[lp][pp] = W;
        }
        IdxVec o;
        for (int32_t x : bf.Ssk[l][p]) o.push_back(x - (int32_t)cb0);
        ch->Ssk[lp][pp] = o;
      }
  }
  for (int ip = 0; ip < (1 << ch->lc); ++ip)
    for (int jp = 0; jp < (1 << (Lp - ch->lc)); ++jp) {
      const int i = a * (1 << ch->lc) + ip, j = b * (1 << (Lp - ch->lc)) + jp;
      ch->B[ch->pidx(ch->lc, ip, jp)] = bf.B[bf.pidx(bf.lc, i, j)];
    }
  gemm(g);
  return ch;
}

// ---------------------------------------------------------------------------
// HOD-BF (Sec. 4)
// ---------------------------------------------------------------------------
template <typename T>
void BFContext<T>::hodbf_entry_eval_batch(const DExtract<T>& ext, std::vector<HProblem<T>>& probs, const BFParams& P) {
  // leaves of every problem in one extraction call
  {
    std::vector<std::pair<IdxVec, IdxVec>> lst;
    std::vector<Blk<T>> blocks;
    for (auto& hp : probs) {
      hp.out = std::make_unique<DHODBF<T>>();
      DHODBF<T>& H = *hp.out;
      H.n = hp.n;
      H.tree = hp.tree;
      H.LH = (int)hp.tree.size() - 1;
      for (auto& r : hp.tree[H.LH]) {
        IdxVec v = range_vec(r.a + hp.off, r.b + hp.off);
        lst.push_back({v, v});
        H.D.push_back(new_blk<T>(persist, (int)(r.b - r.a), (int)(r.b - r.a)));
        blocks.push_back(H.D.back());
      }
      H.off.clear();
      H.off.resize(H.LH + 1);
    }
    ext(lst, blocks);
  }
  // off-diagonal butterflies grouped by level count
  std::map<int, std::vector<BFProblem<T>>> groups;
  std::map<int, std::vector<std::pair<size_t, std::pair<int, int>>>> where;
  for (size_t q = 0; q < probs.size(); ++q) {
    const HProblem<T>& hp = probs[q];
    const Tree& tree = hp.tree;
    const int LH = (int)tree.size() - 1;
    for (int l = 1; l <= LH; ++l) {
      probs[q].out->off[l].resize((size_t)1 << l);
      for (int i = 0; i < (1 << l); ++i) {
        const Range rr = tree[l][i], cr = tree[l][i ^ 1];
        const int a = (int)rr.a, c = (int)cr.a, nr = (int)(rr.b - rr.a), nc = (int)(cr.b - cr.a);
        BFProblem<T> bp;
        bp.m = nr; bp.n = nc; bp.L = LH - l;
        bp.rt = subtree(tree, l, i, bp.L);
        bp.ct = subtree(tree, l, i ^ 1, bp.L);
        bp.row_off = hp.off + a;
        bp.col_off = hp.off + c;
        bp.nn_r.resize(nr);
        bp.nn_c.resize(nc);
        const std::vector<IdxVec>& nn = *hp.nn;
        for (int x = 0; x < nr; ++x)
          if (a + x < (int)nn.size())
            for (int32_t v : nn[a + x])
              if (v >= c && v < c + nc) bp.nn_r[x].push_back(v - c);
        for (int y = 0; y < nc; ++y)
          if (c + y < (int)nn.size())
            for (int32_t v : nn[c + y])
              if (v >= a && v < a + nr) bp.nn_c[y].push_back(v - a);
        where[bp.L].push_back({q, {l, i}});
        groups[bp.L].push_back(std::move(bp));
      }
    }
  }
  for (auto& kv : groups) {
    entry_eval_batch(ext, kv.second, P);
    auto& wh = where[kv.first];
    for (size_t t = 0; t < kv.second.size(); ++t)
      probs[wh[t].first].out->off[wh[t].second.first][wh[t].second.second] = std::move(kv.second[t].out);
  }
}

template <typename T>
std::unique_ptr<DHODBF<T>> BFContext<T>::hodbf_entry_eval(const DExtract<T>& ext, int n, const Tree& tree,
                                                           const std::vector<IdxVec>& nn, const BFParams& P) {
  std::vector<HProblem<T>> hp(1);
  hp[0].n = n; hp[0].tree = tree; hp[0].nn = &nn; hp[0].off = 0;
  hodbf_entry_eval_batch(ext, hp, P);
  return std::move(hp[0].out);
}

template <typename T>
void BFContext<T>::hodbf_apply(const DHODBF<T>& H, const Blk<T>& X, Blk<T>& Y, bool transpose) {
  const int LH = H.LH, k = X.cols;
  std::vector<GemmDesc<T>> g;
  for (size_t q = 0; q < H.D.size(); ++q) {
    const Range r = H.tree[LH][q];
    const int nr = (int)(r.b - r.a);
    g.push_back(gdesc<T>(nr, k, nr, transpose ? 1 : 0, 0, T(1), T(0), H.D[q], X.sub((int)r.a, 0, nr, k),
                         Y.sub((int)r.a, 0, nr, k)));
  }
  gemm(g);
  for (int l = 1; l <= LH; ++l) {
    std::vector<const DBF<T>*> bfs;
    std::vector<Blk<T>> xs, ys;
    for (int i = 0; i < (1 << l); ++i) {
      const Range rr = H.tree[l][i], cr = H.tree[l][i ^ 1];
      bfs.push_back(H.off[l][i].get());
      if (!transpose) {
        xs.push_back(X.sub((int)cr.a, 0, (int)(cr.b - cr.a), k));
        ys.push_back(Y.sub((int)rr.a, 0, (int)(rr.b - rr.a), k));
      } else {
        xs.push_back(X.sub((int)rr.a, 0, (int)(rr.b - rr.a), k));
        ys.push_back(Y.sub((int)cr.a, 0, (int)(cr.b - cr.a), k));
      }
    }
    apply(bfs, xs, ys, transpose, true);
  }
}

template <typename T>
void BFContext<T>::hodbf_extract(const DHODBF<T>& H, const std::vector<std::pair<IdxVec, IdxVec>>& lst,
                                 std::vector<Blk<T>>& dst, T sign) {
  HostTimer ht_(t_host + H_HEXTRACT);
  const int LH = H.LH;
  std::vector<Blk2Job<T>> gj;
  std::vector<PlaceJob<T>> pj;
  struct Req {
    const DBF<T>* bf;
    std::vector<std::pair<IdxVec, IdxVec>> lst;
    std::vector<Blk<T>> tmp;
    std::vector<IdxVec> px, py;
    int q;
  };
  std::vector<Req> reqs;
  std::map<const DBF<T>*, size_t> req_of;
  std::vector<std::pair<char*, size_t>> zspans;   // accumulation targets, zeroed in as few memsets as possible
  // each list item's indices sorted once (value, position): the part inside a tree range is a slice
  std::vector<std::pair<int32_t, int32_t>> xs, ys;
  auto sorted_of = [](const IdxVec& v, std::vector<std::pair<int32_t, int32_t>>& out) {
    out.resize(v.size());
    for (size_t a = 0; a < v.size(); ++a) out[a] = {v[a], (int32_t)a};
    std::sort(out.begin(), out.end());
  };
  auto slice = [](const std::vector<std::pair<int32_t, int32_t>>& v, Range r, IdxVec& pos, IdxVec& loc) {
    pos.clear();
    loc.clear();
    auto lo = std::lower_bound(v.begin(), v.end(), std::make_pair((int32_t)r.a, INT32_MIN));
    auto hi = std::lower_bound(lo, v.end(), std::make_pair((int32_t)r.b, INT32_MIN));
    for (auto it = lo; it != hi; ++it) {
      pos.push_back(it->second);
      loc.push_back(it->first - (int32_t)r.a);
    }
    return lo != hi;
  };
  for (size_t q = 0; q < lst.size(); ++q) {
    const IdxVec& X = lst[q].first;
    const IdxVec& Y = lst[q].second;
    if (X.empty() || Y.empty()) continue;
    sorted_of(X, xs);
    sorted_of(Y, ys);
    // leaves
    for (size_t li = 0; li < H.tree[LH].size(); ++li) {
      const Range r = H.tree[LH][li];
      IdxVec px, py, rx, ry;
      if (!slice(xs, r, px, rx) || !slice(ys, r, py, ry)) continue;
      Blk<T> t = new_blk<T>(scratch, (int)px.size(), (int)py.size());
      Blk2Job<T> j{};
      j.src = H.D[li].p; j.splane = H.D[li].plane; j.sld = H.D[li].ld;
      j.dst = t.p; j.dplane = t.plane; j.dld = t.ld; j.rows = t.rows; j.cols = t.cols; j.alpha = T(1);
      j.ridx = dev_idx(*this, rx); j.cidx = dev_idx(*this, ry); j.mode = 4;
      gj.push_back(j);
      PlaceJob<T> pl{};
      pl.src = t.p; pl.splane = t.plane; pl.sld = t.ld;
      pl.rows = dev_idx(*this, px); pl.cols = dev_idx(*this, py); pl.nr = t.rows; pl.nc = t.cols;
      pl.dst = dst[q].p; pl.dplane = dst[q].plane; pl.dld = dst[q].ld; pl.sign = sign;
      pj.push_back(pl);
    }
    // off-diagonal butterflies
    for (int l = 1; l <= LH; ++l)
      for (int i = 0; i < (1 << l); ++i) {
        const Range rr = H.tree[l][i], cr = H.tree[l][i ^ 1];
        IdxVec px, py, rx, ry;
        if (!slice(xs, rr, px, rx) || !slice(ys, cr, py, ry)) continue;
        const DBF<T>* bf = H.off[l][i].get();
        auto it = req_of.find(bf);
        if (it == req_of.end()) {
          req_of[bf] = reqs.size();
          reqs.push_back(Req{bf, {}, {}, {}, {}, 0});
          it = req_of.find(bf);
        }
        Req& R = reqs[it->second];
        Blk<T> t = new_blk<T>(scratch, (int)rx.size(), (int)ry.size());
        R.lst.emplace_back(std::move(rx), std::move(ry));   // rx, ry are not used below
        zspans.push_back({reinterpret_cast<char*>(t.p), (size_t)2 * t.plane * sizeof(T)});
        R.tmp.push_back(t);
        PlaceJob<T> pl{};
        pl.src = t.p; pl.splane = t.plane; pl.sld = t.ld;
        pl.rows = dev_idx(*this, px); pl.cols = dev_idx(*this, py); pl.nr = t.rows; pl.nc = t.cols;
        pl.dst = dst[q].p; pl.dplane = dst[q].plane; pl.dld = dst[q].ld; pl.sign = sign;
        pj.push_back(pl);
      }
  }
  for (size_t a = 0; a < zspans.size();) {   // merge adjacent spans (consecutive scratch allocations)
    char* p0 = zspans[a].first;
    char* p1 = p0 + zspans[a].second;
    size_t b = a + 1;
    while (b < zspans.size() && zspans[b].first >= p1 && zspans[b].first - p1 < 256) {
      p1 = zspans[b].first + zspans[b].second;
      ++b;
    }
    MF_CUDA(cudaMemsetAsync(p0, 0, (size_t)(p1 - p0), st));
    a = b;
  }
  run_blk2(*this, gj);
  std::vector<const DBF<T>*> bfs;
  std::vector<const std::vector<std::pair<IdxVec, IdxVec>>*> ls;
  std::vector<std::vector<Blk<T>>*> ds;
  for (auto& R : reqs) {
    bfs.push_back(R.bf);
    ls.push_back(&R.lst);
    ds.push_back(&R.tmp);
  }
  extract_multi(bfs, ls, ds);
  if (!pj.empty()) {
    int64_t mx = 0;
    for (auto& p : pj) mx = std::max<int64_t>(mx, (int64_t)p.nr * p.nc);
    const PlaceJob<T>* d = stage(pj.data(), pj.size());
    launch_place<T>(d, (int)pj.size(), mx, st);
  }
}

// ---------------------------------------------------------------------------
// HOD-BF inversion (Alg. 4) and BF_SMW
// ---------------------------------------------------------------------------
template <typename T>
void BFContext<T>::inv_apply(const DHODBFInv<T>& Hi, const Blk<T>& X, Blk<T>& Y, bool transpose, int l0, int i0) {
  const int LH = Hi.LH, k = X.cols;
  const int64_t a0 = Hi.tree[l0][i0].a;
  const int nsub = 1 << (LH - l0);
  auto leaves = [&](const Blk<T>& src, Blk<T>& out) {
    std::vector<GemmDesc<T>> g;
    for (int li = i0 * nsub; li < (i0 + 1) * nsub; ++li) {
      const Range r = Hi.tree[LH][li];
      const int nr = (int)(r.b - r.a);
      if (nr == 0) continue;
      g.push_back(gdesc<T>(nr, k, nr, transpose ? 1 : 0, 0, T(1), T(0), Hi.Dinv[li], src.sub((int)(r.a - a0), 0, nr, k),
                           out.sub((int)(r.a - a0), 0, nr, k)));
    }
    gemm(g);
  };
  const size_t mk = scratch.mark();
  Blk<T> Z = new_blk<T>(scratch, X.rows, k);
  auto level = [&](int l) {
    const int span = 1 << (l - l0);
    std::vector<const DBF<T>*> bfs;
    std::vector<Blk<T>> xs, zs;
    for (int i = i0 * span; i < (i0 + 1) * span; ++i) {
      const Range r = Hi.tree[l][i];
      bfs.push_back(Hi.M[l][i].get());
      xs.push_back(Y.sub((int)(r.a - a0), 0, (int)(r.b - r.a), k));
      zs.push_back(Z.sub((int)(r.a - a0), 0, (int)(r.b - r.a), k));
    }
    apply(bfs, xs, zs, transpose, false);
    std::vector<Blk2Job<T>> aj;
    Blk2Job<T> j{};
    j.src = Z.p; j.splane = Z.plane; j.sld = Z.ld;
    j.dst = Y.p; j.dplane = Y.plane; j.dld = Y.ld; j.rows = X.rows; j.cols = k; j.alpha = T(1); j.mode = 2;
    aj.push_back(j);
    run_blk2(*this, aj);
  };
  if (!transpose) {
    leaves(X, Y);
    for (int l = LH - 1; l >= l0; --l) level(l);
  } else {
    // Y = X first, then the level factors in reverse order, then the leaves
    std::vector<Blk2Job<T>> cj;
    Blk2Job<T> j{};
    j.src = X.p; j.splane = X.plane; j.sld = X.ld;
    j.dst = Y.p; j.dplane = Y.plane; j.dld = Y.ld; j.rows = X.rows; j.cols = k; j.alpha = T(1); j.mode = 3;
    cj.push_back(j);
    run_blk2(*this, cj);
    for (int l = l0; l <= LH - 1; ++l) level(l);
    leaves(Y, Z);
    std::vector<Blk2Job<T>> bj;
    Blk2Job<T> b{};
    b.src = Z.p; b.splane = Z.plane; b.sld = Z.ld;
    b.dst = Y.p; b.dplane = Y.plane; b.dld = Y.ld; b.rows = X.rows; b.cols = k; b.alpha = T(1); b.mode = 3;
    bj.push_back(b);
    run_blk2(*this, bj);
  }
  (void)mk;   // Z stays reserved until the caller releases its scratch mark
}

template <typename T>
void BFContext<T>::inv_apply_multi(const std::vector<const DHODBFInv<T>*>& His, const std::vector<Blk<T>>& X,
                                   std::vector<Blk<T>>& Y, bool transpose) {
  // several full inverses in lockstep: one launch per step for all of them.  Without transpose
  // inverse q applies its level LH_q - 1 - d at step d (deepest first); with transpose the
  // levels run top-down and an inverse with fewer levels starts maxLH - LH_q steps later.
  const size_t nq = His.size();
  if (!nq) return;
  int maxLH = 0;
  for (auto* h : His) maxLH = std::max(maxLH, h->LH);
  std::vector<Blk<T>> Z(nq);
  for (size_t q = 0; q < nq; ++q) Z[q] = new_blk<T>(scratch, X[q].rows, X[q].cols);
  auto leaves = [&](const std::vector<Blk<T>>& src, std::vector<Blk<T>>& out) {
    std::vector<GemmDesc<T>> g;
    for (size_t q = 0; q < nq; ++q) {
      const DHODBFInv<T>& Hi = *His[q];
      const int k = X[q].cols;
      for (size_t li = 0; li < Hi.tree[Hi.LH].size(); ++li) {
        const Range r = Hi.tree[Hi.LH][li];
        const int nr = (int)(r.b - r.a);
        if (nr == 0) continue;
        g.push_back(gdesc<T>(nr, k, nr, transpose ? 1 : 0, 0, T(1), T(0), Hi.Dinv[li],
                             src[q].sub((int)r.a, 0, nr, k), out[q].sub((int)r.a, 0, nr, k)));
      }
    }
    gemm(g);
  };
  auto copies = [&](const std::vector<Blk<T>>& src, std::vector<Blk<T>>& dst) {
    std::vector<Blk2Job<T>> cj;
    for (size_t q = 0; q < nq; ++q) {
      Blk2Job<T> j{};
      j.src = src[q].p; j.splane = src[q].plane; j.sld = src[q].ld;
      j.dst = dst[q].p; j.dplane = dst[q].plane; j.dld = dst[q].ld;
      j.rows = src[q].rows; j.cols = src[q].cols; j.alpha = T(1); j.mode = 3;
      if (j.rows && j.cols) cj.push_back(j);
    }
    run_blk2(*this, cj);
  };
  auto step = [&](int d) {
    std::vector<const DBF<T>*> bfs;
    std::vector<Blk<T>> xs, zs, ys, zz;
    for (size_t q = 0; q < nq; ++q) {
      const DHODBFInv<T>& Hi = *His[q];
      const int l = transpose ? d - (maxLH - Hi.LH) : Hi.LH - 1 - d;
      if (l < 0 || l >= Hi.LH) continue;
      const int k = X[q].cols;
      for (int i = 0; i < (1 << l); ++i) {
        const Range r = Hi.tree[l][i];
        bfs.push_back(Hi.M[l][i].get());
        xs.push_back(Y[q].sub((int)r.a, 0, (int)(r.b - r.a), k));
        zs.push_back(Z[q].sub((int)r.a, 0, (int)(r.b - r.a), k));
      }
      ys.push_back(Y[q]);
      zz.push_back(Z[q]);
    }
    if (bfs.empty()) return;
    apply(bfs, xs, zs, transpose, false);
    axpy_b(zz, ys, T(1));
  };
  if (!transpose) {
    leaves(X, Y);
    for (int d = 0; d < maxLH; ++d) step(d);
  } else {
    copies(X, Y);
    for (int d = 0; d < maxLH; ++d) step(d);
    leaves(Y, Z);
    copies(Z, Y);
  }
}

template <typename T>
static void small_inverse(BFContext<T>& cx, const std::vector<Blk<T>>& A, std::vector<Blk<T>>& X) {
  std::vector<InvJob<T>> jobs;
  int mx = 1;
  for (size_t q = 0; q < A.size(); ++q) {
    if (A[q].rows == 0) continue;
    InvJob<T> j;
    j.A = A[q].p; j.aplane = A[q].plane; j.lda = A[q].ld; j.n = A[q].rows;
    j.X = X[q].p; j.xplane = X[q].plane; j.ldx = X[q].ld;
    j.W = nullptr;
    jobs.push_back(j);
    mx = std::max(mx, A[q].rows);
    cx.flops += 8.0 * A[q].rows * (double)A[q].rows * A[q].rows;
  }
  if (jobs.empty()) return;
  const bool in_smem = small_inverse_smem_bytes(mx, sizeof(double)) <= kSmallInvSmemCap;
  if (!in_smem)
    for (auto& j : jobs) j.W = cx.scratch.template takeT<double>(2 * (size_t)j.n * j.n);
  const InvJob<T>* d = cx.stage(jobs.data(), jobs.size());
  if (launch_small_inverse<T>(d, (int)jobs.size(), mx, in_smem, cx.status.template as<int32_t>(), cx.st) != 0)
    throw std::runtime_error("block too large for the small dense inverse (" + std::to_string(mx) + ")");
}

template <typename T>
std::unique_ptr<DBF<T>> BFContext<T>::bf_smw(const DBF<T>& K, const BFParams& P, uint32_t key) {
  const int L = K.L;
  if (L == 0) {
    // (I + U B V^T)^-1 = I - U B (I + V^T U B)^-1 V^T
    auto out = std::make_unique<DBF<T>>();
    out->init(K.m, K.n, K.rt, K.ct, 0);
    out->U = K.U; out->Osk = K.Osk; out->V = K.V; out->Ssk = K.Ssk;
    const Blk<T>& U = K.U[0][0];
    const Blk<T>& V = K.V[0][0];
    const Blk<T>& B = K.B[0];
    const int r = B.rows, c = B.cols;
    Blk<T> Bn = new_blk<T>(persist, r, std::max(c, 1));
    Bn.cols = c;
    out->B[0] = Bn;
    if (r == 0 || c == 0) return out;
    const size_t mk = scratch.mark();
    Blk<T> VU = new_blk<T>(scratch, c, r), G = new_blk<T>(scratch, c, c), Gi = new_blk<T>(scratch, c, c);
    std::vector<GemmDesc<T>> g{gdesc<T>(c, r, V.rows, 1, 0, T(1), T(0), V, U, VU)};
    gemm(g);
    // G = I + VU B : set G = I then G += VU B
    {
      std::vector<T> eye(2 * (size_t)G.plane, T(0));
      for (int a = 0; a < c; ++a) eye[(size_t)a * G.ld + a] = T(1);
      h2d(G.p, eye.data(), eye.size() * sizeof(T));
      sync();
    }
    g = {gdesc<T>(c, c, r, 0, 0, T(1), T(1), VU, B, G)};
    gemm(g);
    std::vector<Blk<T>> A1{G}, X1{Gi};
    small_inverse(*this, A1, X1);
    g = {gdesc<T>(r, c, c, 0, 0, T(-1), T(0), B, Gi, Bn)};
    gemm(g);
    sync();
    scratch.release(mk);
    return out;
  }
  if (L == 1) {
    // K = Ubar Mbar, Ubar = diag(U_0, U_1); R'_j = -(I + Mbar Ubar)^-1 R_j
    auto out = std::make_unique<DBF<T>>();
    out->init(K.m, K.n, K.rt, K.ct, 1);
    out->U = K.U; out->Osk = K.Osk; out->V = K.V; out->Ssk = K.Ssk; out->B = K.B;
    const int r0 = K.rr(1, 0, 0), r1 = K.rr(1, 1, 0), rs = r0 + r1;
    if (rs == 0) return out;
    const size_t mk = scratch.mark();
    Blk<T> G = new_blk<T>(scratch, rs, rs), Gi = new_blk<T>(scratch, rs, rs);
    {
      std::vector<T> eye(2 * (size_t)G.plane, T(0));
      for (int a = 0; a < rs; ++a) eye[(size_t)a * G.ld + a] = T(1);
      h2d(G.p, eye.data(), eye.size() * sizeof(T));
      sync();
    }
    for (int j = 0; j < 2; ++j) {
      // column block j of Mbar Ubar:  R_j B_j (V_j^T U_j)  into G[:, off_j : off_j + r_j]
      const Blk<T>& V = K.V[0][j];
      const Blk<T>& Uj = K.U[1][j];
      const Blk<T>& Bj = K.B[j];
      const Blk<T>& Rj = K.U[0][j];
      const int c = V.cols, rj = j == 0 ? r0 : r1, off = j == 0 ? 0 : r0;
      if (c == 0 || rj == 0 || Bj.rows == 0) continue;
      Blk<T> VU = new_blk<T>(scratch, c, rj), BVU = new_blk<T>(scratch, Bj.rows, rj);
      std::vector<GemmDesc<T>> g{gdesc<T>(c, rj, V.rows, 1, 0, T(1), T(0), V, Uj, VU)};
      gemm(g);
      g = {gdesc<T>(Bj.rows, rj, c, 0, 0, T(1), T(0), Bj, VU, BVU)};
      gemm(g);
      g = {gdesc<T>(rs, rj, Bj.rows, 0, 0, T(1), T(1), Rj, BVU, G.sub(0, off, rs, rj))};
      gemm(g);
    }
    std::vector<Blk<T>> A1{G}, X1{Gi};
    small_inverse(*this, A1, X1);
    for (int j = 0; j < 2; ++j) {
      const Blk<T>& Rj = K.U[0][j];
      Blk<T> Rn = new_blk<T>(persist, rs, std::max(Rj.cols, 1));
      Rn.cols = Rj.cols;
      if (Rj.cols > 0) {
        std::vector<GemmDesc<T>> g{gdesc<T>(rs, Rj.cols, rs, 0, 0, T(-1), T(0), Gi, Rj, Rn)};
        gemm(g);
      }
      out->U[0][j] = Rn;
    }
    sync();
    scratch.release(mk);
    return out;
  }
  auto K11 = split_child(K, 0, 0), K12 = split_child(K, 0, 1), K21 = split_child(K, 1, 0), K22 = split_child(K, 1, 1);
  auto K22i = bf_smw(*K22, P, key * 4u + 1u);
  return smw_assemble(K.m, K.rt, L, K11.get(), *K12, *K21, K22i.get(), P, key);
}

template <typename T>
std::unique_ptr<DBF<T>> BFContext<T>::smw_assemble(int n, const Tree& tr, int L, const DBF<T>* K11, const DBF<T>& K12,
                                                    const DBF<T>& K21, const DBF<T>* K22i, const BFParams& P,
                                                    uint32_t key) {
  const int n1 = (int)tr[1][0].b, n2 = n - n1;
  // z = (I + K22i) y, into a new scratch block (y unchanged)
  auto inv22 = [this, K22i](const Blk<T>& y, bool tr_) -> Blk<T> {
    Blk<T> z = new_blk<T>(scratch, y.rows, y.cols);
    std::vector<Blk2Job<T>> cj;
    Blk2Job<T> j{};
    j.src = y.p; j.splane = y.plane; j.sld = y.ld; j.dst = z.p; j.dplane = z.plane; j.dld = z.ld;
    j.rows = y.rows; j.cols = y.cols; j.alpha = T(1); j.mode = 3;
    cj.push_back(j);
    run_blk2(*this, cj);
    if (K22i) {
      std::vector<const DBF<T>*> b{K22i};
      std::vector<Blk<T>> xs{y}, ys{z};
      apply(b, xs, ys, tr_, true);
    }
    return z;
  };
  auto app = [this](const DBF<T>& K, const Blk<T>& x, Blk<T>& y, bool tr_, bool acc) {
    std::vector<const DBF<T>*> b{&K};
    std::vector<Blk<T>> xs{x}, ys{y};
    apply(b, xs, ys, tr_, acc);
  };
  auto axpy = [this](const Blk<T>& x, Blk<T>& y, T alpha) {
    std::vector<Blk2Job<T>> cj;
    Blk2Job<T> j{};
    j.src = x.p; j.splane = x.plane; j.sld = x.ld; j.dst = y.p; j.dplane = y.plane; j.dld = y.ld;
    j.rows = x.rows; j.cols = x.cols; j.alpha = alpha; j.mode = 2;
    cj.push_back(j);
    run_blk2(*this, cj);
  };
  // S = K11 - K12 (I + K22i) K21, an (L-2)-level butterfly on the first child's trees
  DOp<T> sop;
  sop.rows = n1;
  sop.cols = n1;
  sop.apply = [&, this](const Blk<T>& X, Blk<T>& Y, bool tr_) {
    const int k = X.cols;
    if (!tr_) {
      Blk<T> t = new_blk<T>(scratch, n2, k);
      app(K21, X, t, false, false);
      Blk<T> u = inv22(t, false);
      app(K12, u, Y, false, false);
      std::vector<Blk2Job<T>> neg;
      Blk2Job<T> j{};
      j.src = Y.p; j.splane = Y.plane; j.sld = Y.ld; j.dst = Y.p; j.dplane = Y.plane; j.dld = Y.ld;
      j.rows = Y.rows; j.cols = k; j.alpha = T(-2); j.mode = 2;   // Y <- Y - 2Y = -Y
      neg.push_back(j);
      run_blk2(*this, neg);
      if (K11) app(*K11, X, Y, false, true);
    } else {
      Blk<T> t = new_blk<T>(scratch, n2, k);
      app(K12, X, t, true, false);
      Blk<T> u = inv22(t, true);
      app(K21, u, Y, true, false);
      std::vector<Blk2Job<T>> neg;
      Blk2Job<T> j{};
      j.src = Y.p; j.splane = Y.plane; j.sld = Y.ld; j.dst = Y.p; j.dplane = Y.plane; j.dld = Y.ld;
      j.rows = Y.rows; j.cols = k; j.alpha = T(-2); j.mode = 2;
      neg.push_back(j);
      run_blk2(*this, neg);
      if (K11) app(*K11, X, Y, true, true);
    }
  };
  Tree rt1 = subtree(tr, 1, 0, L - 2);
  auto S = random_matvec(sop, rt1, rt1, L - 2, P, key * 4u + 2u);
  auto K11i = bf_smw(*S, P, key * 4u + 3u);
  const DBF<T>* K11ip = K11i.get();
  // A^-1 - I with A^-1 = [I 0; -A22^-1 A21 I] diag(A11^-1, A22^-1) [I -A12 A22^-1; 0 I]
  DOp<T> fop;
  fop.rows = n;
  fop.cols = n;
  fop.apply = [&, this](const Blk<T>& X, Blk<T>& Y, bool tr_) {
    const int k = X.cols;
    Blk<T> x1 = X.sub(0, 0, n1, k), x2 = X.sub(n1, 0, n2, k);
    Blk<T> y1 = Y.sub(0, 0, n1, k), y2 = Y.sub(n1, 0, n2, k);
    if (!tr_) {
      Blk<T> w = inv22(x2, false);                    // A22^-1 x2
      Blk<T> t1 = new_blk<T>(scratch, n1, k);
      app(K12, w, t1, false, false);                  // K12 A22^-1 x2
      std::vector<Blk2Job<T>> cj;                     // t1 = x1 - t1
      Blk2Job<T> j{};
      j.src = t1.p; j.splane = t1.plane; j.sld = t1.ld; j.dst = t1.p; j.dplane = t1.plane; j.dld = t1.ld;
      j.rows = n1; j.cols = k; j.alpha = T(-2); j.mode = 2;
      cj.push_back(j);
      run_blk2(*this, cj);
      axpy(x1, t1, T(1));
      // u1 = t1 + K11i t1 -> y1 ; y1 currently = u1
      std::vector<Blk2Job<T>> c2;
      Blk2Job<T> j2{};
      j2.src = t1.p; j2.splane = t1.plane; j2.sld = t1.ld; j2.dst = y1.p; j2.dplane = y1.plane; j2.dld = y1.ld;
      j2.rows = n1; j2.cols = k; j2.alpha = T(1); j2.mode = 3;
      c2.push_back(j2);
      run_blk2(*this, c2);
      app(*K11ip, t1, y1, false, true);
      // y2 = A22^-1 x2 - A22^-1 K21 u1
      Blk<T> v = new_blk<T>(scratch, n2, k);
      app(K21, y1, v, false, false);
      Blk<T> vv = inv22(v, false);
      std::vector<Blk2Job<T>> c3;
      Blk2Job<T> j3{};
      j3.src = w.p; j3.splane = w.plane; j3.sld = w.ld; j3.dst = y2.p; j3.dplane = y2.plane; j3.dld = y2.ld;
      j3.rows = n2; j3.cols = k; j3.alpha = T(1); j3.mode = 3;
      c3.push_back(j3);
      run_blk2(*this, c3);
      axpy(vv, y2, T(-1));
    } else {
      Blk<T> w = inv22(x2, true);                     // A22^-T x2
      Blk<T> t1 = new_blk<T>(scratch, n1, k);
      app(K21, w, t1, true, false);                   // K21^T A22^-T x2
      std::vector<Blk2Job<T>> cj;
      Blk2Job<T> j{};
      j.src = t1.p; j.splane = t1.plane; j.sld = t1.ld; j.dst = t1.p; j.dplane = t1.plane; j.dld = t1.ld;
      j.rows = n1; j.cols = k; j.alpha = T(-2); j.mode = 2;
      cj.push_back(j);
      run_blk2(*this, cj);
      axpy(x1, t1, T(1));                             // v1 = x1 - K21^T A22^-T x2
      std::vector<Blk2Job<T>> c2;
      Blk2Job<T> j2{};
      j2.src = t1.p; j2.splane = t1.plane; j2.sld = t1.ld; j2.dst = y1.p; j2.dplane = y1.plane; j2.dld = y1.ld;
      j2.rows = n1; j2.cols = k; j2.alpha = T(1); j2.mode = 3;
      c2.push_back(j2);
      run_blk2(*this, c2);
      app(*K11ip, t1, y1, true, true);                // w1 = A11^-T v1
      Blk<T> v = new_blk<T>(scratch, n2, k);
      app(K12, y1, v, true, false);                   // K12^T w1
      Blk<T> vv = inv22(v, true);
      std::vector<Blk2Job<T>> c3;
      Blk2Job<T> j3{};
      j3.src = w.p; j3.splane = w.plane; j3.sld = w.ld; j3.dst = y2.p; j3.dplane = y2.plane; j3.dld = y2.ld;
      j3.rows = n2; j3.cols = k; j3.alpha = T(1); j3.mode = 3;
      c3.push_back(j3);
      run_blk2(*this, c3);
      axpy(vv, y2, T(-1));
    }
    axpy(X, Y, T(-1));                                // minus the identity
  };
  return random_matvec(fop, tr, tr, L, P, key * 4u);
}

template <typename T>
std::unique_ptr<DHODBFInv<T>> BFContext<T>::hodbf_invert(const DHODBF<T>& H, const BFParams& P, uint32_t key) {
  auto inv = std::make_unique<DHODBFInv<T>>();
  inv->n = H.n;
  inv->tree = H.tree;
  inv->LH = H.LH;
  const int LH = H.LH;
  inv->Dinv.resize(H.D.size());
  for (size_t q = 0; q < H.D.size(); ++q) inv->Dinv[q] = new_blk<T>(persist, H.D[q].rows, H.D[q].rows);
  small_inverse(*this, H.D, inv->Dinv);
  inv->M.clear();
  inv->M.resize(LH + 1);
  DHODBFInv<T>* ip = inv.get();
  for (int l = LH - 1; l >= 0; --l) {
    const int nn = 1 << l, Lq = LH - l - 1;
    inv->M[l].resize((size_t)nn);
    // B_tau_i <- D_tau_i^-1 B_tau_i for both children of every node of level l, in lockstep
    std::vector<RMProblem<T>> probs(2 * (size_t)nn);
    std::vector<int> tt(2 * (size_t)nn);
    std::vector<const DBF<T>*> Boff(2 * (size_t)nn);
    for (int i = 0; i < nn; ++i)
      for (int side = 0; side < 2; ++side) {
        const size_t q = 2 * (size_t)i + side;
        const int t = 2 * i + side, ts = 2 * i + 1 - side;
        tt[q] = t;
        Boff[q] = H.off[l + 1][t].get();
        const Range ra = H.tree[l + 1][t], rb = H.tree[l + 1][ts];
        probs[q].m = (int)(ra.b - ra.a);
        probs[q].n = (int)(rb.b - rb.a);
        probs[q].rt = subtree(H.tree, l + 1, t, Lq);
        probs[q].ct = subtree(H.tree, l + 1, ts, Lq);
        probs[q].key = (key * 131u + (uint32_t)l * 17u + (uint32_t)t) & 0xFFFFFu;
      }
    DOpB<T> op = [&, ip, l](const std::vector<Blk<T>>& X, std::vector<Blk<T>>& Y, bool tr) {
      std::vector<Blk<T>> tmp(X.size());
      for (size_t q = 0; q < X.size(); ++q) tmp[q] = new_blk<T>(scratch, probs[q].m, X[q].cols);
      if (!tr) {
        apply(Boff, X, tmp, false, false);
        inv_apply_b(*ip, l + 1, tt, tmp, Y, false);
      } else {
        inv_apply_b(*ip, l + 1, tt, X, tmp, true);
        apply(Boff, tmp, Y, true, false);
      }
    };
    random_matvec_batch(op, probs, Lq, P);
    // BF_SMW([I B1; B2 I]) as an (Lq + 2)-level butterfly per node, all nodes of the level in lockstep
    std::vector<SmwItem<T>> items(nn);
    for (int i = 0; i < nn; ++i) {
      const Range r = H.tree[l][i];
      items[i].n = (int)(r.b - r.a);
      items[i].tr = extend_tree(subtree(H.tree, l, i, LH - l), Lq + 2);
      items[i].K12 = probs[2 * (size_t)i].out.get();
      items[i].K21 = probs[2 * (size_t)i + 1].out.get();
      items[i].key = (key * 977u + (uint32_t)l * 31u + (uint32_t)i) & 0xFFFFFu;
    }
    smw_assemble_batch(items, Lq + 2, P);
    for (int i = 0; i < nn; ++i) inv->M[l][i] = std::move(items[i].out);
  }
  check_status();
  return inv;
}

// ---------------------------------------------------------------------------
// Batched forms: every problem of a call runs in lockstep, one launch per step
// for all of them (the HOD-BF inversion treats all nodes of a T_H level at once).
// ---------------------------------------------------------------------------
template <typename T>
void BFContext<T>::run_lstsq(std::vector<LstsqJob<T>>& lj) {
  if (lj.empty()) return;
  int mc = 1, mr = 1, mw = 1;
  for (auto& j : lj) {
    mc = std::max(mc, (int)j.c);
    mr = std::max(mr, (int)j.r);
    mw = std::max(mw, (int)j.w);
  }
  const bool in_smem = lstsq_smem_bytes<T>(mc, mr, mw, true) <= kLstsqSmemCap;
  if (!in_smem)
    for (auto& j : lj) j.W = scratch.takeT<T>((size_t)lstsq_work_elems(j.c, j.r, j.w));
  const LstsqJob<T>* d = stage(lj.data(), lj.size());
  if (launch_lstsq<T>(d, (int)lj.size(), mc, mr, mw, in_smem, status.as<int32_t>(), st) != 0)
    throw std::runtime_error("centre block too large for the least-squares kernel");
}

template <typename T>
Blk<T> BFContext<T>::make_sketch(int rows, const std::vector<Range>& groups, int q, int level, int side, uint32_t key,
                                 std::vector<std::pair<int, int>>& cols) {
  HostTimer ht_(t_host + H_SKETCH);
  cols.clear();
  int tot = 0;
  std::vector<SketchGroup> sg;
  for (size_t g = 0; g < groups.size(); ++g) {
    int size = (int)(groups[g].b - groups[g].a);
    int w = size <= q ? size : q;
    cols.push_back({tot, tot + w});
    SketchGroup sgr;
    sgr.a = groups[g].a; sgr.b = groups[g].b; sgr.c0 = tot; sgr.w = w;
    sgr.key = (int32_t)((key * 1000003u + (uint32_t)level * 7919u + (uint32_t)side * 104729u + (uint32_t)g) & 0xFFFFFF);
    sgr.identity = (w == size) ? 1 : 0;
    if (w > 0) sg.push_back(sgr);
    tot += w;
  }
  Blk<T> Om = new_blk<T>(scratch, rows, std::max(tot, 1));
  Om.cols = tot;
  zero(Om);
  if (!sg.empty()) {
    int mx = 0;
    for (auto& g : sg) mx = std::max<int>(mx, (int)((g.b - g.a) * g.w));
    const SketchGroup* dg = stage(sg.data(), sg.size());
    launch_sketch<T>(dg, (int)sg.size(), mx, Om.p, Om.plane, (int)Om.ld, st);
  }
  return Om;
}

template <typename T>
Blk<T> BFContext<T>::make_sketch_levels(int rows, const std::vector<std::pair<const std::vector<Range>*, int>>& lv,
                                        int q, int side, uint32_t key,
                                        std::vector<std::vector<std::pair<int, int>>>& cols, std::vector<int>& base) {
  HostTimer ht_(t_host + H_SKETCH);
  cols.assign(lv.size(), {});
  base.assign(lv.size(), 0);
  int tot = 0;
  std::vector<SketchGroup> sg;
  for (size_t k = 0; k < lv.size(); ++k) {
    const std::vector<Range>& groups = *lv[k].first;
    const int level = lv[k].second;
    base[k] = tot;
    int tl = 0;
    for (size_t g = 0; g < groups.size(); ++g) {
      int size = (int)(groups[g].b - groups[g].a);
      int w = size <= q ? size : q;
      cols[k].push_back({tl, tl + w});
      SketchGroup sgr;
      sgr.a = groups[g].a; sgr.b = groups[g].b; sgr.c0 = tot + tl; sgr.w = w;
      sgr.key = (int32_t)((key * 1000003u + (uint32_t)level * 7919u + (uint32_t)side * 104729u + (uint32_t)g) & 0xFFFFFF);
      sgr.identity = (w == size) ? 1 : 0;
      if (w > 0) sg.push_back(sgr);
      tl += w;
    }
    tot += tl;
  }
  Blk<T> Om = new_blk<T>(scratch, rows, std::max(tot, 1));
  Om.cols = tot;
  zero(Om);
  if (!sg.empty()) {
    int mx = 0;
    for (auto& g : sg) mx = std::max<int>(mx, (int)((g.b - g.a) * g.w));
    const SketchGroup* dg = stage(sg.data(), sg.size());
    launch_sketch<T>(dg, (int)sg.size(), mx, Om.p, Om.plane, (int)Om.ld, st);
  }
  return Om;
}

template <typename T>
std::vector<Blk<T>> BFContext<T>::copy_b(const std::vector<Blk<T>>& x) {
  std::vector<Blk<T>> out(x.size());
  std::vector<Blk2Job<T>> jobs;
  for (size_t q = 0; q < x.size(); ++q) {
    out[q] = new_blk<T>(scratch, x[q].rows, x[q].cols);
    Blk2Job<T> j{};
    j.src = x[q].p; j.splane = x[q].plane; j.sld = x[q].ld;
    j.dst = out[q].p; j.dplane = out[q].plane; j.dld = out[q].ld;
    j.rows = x[q].rows; j.cols = x[q].cols; j.alpha = T(1); j.mode = 3;
    if (j.rows && j.cols) jobs.push_back(j);
  }
  run_blk2(*this, jobs);
  return out;
}

template <typename T>
void BFContext<T>::axpy_b(const std::vector<Blk<T>>& x, std::vector<Blk<T>>& y, T alpha) {
  std::vector<Blk2Job<T>> jobs;
  for (size_t q = 0; q < x.size(); ++q) {
    Blk2Job<T> j{};
    j.src = x[q].p; j.splane = x[q].plane; j.sld = x[q].ld;
    j.dst = y[q].p; j.dplane = y[q].plane; j.dld = y[q].ld;
    j.rows = x[q].rows; j.cols = x[q].cols; j.alpha = alpha; j.mode = 2;
    if (j.rows && j.cols) jobs.push_back(j);
  }
  run_blk2(*this, jobs);
}

template <typename T>
void BFContext<T>::random_matvec_batch(const DOpB<T>& op, std::vector<RMProblem<T>>& probs, int L,
                                       const BFParams& P) {
  HostTimer ht_(t_host + H_RMV);
  const size_t nq = probs.size();
  if (!nq) return;
  const int lc = L / 2;
  const int q0 = (P.max_rank > 0 ? P.max_rank : P.q_start) + P.p;
  for (auto& pb : probs) {
    pb.out = std::make_unique<DBF<T>>();
    pb.out->init(pb.m, pb.n, pb.rt, pb.ct, L);
  }
  const size_t mk = scratch.mark();
  std::vector<Blk<T>> cOm(nq), cY(nq);
  std::vector<std::vector<std::pair<int, int>>> ccols(nq);
  auto gather_blk = [&](const Blk<T>& Y, const IdxVec& rows, std::pair<int, int> cols, std::vector<GatherJob<T>>& gj) {
    Blk<T> M = new_blk<T>(scratch, (int)rows.size(), cols.second - cols.first);
    GatherJob<T> g;
    g.src = Y.p; g.splane = Y.plane; g.sld = Y.ld;
    g.rows = dev_idx(*this, rows);
    g.c0 = cols.first;
    g.nrows = (int)rows.size();
    g.ncols = cols.second - cols.first;
    g.dst = M.p; g.dplane = M.plane; g.dld = M.ld;
    if (g.nrows && g.ncols) gj.push_back(g);
    return M;
  };
  auto run_gathers = [&](std::vector<GatherJob<T>>& gj) {
    if (gj.empty()) return;
    int64_t mx = 0;
    for (auto& g : gj) mx = std::max<int64_t>(mx, (int64_t)g.nrows * g.ncols);
    const GatherJob<T>* d = stage(gj.data(), gj.size());
    launch_gather_rows<T>(d, (int)gj.size(), mx, st);
  };
  // With a rank cap the sketch widths are fixed and no sketch depends on an earlier level's
  // IDs, so all levels of one side go through the operator in one application (fused);
  // without a cap the width may grow per level and each level applies the operator itself.
  const bool fused = P.max_rank > 0;
  for (int side = 0; side < 2; ++side) {
    const int lfirst = side == 0 ? L : 0, llast = lc, step = side == 0 ? -1 : 1;
    std::vector<Blk<T>> OmAll(nq), YAll(nq);
    std::vector<std::vector<std::vector<std::pair<int, int>>>> lcols(nq);
    std::vector<std::vector<int>> lbase(nq);
    if (fused) {
      for (size_t t = 0; t < nq; ++t) {
        DBF<T>& bf = *probs[t].out;
        std::vector<std::pair<const std::vector<Range>*, int>> lv;
        for (int l = lfirst;; l += step) {
          lv.push_back({side == 0 ? &bf.ct[L - l] : &bf.rt[l], l});
          if (l == llast) break;
        }
        OmAll[t] = make_sketch_levels(side == 0 ? bf.n : bf.m, lv, q0, side, probs[t].key, lcols[t], lbase[t]);
        YAll[t] = new_blk<T>(scratch, side == 0 ? bf.m : bf.n, std::max(OmAll[t].cols, 1));
        YAll[t].cols = OmAll[t].cols;
      }
      op(OmAll, YAll, side == 1);
    }
    for (int l = lfirst;; l += step) {
      int q = q0;
      const size_t mkl = scratch.mark();
      const int li = side == 0 ? lfirst - l : l - lfirst;   // position of l in the fused sketch
      for (;;) {
        std::vector<Blk<T>> Om(nq), Yb(nq);
        std::vector<std::vector<std::pair<int, int>>> cols(nq);
        if (fused) {
          for (size_t t = 0; t < nq; ++t) {
            const int w = li + 1 < (int)lbase[t].size() ? lbase[t][li + 1] - lbase[t][li] : OmAll[t].cols - lbase[t][li];
            Om[t] = OmAll[t].sub(0, lbase[t][li], OmAll[t].rows, w);
            Yb[t] = YAll[t].sub(0, lbase[t][li], YAll[t].rows, w);
            cols[t] = lcols[t][li];
          }
        } else {
          for (size_t t = 0; t < nq; ++t) {
            DBF<T>& bf = *probs[t].out;
            const auto& groups = side == 0 ? bf.ct[L - l] : bf.rt[l];
            Om[t] = make_sketch(side == 0 ? bf.n : bf.m, groups, q, l, side, probs[t].key, cols[t]);
            Yb[t] = new_blk<T>(scratch, side == 0 ? bf.m : bf.n, std::max(Om[t].cols, 1));
            Yb[t].cols = Om[t].cols;
          }
          op(Om, Yb, side == 1);
        }
        std::vector<Blk<T>> Ms;
        std::vector<GatherJob<T>> gj;
        std::vector<IdxVec> sets;
        std::vector<std::pair<size_t, int>> owner;
        for (size_t t = 0; t < nq; ++t) {
          DBF<T>& bf = *probs[t].out;
          for (int i = 0; i < (1 << l); ++i)
            for (int j = 0; j < (1 << (L - l)); ++j) {
              IdxVec X;
              int grp;
              if (side == 0) {
                X = l == L ? range_vec(bf.rt[L][i].a, bf.rt[L][i].b)
                           : cat(bf.Osk[l + 1][bf.pidx(l + 1, 2 * i, j / 2)],
                                 bf.Osk[l + 1][bf.pidx(l + 1, 2 * i + 1, j / 2)]);
                grp = j;
              } else {
                X = l == 0 ? range_vec(bf.ct[L][j].a, bf.ct[L][j].b)
                           : cat(bf.Ssk[l - 1][bf.pidx(l - 1, i / 2, 2 * j)],
                                 bf.Ssk[l - 1][bf.pidx(l - 1, i / 2, 2 * j + 1)]);
                grp = i;
              }
              Ms.push_back(gather_blk(Yb[t], X, cols[t][grp], gj));
              sets.push_back(X);
              owner.push_back({t, grp});
            }
        }
        run_gathers(gj);
        std::vector<IdxVec> sk;
        std::vector<Blk<T>> Us;
        row_ids(Ms, P.tol, P.max_rank, sk, Us);
        bool grow = false;
        if (P.max_rank <= 0)
          for (size_t p = 0; p < Ms.size(); ++p) {
            const size_t t = owner[p].first;
            const int grp = owner[p].second;
            const DBF<T>& bf = *probs[t].out;
            const Range g = side == 0 ? bf.ct[L - l][grp] : bf.rt[l][grp];
            const int w = cols[t][grp].second - cols[t][grp].first;
            if (w < (int)(g.b - g.a) && (int)sk[p].size() > w - P.p) grow = true;
          }
        if (grow && q < 4096) {
          q *= 2;
          scratch.release(mkl);
          continue;
        }
        size_t p = 0;
        for (size_t t = 0; t < nq; ++t) {
          DBF<T>& bf = *probs[t].out;
          for (int k = 0; k < (1 << L); ++k, ++p) {
            IdxVec o;
            for (int32_t x : sk[p]) o.push_back(sets[p][x]);
            if (side == 0) { bf.U[l][k] = Us[p]; bf.Osk[l][k] = o; }
            else { bf.V[l][k] = Us[p]; bf.Ssk[l][k] = o; }
          }
        }
        if (side == 0 && l == lc) {
          cOm = Om;
          cY = Yb;
          ccols = cols;
        }
        break;
      }
      if (side == 1) scratch.release(mkl);
      if (l == llast) break;
    }
  }
  // centre blocks by least squares, all problems in one launch
  std::vector<LstsqJob<T>> lj;
  std::vector<GatherJob<T>> gj;
  for (size_t t = 0; t < nq; ++t) {
    DBF<T>& bf = *probs[t].out;
    std::vector<Blk<T>> xs;
    right_transform(bf, cOm[t], xs);
    for (int i = 0; i < (1 << lc); ++i)
      for (int j = 0; j < (1 << (L - lc)); ++j) {
        const int p = bf.pidx(lc, i, j);
        const int r = bf.rr(lc, i, j), c = bf.rc(lc, i, j);
        Blk<T> Bm = new_blk<T>(persist, r, std::max(c, 1));
        Bm.cols = c;
        bf.B[p] = Bm;
        if (r == 0 || c == 0) continue;
        Blk<T> Yr = gather_blk(cY[t], bf.Osk[lc][p], ccols[t][j], gj);
        LstsqJob<T> L1;
        L1.Tm = xs[p].p + ccols[t][j].first; L1.tplane = xs[p].plane; L1.tld = xs[p].ld;
        L1.Y = Yr.p; L1.yplane = Yr.plane; L1.yld = Yr.ld;
        L1.B = Bm.p; L1.bplane = Bm.plane; L1.bld = Bm.ld;
        L1.c = c; L1.r = r; L1.w = ccols[t][j].second - ccols[t][j].first;
        L1.W = nullptr;
        lj.push_back(L1);
        flops += 8.0 * ((double)c * c * L1.w + (double)r * c * L1.w);
      }
  }
  run_gathers(gj);
  run_lstsq(lj);
  sync();
  scratch.release(mk);
}

template <typename T>
void BFContext<T>::inv_apply_b(const DHODBFInv<T>& Hi, int l0, const std::vector<int>& i0s, const std::vector<Blk<T>>& X,
                               std::vector<Blk<T>>& Y, bool transpose) {
  const int LH = Hi.LH;
  const size_t nq = i0s.size();
  if (!nq) return;
  const int nsub = 1 << (LH - l0);
  std::vector<Blk<T>> Z(nq);
  for (size_t q = 0; q < nq; ++q) Z[q] = new_blk<T>(scratch, X[q].rows, X[q].cols);
  auto leaves = [&](const std::vector<Blk<T>>& src, std::vector<Blk<T>>& out) {
    std::vector<GemmDesc<T>> g;
    for (size_t q = 0; q < nq; ++q) {
      const int64_t a0 = Hi.tree[l0][i0s[q]].a;
      const int k = X[q].cols;
      for (int li = i0s[q] * nsub; li < (i0s[q] + 1) * nsub; ++li) {
        const Range r = Hi.tree[LH][li];
        const int nr = (int)(r.b - r.a);
        if (nr == 0) continue;
        g.push_back(gdesc<T>(nr, k, nr, transpose ? 1 : 0, 0, T(1), T(0), Hi.Dinv[li],
                             src[q].sub((int)(r.a - a0), 0, nr, k), out[q].sub((int)(r.a - a0), 0, nr, k)));
      }
    }
    gemm(g);
  };
  auto level = [&](int l) {
    const int span = 1 << (l - l0);
    std::vector<const DBF<T>*> bfs;
    std::vector<Blk<T>> xs, zs;
    for (size_t q = 0; q < nq; ++q) {
      const int64_t a0 = Hi.tree[l0][i0s[q]].a;
      const int k = X[q].cols;
      for (int i = i0s[q] * span; i < (i0s[q] + 1) * span; ++i) {
        const Range r = Hi.tree[l][i];
        bfs.push_back(Hi.M[l][i].get());
        xs.push_back(Y[q].sub((int)(r.a - a0), 0, (int)(r.b - r.a), k));
        zs.push_back(Z[q].sub((int)(r.a - a0), 0, (int)(r.b - r.a), k));
      }
    }
    apply(bfs, xs, zs, transpose, false);
    axpy_b(Z, Y, T(1));
  };
  if (!transpose) {
    leaves(X, Y);
    for (int l = LH - 1; l >= l0; --l) level(l);
  } else {
    std::vector<Blk2Job<T>> cj;
    for (size_t q = 0; q < nq; ++q) {
      Blk2Job<T> j{};
      j.src = X[q].p; j.splane = X[q].plane; j.sld = X[q].ld;
      j.dst = Y[q].p; j.dplane = Y[q].plane; j.dld = Y[q].ld; j.rows = X[q].rows; j.cols = X[q].cols; j.alpha = T(1);
      j.mode = 3;
      cj.push_back(j);
    }
    run_blk2(*this, cj);
    for (int l = l0; l <= LH - 1; ++l) {
      // Z must not carry the previous level's values into the axpy: level() overwrites Z first
      level(l);
    }
    leaves(Y, Z);
    std::vector<Blk2Job<T>> bj;
    for (size_t q = 0; q < nq; ++q) {
      Blk2Job<T> j{};
      j.src = Z[q].p; j.splane = Z[q].plane; j.sld = Z[q].ld;
      j.dst = Y[q].p; j.dplane = Y[q].plane; j.dld = Y[q].ld; j.rows = X[q].rows; j.cols = X[q].cols; j.alpha = T(1);
      j.mode = 3;
      bj.push_back(j);
    }
    run_blk2(*this, bj);
  }
}

template <typename T>
std::vector<std::unique_ptr<DBF<T>>> BFContext<T>::bf_smw_batch(const std::vector<const DBF<T>*>& Ks,
                                                               const std::vector<uint32_t>& keys,
                                                               const BFParams& P) {
  std::vector<std::unique_ptr<DBF<T>>> out(Ks.size());
  if (Ks.empty()) return out;
  const int L = Ks[0]->L;
  if (L <= 1) {
    for (size_t q = 0; q < Ks.size(); ++q) out[q] = bf_smw(*Ks[q], P, keys[q]);
    return out;
  }
  std::vector<std::unique_ptr<DBF<T>>> k11(Ks.size()), k12(Ks.size()), k21(Ks.size()), k22(Ks.size());
  std::vector<const DBF<T>*> k22p;
  std::vector<uint32_t> k22keys;
  for (size_t q = 0; q < Ks.size(); ++q) {
    k11[q] = split_child(*Ks[q], 0, 0);
    k12[q] = split_child(*Ks[q], 0, 1);
    k21[q] = split_child(*Ks[q], 1, 0);
    k22[q] = split_child(*Ks[q], 1, 1);
    k22p.push_back(k22[q].get());
    k22keys.push_back(keys[q] * 4u + 1u);
  }
  auto k22i = bf_smw_batch(k22p, k22keys, P);
  std::vector<SmwItem<T>> items(Ks.size());
  for (size_t q = 0; q < Ks.size(); ++q) {
    items[q].n = Ks[q]->m;
    items[q].tr = Ks[q]->rt;
    items[q].K11 = k11[q].get();
    items[q].K12 = k12[q].get();
    items[q].K21 = k21[q].get();
    items[q].K22i = k22i[q].get();
    items[q].key = keys[q];
  }
  smw_assemble_batch(items, L, P);
  for (size_t q = 0; q < Ks.size(); ++q) out[q] = std::move(items[q].out);
  return out;
}

template <typename T>
void BFContext<T>::smw_assemble_batch(std::vector<SmwItem<T>>& items, int L, const BFParams& P) {
  const size_t nq = items.size();
  if (!nq) return;
  std::vector<int> n1(nq), n2(nq);
  for (size_t q = 0; q < nq; ++q) {
    n1[q] = (int)items[q].tr[1][0].b;
    n2[q] = items[q].n - n1[q];
  }
  auto apply_list = [&](const std::vector<const DBF<T>*>& K, const std::vector<Blk<T>>& x, std::vector<Blk<T>>& y,
                        bool tr, bool acc) {
    std::vector<const DBF<T>*> b;
    std::vector<Blk<T>> xs, ys;
    for (size_t q = 0; q < K.size(); ++q)
      if (K[q]) { b.push_back(K[q]); xs.push_back(x[q]); ys.push_back(y[q]); }
    apply(b, xs, ys, tr, acc);
  };
  std::vector<const DBF<T>*> K11(nq), K12(nq), K21(nq), K22i(nq);
  for (size_t q = 0; q < nq; ++q) {
    K11[q] = items[q].K11; K12[q] = items[q].K12; K21[q] = items[q].K21; K22i[q] = items[q].K22i;
  }
  // z = (I + K22i) y
  auto inv22 = [&](const std::vector<Blk<T>>& y, bool tr) {
    std::vector<Blk<T>> z = copy_b(y);
    apply_list(K22i, y, z, tr, true);
    return z;
  };
  auto newb = [&](const std::vector<int>& rows, const std::vector<Blk<T>>& like) {
    std::vector<Blk<T>> v(nq);
    for (size_t q = 0; q < nq; ++q) v[q] = new_blk<T>(scratch, rows[q], like[q].cols);
    return v;
  };
  // S = K11 - K12 (I + K22i) K21
  DOpB<T> sop = [&](const std::vector<Blk<T>>& X, std::vector<Blk<T>>& Y, bool tr) {
    std::vector<Blk<T>> t = newb(n2, X);
    apply_list(tr ? K12 : K21, X, t, tr, false);
    std::vector<Blk<T>> u = inv22(t, tr);
    apply_list(tr ? K21 : K12, u, Y, tr, false);
    axpy_b(Y, Y, T(-2));
    apply_list(K11, X, Y, tr, true);
  };
  std::vector<RMProblem<T>> sp(nq);
  for (size_t q = 0; q < nq; ++q) {
    sp[q].m = sp[q].n = n1[q];
    sp[q].rt = subtree(items[q].tr, 1, 0, L - 2);
    sp[q].ct = sp[q].rt;
    sp[q].key = items[q].key * 4u + 2u;
  }
  random_matvec_batch(sop, sp, L - 2, P);
  std::vector<const DBF<T>*> Sl;
  std::vector<uint32_t> skeys;
  for (size_t q = 0; q < nq; ++q) {
    Sl.push_back(sp[q].out.get());
    skeys.push_back(items[q].key * 4u + 3u);
  }
  auto K11i = bf_smw_batch(Sl, skeys, P);
  std::vector<const DBF<T>*> K11ip(nq);
  for (size_t q = 0; q < nq; ++q) K11ip[q] = K11i[q].get();
  // A^-1 - I, A^-1 = [I 0; -A22^-1 A21 I] diag(A11^-1, A22^-1) [I -A12 A22^-1; 0 I]
  DOpB<T> fop = [&](const std::vector<Blk<T>>& X, std::vector<Blk<T>>& Y, bool tr) {
    std::vector<Blk<T>> x1(nq), x2(nq), y1(nq), y2(nq);
    for (size_t q = 0; q < nq; ++q) {
      const int k = X[q].cols;
      x1[q] = X[q].sub(0, 0, n1[q], k); x2[q] = X[q].sub(n1[q], 0, n2[q], k);
      y1[q] = Y[q].sub(0, 0, n1[q], k); y2[q] = Y[q].sub(n1[q], 0, n2[q], k);
    }
    std::vector<Blk<T>> w = inv22(x2, tr);                 // A22^-1 x2   (or A22^-T x2)
    std::vector<Blk<T>> t1 = newb(n1, X);
    apply_list(tr ? K21 : K12, w, t1, tr, false);         // K12 w  (or K21^T w)
    axpy_b(t1, t1, T(-2));                                // t1 = -t1
    axpy_b(x1, t1, T(1));                                 // t1 = x1 - K12 A22^-1 x2
    std::vector<Blk2Job<T>> cj;
    for (size_t q = 0; q < nq; ++q) {
      Blk2Job<T> j{};
      j.src = t1[q].p; j.splane = t1[q].plane; j.sld = t1[q].ld;
      j.dst = y1[q].p; j.dplane = y1[q].plane; j.dld = y1[q].ld; j.rows = n1[q]; j.cols = X[q].cols; j.alpha = T(1);
      j.mode = 3;
      cj.push_back(j);
    }
    run_blk2(*this, cj);
    apply_list(K11ip, t1, y1, tr, true);                  // y1 = A11^-1 t1
    std::vector<Blk<T>> v = newb(n2, X);
    apply_list(tr ? K12 : K21, y1, v, tr, false);         // K21 y1  (or K12^T y1)
    std::vector<Blk<T>> vv = inv22(v, tr);
    std::vector<Blk2Job<T>> c3;
    for (size_t q = 0; q < nq; ++q) {
      Blk2Job<T> j{};
      j.src = w[q].p; j.splane = w[q].plane; j.sld = w[q].ld;
      j.dst = y2[q].p; j.dplane = y2[q].plane; j.dld = y2[q].ld; j.rows = n2[q]; j.cols = X[q].cols; j.alpha = T(1);
      j.mode = 3;
      c3.push_back(j);
    }
    run_blk2(*this, c3);
    axpy_b(vv, y2, T(-1));
    axpy_b(X, Y, T(-1));                                  // minus the identity
  };
  std::vector<RMProblem<T>> fp(nq);
  for (size_t q = 0; q < nq; ++q) {
    fp[q].m = fp[q].n = items[q].n;
    fp[q].rt = items[q].tr;
    fp[q].ct = items[q].tr;
    fp[q].key = items[q].key * 4u;
  }
  random_matvec_batch(fop, fp, L, P);
  for (size_t q = 0; q < nq; ++q) items[q].out = std::move(fp[q].out);
}

template struct DBF<float>;
template struct DBF<double>;
template struct DHODBF<float>;
template struct DHODBF<double>;
template struct DHODBFInv<float>;
template struct DHODBFInv<double>;
template class BFContext<float>;
template class BFContext<double>;

}  // namespace mf
