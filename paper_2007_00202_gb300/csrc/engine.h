// Runtime of the GPU multifrontal solver: device memory plan, the factor and
// solve launch programs, and the FP64 refinement loop.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "analysis.h"
#include "kernels.h"
#include "mf_device.h"

namespace mf {

struct CudaError : std::runtime_error {
  using std::runtime_error::runtime_error;
};
struct SingularError : std::runtime_error {
  using std::runtime_error::runtime_error;
};
// a bounded device-side wait expired (MF_ERR_TIMEOUT)
struct TimeoutError : std::runtime_error {
  using std::runtime_error::runtime_error;
};

#define MF_CUDA(x)                                                                                         \
  do {                                                                                                     \
    cudaError_t e_ = (x);                                                                                  \
    if (e_ != cudaSuccess)                                                                                 \
      throw ::mf::CudaError(std::string(#x) + ": " + cudaGetErrorString(e_) + " (" + __FILE__ + ":" +      \
                            std::to_string(__LINE__) + ")");                                               \
  } while (0)

// Owning device buffer.
struct DevMem {
  void* p = nullptr;
  size_t bytes = 0;
  DevMem() = default;
  DevMem(const DevMem&) = delete;
  DevMem& operator=(const DevMem&) = delete;
  DevMem(DevMem&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
  DevMem& operator=(DevMem&& o) noexcept {
    if (this != &o) { reset(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
    return *this;
  }
  ~DevMem() { reset(); }
  void reset() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  void alloc(size_t b) {
    reset();
    if (b == 0) b = 256;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      p = nullptr;
      throw CudaError(std::string("cudaMalloc of ") + std::to_string(b) + " bytes: " + cudaGetErrorString(e));
    }
    bytes = b;
  }
  template <typename U>
  U* as() const { return reinterpret_cast<U*>(p); }
};

template <typename U>
void upload(DevMem& m, const std::vector<U>& v, cudaStream_t st) {
  m.alloc(v.size() * sizeof(U));
  if (!v.empty()) MF_CUDA(cudaMemcpyAsync(m.p, v.data(), v.size() * sizeof(U), cudaMemcpyHostToDevice, st));
}

// Device copy of the permuted matrix (new numbering).
struct DeviceMatrix {
  int64_t n = 0, nnz = 0;
  DevMem rowptr, col64, col32, vals;   // vals: interleaved complex128
};

// CUDA-event timing of the launches of one kernel family: a start and a stop event
// around every launch; collect() reads the finished pairs and adds them up.  Inside a
// CUDA graph capture the events come from the graph's own list (capture_into), and
// every replay of the graph hands that list back through replayed().
struct LaunchProfiler {
  struct Rec {
    cudaEvent_t a, b;
    double flops, bytes;
  };
  bool on = false;
  int every = 1;                    // time one eager launch (and one graph replay) in `every`
  int64_t calls = 0;
  std::vector<Rec>* capture_into = nullptr;
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  int64_t launches = 0, recorded = 0;
  double ms = 0, flops = 0, bytes = 0;

  LaunchProfiler() = default;
  LaunchProfiler(const LaunchProfiler&) = delete;
  LaunchProfiler& operator=(const LaunchProfiler&) = delete;
  ~LaunchProfiler() {
    for (auto e : pool) cudaEventDestroy(e);
  }
  static cudaEvent_t make_event() {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) throw CudaError("cudaEventCreate failed");
    return e;
  }
  std::mutex mu;   // two host threads may launch timed kernels (fronts of one level)
  template <class F>
  void time(cudaStream_t st, double fl, double by, F&& launch) {
    std::unique_lock<std::mutex> lk(mu);
    if (!on || (!capture_into && (calls++ % every) != 0)) {
      lk.unlock();
      launch();
      return;
    }
    Rec r;
    if (capture_into) {   // events of the graph: created by reserve_graph before the capture
      const size_t i = capture_into->size();
      if (i >= graph_reserve.size()) {   // not reserved: leave this launch untimed
        lk.unlock();
        launch();
        return;
      }
      r = graph_reserve[i];
    } else {
      while (pool.size() < pool_used + 2) pool.push_back(make_event());
      r.a = pool[pool_used++];
      r.b = pool[pool_used++];
    }
    r.flops = fl;
    r.bytes = by;
    std::vector<Rec>* into = capture_into ? capture_into : &pending;
    lk.unlock();
    // inside a capture an event becomes a record node of the graph only as an "external" record
    const unsigned fl_rec = into != &pending ? cudaEventRecordExternal : cudaEventRecordDefault;
    cudaEventRecordWithFlags(r.a, st, fl_rec);
    launch();
    cudaEventRecordWithFlags(r.b, st, fl_rec);
    lk.lock();
    ++recorded;
    into->push_back(r);
  }
  // n event pairs for a graph about to be captured (owned by the caller afterwards)
  std::vector<Rec> graph_reserve;
  void reserve_graph(size_t n) {
    graph_reserve.clear();
    for (size_t i = 0; i < n; ++i) graph_reserve.push_back(Rec{make_event(), make_event(), 0, 0});
  }
  void replayed(const std::vector<Rec>& recs) {
    std::lock_guard<std::mutex> lk(mu);
    if (on) pending.insert(pending.end(), recs.begin(), recs.end());
  }
  void collect() {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& r : pending) {
      float t = 0;
      if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
        ms += t;
        flops += r.flops;
        bytes += r.bytes;
        ++launches;
      }
    }
    pending.clear();
    pool_used = 0;
  }
  void enable(int period) {   // 0: off; N > 0: time one launch in N
    collect();
    std::lock_guard<std::mutex> lk(mu);
    on = period > 0;
    every = period > 0 ? period : 1;
    calls = 0;
    launches = 0;
    ms = flops = bytes = 0;
  }
};

class EngineBase {
 public:
  virtual ~EngineBase() = default;
  virtual void factor(double tol) = 0;
  // preconditioner on planar-free interleaved FP64 data in the new numbering:
  // y = M^-1 x  (x, y: n x nrhs column-major interleaved complex128, ld = n; may alias)
  virtual void apply_precond(const double* x, double* y, int nrhs) = 0;
  virtual double factor_flops() const = 0;
  virtual double factor_bytes() const = 0;
  virtual int launches_factor() const = 0;
  virtual int launches_solve(int nrhs) = 0;
  virtual int max_rank() const { return 0; }
  // Inspection of a compressed front's operators: Y = K X with K one of F11 (which 0), F11^-1
  // (1), F12 (2), F21 (3) or the contribution block C (4) of front fid; X (in x nrhs) and Y
  // (out x nrhs) host, column-major, interleaved complex128.  Returns 0, or -1 when fid is not a
  // compressed front or has no such operator.
  virtual int front_apply(int fid, int which, int nrhs, const double* x, double* y) { return -1; }
  virtual double compressed_seconds() const { return 0; }
  // peak use and capacity of the compressed fronts' device arenas (all contexts)
  virtual void arena_usage(double& peak, double& capacity) const { peak = capacity = 0; }
  // Event timing of two kernel families (see mf_profile in mf.h):
  // prof[0] the narrow GEMM (k_gemm_nrhs) in factor() and apply_precond(), prof[1] the
  // factor's dense front GEMMs (Schur updates).
  LaunchProfiler prof[2];
  virtual void set_profiling(int period) {
    for (auto& p : prof) p.enable(period);
  }
};

// Parameters of the compressed fronts (Alg. 2-5).
struct EngineOptions {
  int max_rank = 0;
  int alpha = 2, knn = 8;
  uint64_t seed = 1;
  size_t persist_bytes = size_t(24) << 30;   // device arena for compressed factors
  size_t scratch_bytes = size_t(12) << 30;   // device arena for construction work, per context
  int max_contexts = 8;                        // construction contexts (host threads) per tree level
};

std::unique_ptr<EngineBase> make_engine_c64(const Analysis& an, const DeviceMatrix& A, cudaStream_t st,
                                            const EngineOptions& eo);
std::unique_ptr<EngineBase> make_engine_c128(const Analysis& an, const DeviceMatrix& A, cudaStream_t st,
                                             const EngineOptions& eo);

}  // namespace mf
