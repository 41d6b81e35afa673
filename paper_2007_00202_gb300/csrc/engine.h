// Runtime of the GPU multifrontal solver: device memory plan, the factor and
// solve launch programs, and the FP64 refinement loop.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <map>
#include <memory>
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
  virtual double compressed_seconds() const { return 0; }
  // Event timing of the dominant kernel (the batched front GEMM) inside factor().
  struct Profile {
    int64_t launches = 0;
    double ms = 0, flops = 0;
  };
  bool profiling = false;
  Profile prof;
};

// Parameters of the compressed fronts (Alg. 2-5).
struct EngineOptions {
  int max_rank = 0;
  int alpha = 2, knn = 8;
  uint64_t seed = 1;
  size_t persist_bytes = size_t(24) << 30;   // device arena for compressed factors
  size_t scratch_bytes = size_t(12) << 30;   // device arena for construction work
};

std::unique_ptr<EngineBase> make_engine_c64(const Analysis& an, const DeviceMatrix& A, cudaStream_t st,
                                            const EngineOptions& eo);
std::unique_ptr<EngineBase> make_engine_c128(const Analysis& an, const DeviceMatrix& A, cudaStream_t st,
                                             const EngineOptions& eo);

}  // namespace mf
