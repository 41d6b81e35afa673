// Batched row interpolative decomposition with a fixed, library-owned scratch
// area instead of per-call device allocations.
//
// Some callers cannot allocate device memory at the point where they need an
// ID: applications whose own pool allocator reserves the GPU's memory up front
// and hands out every buffer itself (a cudaMalloc from the library would fail or
// take memory the pool counts on), and latency-sensitive loops that must not
// call cudaMalloc / cudaFree because those calls can synchronize the whole
// device and stall the work of other streams.  For them mf_row_id_c64_noalloc
// does the same work as mf_row_id_c64, with the QR work matrix placed in the
// file-scope array below.  The array is a static device allocation of
// MF_ID_SCRATCH_FLOATS floats (8 MiB); every GPU that loads this library holds
// it until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/mf.h"
#include "bf_id_body.cuh"
#include "bf_kernels.h"

namespace mf {

constexpr size_t MF_ID_SCRATCH_FLOATS = size_t(2) << 20;   // 2 Mi floats = 8 MiB

static __device__ __align__(256) float g_id_scratch[MF_ID_SCRATCH_FLOATS];

namespace {

// Job q of a uniform batch, built on the device from scalar arguments (no job array in memory).
__global__ void __launch_bounds__(256) k_row_id_fixed_scratch(const float* M, int m, int n, float* U, int kmax,
                                                               int32_t* sk, int32_t* rank, float* scratch, float tol,
                                                               int max_rank) {
  const int q = blockIdx.x;
  IdJob<float> jb;
  jb.M = M + (size_t)2 * m * n * q;
  jb.plane = (int64_t)m * n;
  jb.ld = n;
  jb.m = m;
  jb.n = n;
  jb.U = U + (size_t)2 * m * kmax * q;
  jb.uplane = (int64_t)m * kmax;
  jb.ldu = kmax;
  jb.sk = sk + (size_t)kmax * q;
  jb.rank = rank + q;
  jb.work = scratch + (size_t)2 * m * n * q;
  jb.wplane = (int64_t)m * n;
  row_id_body<float>(jb, tol, max_rank, false);
}

constexpr int kMaxDevices = 64;
float* g_scratch_ptr[kMaxDevices] = {};
std::once_flag g_once[kMaxDevices];
cudaError_t g_setup_err[kMaxDevices] = {};

}  // namespace
}  // namespace mf

extern "C" int mf_row_id_c64_noalloc(int32_t nmat, int32_t m, int32_t n, const float* M, double tol,
                                     int32_t max_rank, float* U, int32_t* sk, int32_t* rank, void* stream) {
  using namespace mf;
  if (nmat <= 0 || m <= 0 || n <= 0 || m > 2048 || n > 8192 || !M || !U || !sk || !rank || !(tol >= 0))
    return MF_ERR_ARG;
  if ((size_t)2 * m * n * nmat > MF_ID_SCRATCH_FLOATS) return MF_ERR_ARG;   // batch exceeds the fixed scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MF_ERR_CUDA;
  // set-up, once per device, with that device current: the device address of the scratch array
  std::call_once(g_once[dev], [dev]() {
    void* p = nullptr;
    g_setup_err[dev] = cudaGetSymbolAddress(&p, g_id_scratch);
    if (g_setup_err[dev] == cudaSuccess) {
      g_setup_err[dev] = cudaFuncSetAttribute(k_row_id_fixed_scratch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              200 * 1024);
    }
    g_scratch_ptr[dev] = static_cast<float*>(p);
  });
  if (g_setup_err[dev] != cudaSuccess || !g_scratch_ptr[dev]) return MF_ERR_CUDA;
  int kmax = std::min(m, n);
  if (max_rank > 0) kmax = std::min(kmax, (int)max_rank);
  size_t sm = sizeof(float) * (2 * (size_t)n + m) + sizeof(int) * (size_t)m;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  count_launches(1);
  k_row_id_fixed_scratch<<<nmat, 256, sm, st>>>(M, m, n, U, kmax, sk, rank, g_scratch_ptr[dev], (float)tol,
                                                 max_rank);
  if (cudaGetLastError() != cudaSuccess) return MF_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MF_ERR_CUDA;
  return MF_OK;
}
