// Host-callable launchers of the CUDA kernels (all asynchronous on `st`).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include <mutex>
#include <utility>

#include "mf_device.h"

namespace mf {

// Iteration limit of the bounded mbarrier waits in the tensor-core kernels (0 restores the
// default, 2^26 polls); on expiry a kernel records status 2 (MF_ERR_TIMEOUT).  The final wait
// before a kernel releases its tensor memory always uses the default.
void set_wait_limit(long long spins);
long long wait_limit();
constexpr long long kDefaultWaitLimit = 1ll << 26;
// A limit of at most kProbeWaitLimit polls (tests of the expiry path) also makes every CTA of those
// kernels first wait on an mbarrier that nothing arrives at: the wait runs out, the CTA issues no
// work and reports the expiry.
constexpr long long kProbeWaitLimit = 16;

// Number of kernel launches issued by this library since it was loaded.
int64_t launch_count();
void count_launches(int k);

// Runs a set-up step (a kernel attribute, which CUDA keeps per device) once per device: on the
// first call made with each device current, thread-safe (other callers wait until it is done).
struct PerDeviceOnce {
  static constexpr int kMaxDevices = 64;
  std::once_flag flag[kMaxDevices];
  template <typename F>
  void operator()(F&& f) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
      f();
      return;
    }
    std::call_once(flag[dev], std::forward<F>(f));
  }
};

// Batched planar complex GEMM over a tile list (SIMT).
template <typename T>
void launch_gemm(const GemmDesc<T>* d_desc, const GemmTile* d_tiles, int ntiles, cudaStream_t st);
// Tile size of the SIMT GEMM (both dimensions).
constexpr int GEMM_TILE = 64;

// Narrow planar complex GEMM (n <= 128) over a tile list of tiles {desc, tm, tn} of 32 rows
// and nb columns: nb = gemm_nrhs_width(max n) (a desc has ceil(n / nb) column tiles), ksplit
// the number of CTAs of a thread-block cluster that share one tile's K range (gemm_nrhs_split),
// max_k the largest k of the descs (sizes the pipeline's shared memory; a smaller value only
// shortens the pipeline).
template <typename T>
void launch_gemm_nrhs(const GemmDesc<T>* d_desc, const GemmTile* d_tiles, int ntiles, int nb, int ksplit, int max_k,
                      cudaStream_t st, bool two_term = false);   // two_term: some descs have k1 > 0
constexpr int GEMM_NRHS_ROWS = 32;
// Algorithmic bytes of one product: A and B read once, C written (and read when beta != 0).
template <typename T>
inline double gemm_bytes(const GemmDesc<T>& d) {
  return 2.0 * sizeof(T) * ((double)d.m * d.k + (double)d.k * d.n + (double)d.m * d.n * (d.beta != T(0) ? 2 : 1));
}
int gemm_nrhs_width(int max_n, size_t elem);   // 16 or 32 (column tile); 0 when max_n > 128
int gemm_nrhs_split(int ntiles, int max_k);

// tcgen05 (kind::tf32) planar complex GEMM, "NT" form only (transA = 0, transB = 1),
// leading dimensions multiples of 4, 16-byte aligned planes; 128 x 128 tiles.
// status receives 2 if a bounded wait expired.
// split = true: three-pass split TF32 (hi*hi + hi*lo + lo*hi), close to FP32 accuracy.
void launch_gemm_tc(const GemmDesc<float>* d_desc, const GemmTile* d_tiles, int ntiles, int32_t* status,
                    cudaStream_t st, bool split = true);
int gemm_tc_tile();

// tcgen05 (kind::tf32, split precision) narrow products for complex64 blocks of at most 64 vectors:
// C = alpha (op(A) B [+ A2 B2]) + beta C, transB = 0, n <= 64, any m and k (tiles {desc, tm, 0}
// of gemm_nrhs_tc_rows() rows); persistent CTAs, two per SM.  status receives 2 if a bounded
// wait expired.
bool gemm_nrhs_tc_ok(const GemmDesc<float>& d);
int gemm_nrhs_tc_rows();
void launch_gemm_nrhs_tc(const GemmDesc<float>* d_desc, const GemmTile* d_tiles, int ntiles, int32_t* status,
                         cudaStream_t st);

// Dense front assembly and extend-add (Sec. 2 step 1).
template <typename T>
void launch_assemble_A(FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int maxrows, const int64_t* rowptr,
                       const int64_t* colind, const double* vals, cudaStream_t st);
template <typename T>
void launch_extend_add(const ExtendAddItem<T>* d_items, int nitems, const FrontDev<T>* d_fronts, int max_uc,
                       cudaStream_t st);

// Partial LU of F11 with partial pivoting (Sec. 2 step 2): one panel step.
template <typename T>
void launch_panel_lu(FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int kb, int nb, int max_rows,
                     int32_t* status, cudaStream_t st);
template <typename T>
void launch_panel_trsm(FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int kb, int nb, int max_s,
                       cudaStream_t st);

// After the LU: UT <- U^T (lower, zero above), pivots applied to F12^T columns,
// pivots turned into a gather permutation.
template <typename T>
void launch_post_lu(FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int max_s, int max_u, cudaStream_t st);

// Diagonal-block inverses of a lower triangular matrix (block 64) into X.
// which = 0: T = strict lower of LU with unit diagonal, X = Linv (stored in W2 slot)
// which = 1: T = UT, X = UinvT
template <typename T>
void launch_trinv_diag(FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int max_s, int which, T* const* d_X,
                       cudaStream_t st);

// Gather / scatter of right-hand sides between the global vector and front work.
template <typename T>
void launch_fwd_gather(const FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int max_s, const T* X, int64_t xpl,
                       int nrhs, T* const* d_tmp, cudaStream_t st);
template <typename T>
void launch_scatter_sep(const FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int max_s, T* X, int64_t xpl,
                        int nrhs, T* const* d_src, cudaStream_t st);
template <typename T>
void launch_scatter_add_upd(const FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int max_u, T* X,
                            int64_t xpl, int nrhs, T* const* d_src, cudaStream_t st);
template <typename T>
void launch_gather_upd(const FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int max_u, const T* X,
                       int64_t xpl, int nrhs, T* const* d_dst, cudaStream_t st);
template <typename T>
void launch_gather_sep(const FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int max_s, const T* X,
                       int64_t xpl, int nrhs, T* const* d_dst, cudaStream_t st);

// Conversions between interleaved complex128 (column-major, original numbering)
// and planar T (row-major N x nrhs, new numbering).
template <typename T>
void launch_to_planar(const double* src, int64_t ld, int64_t n, int nrhs, const int64_t* perm, T* dst, int64_t pl,
                      cudaStream_t st, int pld = 0);   // planar rows of pld >= nrhs values (0: nrhs)
template <typename T>
void launch_from_planar(const T* src, int64_t pl, int64_t n, int nrhs, const int64_t* perm, double* dst, int64_t ld,
                        cudaStream_t st, int pld = 0);

// FP64 sparse residual and Krylov helpers (interleaved complex128, column-major n x nrhs).
void launch_spmv_residual(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* vals,
                          const double* x, const double* b, double* r, int nrhs, int64_t ld, cudaStream_t st);
void launch_spmv(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* vals, const double* x,
                 double* y, int nrhs, int64_t ld, cudaStream_t st);
// out[c] = sum_i conj(V[i,c]) W[i,c]  (complex, per column), written as (re, im) pairs
void launch_coldot(int64_t n, int nrhs, const double* V, int64_t ldv, const double* W, int64_t ldw, double* out,
                   cudaStream_t st);
// W[:,c] -= h[c] V[:,c]  (complex h per column)
void launch_colaxpy(int64_t n, int nrhs, const double* h, const double* V, int64_t ldv, double* W, int64_t ldw,
                    double sign, cudaStream_t st);
// Y[:,c] = X[:,c] * s[c] (complex s) ; Y may alias X
void launch_colscale(int64_t n, int nrhs, const double* s, const double* X, int64_t ldx, double* Y, int64_t ldy,
                     cudaStream_t st);
// out[c] = ||X[:,c]||_2^2
void launch_colnorm2(int64_t n, int nrhs, const double* X, int64_t ldx, double* out, cudaStream_t st);

}  // namespace mf
