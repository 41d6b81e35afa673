// Device job descriptors and launchers of the butterfly-path kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace mf {

// One row interpolative decomposition (Sec. 3) of M (m x n, planar, row-major, ld).
// Outputs: *rank, sk[0..rank) (skeleton rows), U (m x rank used, ld = ldu).
// work: scratch of m x n per plane (overwritten by the QR).
template <typename T>
struct IdJob {
  const T* M;
  int64_t plane, ld;
  int32_t m, n;
  T* U;
  int64_t uplane;
  int32_t ldu;
  int32_t* sk;
  int32_t* rank;
  T* work;
  int64_t wplane;
};

// A group of sketch columns: rows [a, b) x cols [c0, c0 + w) of a row-major
// matrix; identity columns (w == b - a) or counter-based Gaussians keyed by key.
struct SketchGroup {
  int64_t a, b;
  int32_t c0, w;
  int32_t key;
  int32_t identity;
};

// dst[i][c] = src[rows[i]][c0 + c]
template <typename T>
struct GatherJob {
  const T* src;
  int64_t splane, sld;
  const int32_t* rows;
  int32_t c0;
  int32_t nrows, ncols;
  T* dst;
  int64_t dplane, dld;
};

// A dense contribution block of a child and the map front position -> child position (-1 if absent).
template <typename T>
struct DenseKid {
  const T* C;
  int64_t plane, ld;
  const int32_t* inv;
};

template <typename T>
struct FrontCtx {
  int64_t sep_begin;
  int32_t s, u;
  const int64_t* upd;
  int32_t nkids;
  DenseKid<T> kids[2];
};

// Entries of the front at (X[a], Y[b]) (front-local positions): A-part (if with_A) + dense children.
template <typename T>
struct FrontEntryJob {
  int32_t ctx;
  const int32_t* X;
  const int32_t* Y;
  int32_t nx, ny;
  T* dst;
  int64_t dplane, dld;
  int32_t with_A;
  int32_t accumulate;
};

// dst[rows[a]][cols[b]] += sign * src[a][b]
template <typename T>
struct PlaceJob {
  const T* src;
  int64_t splane, sld;
  const int32_t* rows;
  const int32_t* cols;
  int32_t nr, nc;
  T* dst;
  int64_t dplane, dld;
  T sign;
  int32_t atomic;      // 1: jobs of the launch may overlap in dst (atomic adds)
};

template <typename T>
struct InvJob {
  const T* A;
  int64_t aplane, lda;
  int32_t n;
  T* X;
  int64_t xplane, ldx;
  double* W;           // work of 2 n^2 doubles (real and imaginary planes) when not in shared memory
};
// Gauss-Jordan elimination with partial pivoting in FP64 (stored in T); the
// augmented matrix sits in shared memory when the launch's largest job fits.
// per-step vectors (column and row k, re / im, in FP64) and the pivots, 16-byte aligned
__host__ __device__ inline size_t small_inverse_vec_bytes(int n) {
  return ((4 * sizeof(double) + sizeof(int)) * (size_t)n + 15) / 16 * 16;
}
// dynamic shared memory of the small inverse with its n x n FP64 work in shared memory (elem:
// the work's element size, sizeof(double))
inline size_t small_inverse_smem_bytes(int max_n, size_t elem) {
  return small_inverse_vec_bytes(max_n) + 2 * (size_t)max_n * max_n * elem;
}
constexpr size_t kSmallInvSmemCap = 200 * 1024;

// Block-to-block operations on planar row-major blocks:
//   mode 0: dst = src^T (plain transpose), dst is cols x rows
//   mode 1: dst[a][b] += alpha * src[ridx[a]][cidx[b]]   (gather of a sub-block; cidx NULL: b)
//   mode 4: dst[a][b]  = alpha * src[ridx[a]][cidx[b]]   (the same, assigning)
//   mode 2: dst += alpha * src
//   mode 3: dst = src
template <typename T>
struct Blk2Job {
  const T* src;
  int64_t splane, sld;
  T* dst;
  int64_t dplane, dld;
  int32_t rows, cols;
  T alpha;
  const int32_t* ridx;
  const int32_t* cidx;
  int32_t mode;
};

// B (r x c) minimising ||B Tm - Y||_F for Tm (c x w), Y (r x w), row by row:
// Tm^T B[i,:]^T = Y[i,:]^T in the least-squares sense, by Householder QR with
// column pivoting of Tm^T (whose columns are the contiguous rows of Tm), with
// the reflections applied to the rows of Y in the same pass; columns of Tm^T
// below a relative pivot of 64 eps get a zero coefficient.  Work in shared
// memory when the launch's largest job fits, else in W.
template <typename T>
struct LstsqJob {
  const T* Tm;
  int64_t tplane, tld;
  const T* Y;
  int64_t yplane, yld;
  T* B;
  int64_t bplane, bld;
  int32_t c, r, w;
  T* W;                // work of lstsq_work_elems(c, r, w) T values, used only when the launch says so
};

inline int64_t lstsq_work_elems(int c, int r, int w) { return 2 * (int64_t)(c + r) * w; }
// Dynamic shared memory of one k_lstsq CTA: the work (if held there), the
// Householder vector, the column norms and the column permutation.
template <typename T>
inline size_t lstsq_smem_bytes(int max_c, int max_r, int max_w, bool work_in_smem) {
  size_t b = (size_t)(2 * max_w + max_c) * sizeof(T) + (size_t)max_c * 4 + 16;
  if (work_in_smem) b += (size_t)lstsq_work_elems(max_c, max_r, max_w) * sizeof(T);
  return b;
}
constexpr size_t kLstsqSmemCap = 200 * 1024;

template <typename T>
void launch_blk2(const Blk2Job<T>* d_jobs, int njobs, int64_t max_elems, cudaStream_t st);
template <typename T>
int launch_lstsq(const LstsqJob<T>* d_jobs, int njobs, int max_c, int max_r, int max_w, bool work_in_smem,
                 int32_t* status, cudaStream_t st);

// Dynamic shared memory of one row-ID CTA (m x n matrix); the work matrix adds 2 m n values.
// launch_row_id takes the largest per-job figure (smem_bytes), or computes it from max_m, max_n.
inline size_t row_id_smem_bytes(int m, int n, size_t elem, bool work_in_smem) {
  size_t b = elem * (2 * (size_t)n + m) + sizeof(int) * (size_t)m;
  if (work_in_smem) b += elem * 2 * (size_t)m * n;
  return b;
}
constexpr size_t kRowIdSmemCap = 200 * 1024;
// Cluster row ID (the work matrix in global memory, shared by the CTAs of a cluster): per CTA the
// Householder vector, the norms and the position order.
inline size_t row_id_cluster_smem_bytes(int m, int n, size_t elem) {
  return elem * (2 * (size_t)n + m) + 2 * sizeof(int) * (size_t)m;
}
// Register-resident row ID for m <= 128 and n <= 128 (1024 threads, rows in registers): its
// dynamic shared memory (pivot row, the rows' first min(m, n) columns, the pivots).
inline size_t row_id_reg_smem_bytes(int m, int n, size_t elem) {
  const int kw = m < n ? m : n;
  return elem * (2 * (size_t)n + 2 * (size_t)m * kw) + sizeof(int) * (size_t)m + 16;
}
template <typename T>
int launch_row_id_reg(const IdJob<T>* d_jobs, int njobs, int max_m, int max_n, T tol, int max_rank, cudaStream_t st);
template <typename T>
int launch_row_id(const IdJob<T>* d_jobs, int njobs, int max_m, int max_n, T tol, int max_rank, cudaStream_t st,
                  bool work_in_smem = false, size_t smem_bytes = 0);
template <typename T>
void launch_sketch(const SketchGroup* d_groups, int ngroups, int max_elems, T* out, int64_t plane, int ld,
                   cudaStream_t st);
template <typename T>
void launch_gather_rows(const GatherJob<T>* d_jobs, int njobs, int64_t max_elems, cudaStream_t st);
template <typename T>
void launch_front_entries(const FrontEntryJob<T>* d_jobs, int njobs, int64_t max_elems, const FrontCtx<T>* d_ctx,
                          const int64_t* rowptr, const int32_t* colind, const double* vals, cudaStream_t st);
template <typename T>
void launch_place(const PlaceJob<T>* d_jobs, int njobs, int64_t max_elems, cudaStream_t st);
template <typename T>
int launch_small_inverse(const InvJob<T>* d_jobs, int njobs, int max_n, bool work_in_smem, int32_t* status,
                         cudaStream_t st);

}  // namespace mf
