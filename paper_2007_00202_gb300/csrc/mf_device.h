// Device-side descriptors shared by the CUDA kernels and the host runtime.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mf {

// A planar complex matrix: real plane at re, imaginary plane at re + plane.
// Row-major with leading dimension ld (elements).
template <typename T>
struct PMat {
  T* re;
  int64_t plane;
  int64_t ld;
};

// One batched GEMM problem: C = alpha * op(A) op(B) + beta * C  (complex, planar).
// transA = 0: A is M x K row-major (K contiguous); 1: A stored K x M row-major.
// transB = 0: B is K x N row-major (N contiguous); 1: B stored N x K row-major.
// Optional second term (the narrow kernel k_gemm_nrhs only): with k1 > 0 the first k1
// reduction indices use (A, B) and the remaining k - k1 use (A2, B2) with the same
// transposes, i.e. C = alpha (op(A) op(B) + op(A2) op(B2)) + beta C.
template <typename T>
struct GemmDesc {
  int32_t m, n, k;
  int32_t transA, transB;
  T alpha, beta;       // real scalars
  PMat<T> A, B, C;
  int32_t k1 = 0;
  PMat<T> A2{}, B2{};
};

// A tile of a batched GEMM: problem index and tile coordinates.
struct GemmTile {
  int32_t desc;
  int32_t tm, tn;
  int32_t pad;
};

// Per-front device descriptor for the dense multifrontal path.  All matrices
// are planar complex, row-major; the imaginary plane follows at the stated
// plane stride.
template <typename T>
struct FrontDev {
  int64_t sep_begin;     // I^s = [sep_begin, sep_begin + s)
  int32_t s, u;
  const int64_t* upd;    // I^u (device, sorted new indices)
  T* LU;                 // s x s : F11, LU in place (work)
  T* UT;                 // s x s : U^T, lower triangular (work)
  T* Linv;               // s x s : L^-1 (unit lower), zero above the diagonal   [factor]
  T* UinvT;              // s x s : (U^-1)^T (lower), zero above the diagonal     [factor]
  T* F12w;               // u x s : F12^T as assembled (work)
  T* F12p;               // u x s : (P^T F12)^T (work)
  T* F12T;               // u x s : (L^-1 P^T F12)^T                             [factor]
  T* F21w;               // u x s : F21 as assembled (work)
  T* F21f;               // u x s : F21 U^-1                                     [factor]
  T* C;                  // u x u : F22, then the contribution block (until the parent is assembled)
  T* W;                  // s x s work
  int32_t* piv;          // s pivots (LAPACK convention: row k swapped with piv[k] at step k)
  int32_t* perm;         // s gather permutation: (P^T b)[k] = b[perm[k]]
  int32_t ls, lu;        // leading dimensions of s-wide and u-wide rows (s, u rounded up to 4)
  int64_t pl_ss, pl_us, pl_uu;   // plane strides of s x s, u x s and u x u matrices
};

// Work item for the extend-add of one child contribution block into its parent.
template <typename T>
struct ExtendAddItem {
  const T* Cc;           // child's u_c x u_c block (planar)
  int64_t plane_c;
  const int32_t* rel;    // u_c positions in the parent front (0..s_p+u_p-1)
  int32_t uc;
  int32_t ldc;           // leading dimension of the child's block
  int32_t parent;        // index into the FrontDev array
};

// Status word written by kernels (0 = fine).
enum : int32_t { DEV_OK = 0, DEV_ZERO_PIVOT = 1 };

}  // namespace mf
