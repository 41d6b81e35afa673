// CUDA kernels of the butterfly path (Sec. 3-5): batched interpolative
// decomposition, counter-based Gaussian sketches, and the gathers that feed
// entry extraction from a front (A's entries and dense contribution blocks).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "bf_id_body.cuh"
#include "bf_kernels.h"

namespace mf {

// ---------------------------------------------------------------------------
// Batched row ID (Sec. 3), one CTA per matrix (body in bf_id_body.cuh).
// ---------------------------------------------------------------------------
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_row_id(const IdJob<T>* jobs, T tol, int32_t max_rank, int work_in_smem) {
  row_id_body<T>(jobs[blockIdx.x], tol, max_rank, work_in_smem != 0);
}

// the large matrices (QR work in global memory): a cluster of kIdCluster CTAs per matrix
constexpr int kIdCluster = 8;
template <typename T>
__global__ void __launch_bounds__(1024, 1) k_row_id_cluster(const IdJob<T>* jobs, T tol, int32_t max_rank) {
  row_id_body_cluster<T, kIdCluster>(jobs[blockIdx.x / kIdCluster], tol, max_rank);
}

template <typename T, int RC>
__global__ void __launch_bounds__(1024, 1) k_row_id_reg(const IdJob<T>* jobs, T tol, int32_t max_rank) {
  row_id_body_reg<T, RC>(jobs[blockIdx.x], tol, max_rank);
}

template <typename T>
int launch_row_id_reg(const IdJob<T>* d_jobs, int njobs, int max_m, int max_n, T tol, int max_rank,
                      cudaStream_t st) {
  if (njobs <= 0) return 0;
  if (max_m > 128 || max_n > 128) return -1;
  const size_t sm = row_id_reg_smem_bytes(max_m, max_n, sizeof(T));
  static PerDeviceOnce attr;
  attr([] {
    cudaFuncSetAttribute(k_row_id_reg<T, 10>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRowIdSmemCap);
    cudaFuncSetAttribute(k_row_id_reg<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRowIdSmemCap);
  });
  count_launches(1);
  if (max_n <= 80) k_row_id_reg<T, 10><<<njobs, 1024, sm, st>>>(d_jobs, tol, max_rank);
  else k_row_id_reg<T, 16><<<njobs, 1024, sm, st>>>(d_jobs, tol, max_rank);
  return 0;
}

template <typename T>
int launch_row_id(const IdJob<T>* d_jobs, int njobs, int max_m, int max_n, T tol, int max_rank, cudaStream_t st,
                  bool work_in_smem, size_t smem_bytes) {
  if (njobs <= 0) return 0;
  const size_t sm = smem_bytes ? smem_bytes : row_id_smem_bytes(max_m, max_n, sizeof(T), work_in_smem);
  if (sm > kRowIdSmemCap) return -1;
  static PerDeviceOnce attr;
  attr([] {
    cudaFuncSetAttribute(k_row_id<T, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRowIdSmemCap);
    cudaFuncSetAttribute(k_row_id<T, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRowIdSmemCap);
  });
  count_launches(1);
  if (work_in_smem) {
    // large shared-memory work (one or two CTAs per SM): four times the threads per matrix
    if (sm > 64 * 1024) k_row_id<T, 1024><<<njobs, 1024, sm, st>>>(d_jobs, tol, max_rank, 1);
    else k_row_id<T, 256><<<njobs, 256, sm, st>>>(d_jobs, tol, max_rank, 1);
    return 0;
  }
  // matrices in global memory are the large ones (few per launch): a cluster of kIdCluster
  // 1024-thread CTAs each, every CTA updating its share of the rows
  static PerDeviceOnce cattr;
  cattr([] {
    cudaFuncSetAttribute(k_row_id_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRowIdSmemCap);
  });
  const size_t csm = row_id_cluster_smem_bytes(max_m, max_n, sizeof(T));
  if (csm > kRowIdSmemCap) return -1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)njobs * kIdCluster, 1, 1);
  cfg.blockDim = dim3(1024, 1, 1);
  cfg.dynamicSmemBytes = csm;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kIdCluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_row_id_cluster<T>, d_jobs, tol, (int32_t)max_rank);
  return 0;
}

// ---------------------------------------------------------------------------
// Counter-based complex Gaussian sketches: splitmix64 (Steele, Lea, Flood 2014)
// on the counter (key << 40) ^ (col << 24) ^ row, hashed twice (2c, 2c + 1) to
// two uniforms in (0, 1) (24-bit for complex64, 53-bit for complex128), Box-Muller,
// scaled by 1/sqrt(2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t smix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  uint64_t z = x;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__global__ void k_sketch(const SketchGroup* groups, int ngroups, T* out, int64_t plane, int ld) {
  // out: rows x ld row-major planar; group g fills rows [a, b) x cols [c0, c0 + w)
  const SketchGroup g = groups[blockIdx.y];
  const int64_t total = (int64_t)(g.b - g.a) * g.w;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = g.a + e / g.w;
    const int col = (int)(e % g.w);
    T re, im;
    if (g.identity) {
      re = (row - g.a == col) ? T(1) : T(0);
      im = T(0);
    } else {
      uint64_t c = ((uint64_t)(g.key & 0xFFFFFF) << 40) ^ ((uint64_t)(col & 0xFFFF) << 24) ^ (uint64_t)row;
      uint64_t h1 = smix(c * 2ull), h2 = smix(c * 2ull + 1ull);
      if constexpr (sizeof(T) == 4) {   // 24-bit uniforms and single-precision Box-Muller (FP64 is slow here)
        float u1 = ((float)(h1 >> 40) + 0.5f) * (1.0f / 16777216.0f);
        float u2 = ((float)(h2 >> 40) + 0.5f) * (1.0f / 16777216.0f);
        float rad = sqrtf(-2.0f * logf(u1)) * 0.70710678f;
        float s, co;
        sincospif(2.0f * u2, &s, &co);
        re = (T)(rad * co);
        im = (T)(rad * s);
      } else {
        double u1 = ((double)(h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        double u2 = ((double)(h2 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        double rad = sqrt(-2.0 * log(u1));
        double ang = 6.283185307179586476925286766559 * u2;
        re = (T)(rad * cos(ang) * 0.70710678118654752440);
        im = (T)(rad * sin(ang) * 0.70710678118654752440);
      }
    }
    const int64_t off = row * ld + g.c0 + col;
    out[off] = re;
    out[off + plane] = im;
  }
}

template <typename T>
void launch_sketch(const SketchGroup* d_groups, int ngroups, int max_elems, T* out, int64_t plane, int ld,
                   cudaStream_t st) {
  if (ngroups <= 0 || max_elems <= 0) return;
  int bx = (max_elems + 255) / 256;
  if (bx > 256) bx = 256;
  count_launches(1);
  k_sketch<T><<<dim3(bx, ngroups), 256, 0, st>>>(d_groups, ngroups, out, plane, ld);
}

// ---------------------------------------------------------------------------
// Gathers.  Row / column index lists are given per block; dst is row-major
// planar (ld = number of columns of the block).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_gather_rows(const GatherJob<T>* jobs) {
  // dst[i][c] = src[rows[i]][c0 + c]  (c < ncols)
  const GatherJob<T> j = jobs[blockIdx.y];
  const int64_t total = (int64_t)j.nrows * j.ncols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / j.ncols;
    int c = (int)(e % j.ncols);
    int64_t so = (int64_t)j.rows[i] * j.sld + j.c0 + c;
    int64_t dof = i * j.dld + c;
    j.dst[dof] = j.src[so];
    j.dst[dof + j.dplane] = j.src[so + j.splane];
  }
}

template <typename T>
void launch_gather_rows(const GatherJob<T>* d_jobs, int njobs, int64_t max_elems, cudaStream_t st) {
  if (njobs <= 0 || max_elems <= 0) return;
  int bx = (int)((max_elems + 255) / 256);
  if (bx > 512) bx = 512;
  count_launches(1);
  k_gather_rows<T><<<dim3(bx, njobs), 256, 0, st>>>(d_jobs);
}

// Front entries for a list of blocks: out(x, y) = A-part + dense children (+ sign * extra)
template <typename T>
__global__ void k_front_entries(const FrontEntryJob<T>* jobs, const FrontCtx<T>* ctx, const int64_t* rowptr,
                                const int32_t* colind, const double* vals) {
  const FrontEntryJob<T> j = jobs[blockIdx.y];
  const FrontCtx<T> c = ctx[j.ctx];
  const int64_t total = (int64_t)j.nx * j.ny;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / j.ny), b = (int)(e % j.ny);
    const int x = j.X[a], y = j.Y[b];   // front-local positions
    T vr = 0, vi = 0;
    if (j.with_A && (x < c.s || y < c.s)) {
      const int64_t gx = x < c.s ? c.sep_begin + x : c.upd[x - c.s];
      const int64_t gy = y < c.s ? c.sep_begin + y : c.upd[y - c.s];
      for (int64_t k = rowptr[gx]; k < rowptr[gx + 1]; ++k)
        if (colind[k] == gy) {
          vr = (T)vals[2 * k];
          vi = (T)vals[2 * k + 1];
          break;
        }
    }
    for (int q = 0; q < c.nkids; ++q) {
      const DenseKid<T>& kd = c.kids[q];
      if (!kd.C) continue;
      const int px = kd.inv[x], py = kd.inv[y];
      if (px >= 0 && py >= 0) {
        const int64_t o = (int64_t)px * kd.ld + py;
        vr += kd.C[o];
        vi += kd.C[o + kd.plane];
      }
    }
    const int64_t o = (int64_t)a * j.dld + b;
    if (j.accumulate) {
      j.dst[o] += vr;
      j.dst[o + j.dplane] += vi;
    } else {
      j.dst[o] = vr;
      j.dst[o + j.dplane] = vi;
    }
  }
}

template <typename T>
void launch_front_entries(const FrontEntryJob<T>* d_jobs, int njobs, int64_t max_elems, const FrontCtx<T>* d_ctx,
                          const int64_t* rowptr, const int32_t* colind, const double* vals, cudaStream_t st) {
  if (njobs <= 0 || max_elems <= 0) return;
  int bx = (int)((max_elems + 255) / 256);
  if (bx > 512) bx = 512;
  count_launches(1);
  k_front_entries<T><<<dim3(bx, njobs), 256, 0, st>>>(d_jobs, d_ctx, rowptr, colind, vals);
}

// Scatter-add of a dense block into a sub-block of a destination: dst[rows][cols] += src (used to place
// extracted pieces into list blocks).
template <typename T>
__global__ void k_place(const PlaceJob<T>* jobs) {
  const PlaceJob<T> j = jobs[blockIdx.y];
  const int64_t total = (int64_t)j.nr * j.nc;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / j.nc), b = (int)(e % j.nc);
    const int64_t so = (int64_t)a * j.sld + b;
    const int64_t dof = (int64_t)j.rows[a] * j.dld + j.cols[b];
    if (j.atomic) {
      atomicAdd(j.dst + dof, j.sign * j.src[so]);
      atomicAdd(j.dst + dof + j.dplane, j.sign * j.src[so + j.splane]);
    } else {
      j.dst[dof] += j.sign * j.src[so];
      j.dst[dof + j.dplane] += j.sign * j.src[so + j.splane];
    }
  }
}

template <typename T>
void launch_place(const PlaceJob<T>* d_jobs, int njobs, int64_t max_elems, cudaStream_t st) {
  if (njobs <= 0 || max_elems <= 0) return;
  int bx = (int)((max_elems + 255) / 256);
  if (bx > 512) bx = 512;
  count_launches(1);
  k_place<T><<<dim3(bx, njobs), 256, 0, st>>>(d_jobs);
}

// Dense inverse of small square blocks by Gauss-Jordan elimination with
// partial pivoting (largest modulus), computed in FP64 (work matrix in global
// memory, L2-resident) and stored as T.  One CTA per block.  Used for the leaf blocks D_tau of HOD-BF
// inverses (Alg. 4, "directly compute D_tau^-1").
template <typename T>
__global__ void __launch_bounds__(256) k_small_inverse(const InvJob<T>* jobs, int work_in_smem, int32_t* status) {
  // In-place complex Gauss-Jordan with partial pivoting (largest modulus, lowest row on ties), in
  // FP64 whatever the storage precision.  Step k: swap rows k and p, scale row k by 1 / a_kk
  // (a_kk <- 1 / a_kk), eliminate column k from the other rows (a_ik <- -a_ik / a_kk); the row
  // interchanges are undone at the end as column interchanges in reverse order.
  const InvJob<T> j = jobs[blockIdx.x];
  using R = double;
  const int n = j.n;
  extern __shared__ __align__(16) unsigned char smraw[];
  R* colr = reinterpret_cast<R*>(smraw);   // column k before the step (re, im)
  R* coli = colr + n;
  R* rowr = coli + n;                      // row k after scaling (re, im)
  R* rowi = rowr + n;
  int* piv = reinterpret_cast<int*>(rowi + n);
  R* Ar = work_in_smem ? reinterpret_cast<R*>(smraw + small_inverse_vec_bytes(n)) : j.W;   // n x n
  R* Ai = Ar + (int64_t)n * n;
  __shared__ int sp;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int r = e / n, c = e - r * n;
    Ar[e] = (R)j.A[(int64_t)r * j.lda + c];
    Ai[e] = (R)j.A[(int64_t)r * j.lda + c + j.aplane];
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (tid < 32) {
      R best = R(-1);
      int bi = n;
      for (int r = k + tid; r < n; r += 32) {
        const R m2 = Ar[r * n + k] * Ar[r * n + k] + Ai[r * n + k] * Ai[r * n + k];
        if (m2 > best) { best = m2; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const R ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        sp = bi < n ? bi : k;
        piv[k] = sp;
        if (!(best > R(0)) && status) atomicExch(status, (int32_t)DEV_ZERO_PIVOT);
      }
    }
    __syncthreads();
    const int p = sp;
    if (p != k)
      for (int c = tid; c < n; c += blockDim.x) {
        R t = Ar[k * n + c]; Ar[k * n + c] = Ar[p * n + c]; Ar[p * n + c] = t;
        t = Ai[k * n + c]; Ai[k * n + c] = Ai[p * n + c]; Ai[p * n + c] = t;
      }
    __syncthreads();
    R dr = Ar[k * n + k], di = Ai[k * n + k];
    R den = dr * dr + di * di;
    if (den == R(0)) { dr = R(1); di = R(0); den = R(1); }
    const R ir = dr / den, ii = -di / den;   // 1 / a_kk
    for (int e = tid; e < n; e += blockDim.x) {
      colr[e] = Ar[e * n + k];
      coli[e] = Ai[e * n + k];
      const R a = Ar[k * n + e], b = Ai[k * n + e];
      rowr[e] = e == k ? ir : a * ir - b * ii;
      rowi[e] = e == k ? ii : a * ii + b * ir;
    }
    __syncthreads();
    for (int r = ty; r < n; r += 16) {
      const R fr = colr[r], fi = coli[r];
      for (int c = tx; c < n; c += 16) {
        const int e = r * n + c;
        if (r == k) {
          Ar[e] = rowr[c];
          Ai[e] = rowi[c];
        } else if (c == k) {
          Ar[e] = -(fr * ir - fi * ii);
          Ai[e] = -(fr * ii + fi * ir);
        } else {
          const R a = rowr[c], b = rowi[c];
          Ar[e] -= fr * a - fi * b;
          Ai[e] -= fr * b + fi * a;
        }
      }
    }
    __syncthreads();
  }
  // undo the row interchanges: column interchanges in reverse order, each thread on its rows
  for (int r = tid; r < n; r += blockDim.x)
    for (int k = n - 1; k >= 0; --k) {
      const int q = piv[k];
      if (q == k) continue;
      R t = Ar[r * n + k]; Ar[r * n + k] = Ar[r * n + q]; Ar[r * n + q] = t;
      t = Ai[r * n + k]; Ai[r * n + k] = Ai[r * n + q]; Ai[r * n + q] = t;
    }
  __syncthreads();
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int r = e / n, c = e - r * n;
    j.X[(int64_t)r * j.ldx + c] = (T)Ar[e];
    j.X[(int64_t)r * j.ldx + c + j.xplane] = (T)Ai[e];
  }
}

template <typename T>
int launch_small_inverse(const InvJob<T>* d_jobs, int njobs, int max_n, bool work_in_smem, int32_t* status,
                         cudaStream_t st) {
  if (njobs <= 0) return 0;
  // the step vectors always sit in shared memory; the work matrix too when work_in_smem
  const size_t smem = work_in_smem ? small_inverse_smem_bytes(max_n, sizeof(double)) : small_inverse_vec_bytes(max_n);
  if (smem > kSmallInvSmemCap) return -1;
  static PerDeviceOnce attr;
  attr([] {
    cudaFuncSetAttribute(k_small_inverse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallInvSmemCap);
  });
  count_launches(1);
  k_small_inverse<T><<<njobs, 256, smem, st>>>(d_jobs, work_in_smem ? 1 : 0, status);
  return 0;
}

template <typename T>
__global__ void k_blk2(const Blk2Job<T>* jobs) {
  const Blk2Job<T> j = jobs[blockIdx.y];
  const int64_t total = (int64_t)j.rows * j.cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / j.cols), c = (int)(e % j.cols);
    if (j.mode == 0) {
      const int64_t so = (int64_t)r * j.sld + c, dof = (int64_t)c * j.dld + r;
      j.dst[dof] = j.src[so];
      j.dst[dof + j.dplane] = j.src[so + j.splane];
    } else if (j.mode == 1 || j.mode == 4) {
      const int64_t so = (int64_t)j.ridx[r] * j.sld + (j.cidx ? j.cidx[c] : c), dof = (int64_t)r * j.dld + c;
      if (j.mode == 1) {
        j.dst[dof] += j.alpha * j.src[so];
        j.dst[dof + j.dplane] += j.alpha * j.src[so + j.splane];
      } else {
        j.dst[dof] = j.alpha * j.src[so];
        j.dst[dof + j.dplane] = j.alpha * j.src[so + j.splane];
      }
    } else if (j.mode == 2) {
      const int64_t so = (int64_t)r * j.sld + c, dof = (int64_t)r * j.dld + c;
      j.dst[dof] += j.alpha * j.src[so];
      j.dst[dof + j.dplane] += j.alpha * j.src[so + j.splane];
    } else {
      const int64_t so = (int64_t)r * j.sld + c, dof = (int64_t)r * j.dld + c;
      j.dst[dof] = j.src[so];
      j.dst[dof + j.dplane] = j.src[so + j.splane];
    }
  }
}

template <typename T>
void launch_blk2(const Blk2Job<T>* d_jobs, int njobs, int64_t max_elems, cudaStream_t st) {
  if (njobs <= 0 || max_elems <= 0) return;
  int bx = (int)((max_elems + 255) / 256);
  if (bx > 512) bx = 512;
  count_launches(1);
  k_blk2<T><<<dim3(bx, njobs), 256, 0, st>>>(d_jobs);
}

template <typename T>
__global__ void __launch_bounds__(256) k_lstsq(const LstsqJob<T>* jobs, int work_in_smem) {
  const LstsqJob<T> j = jobs[blockIdx.x];
  const int c = j.c, r = j.r, w = j.w;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int64_t wplane = (int64_t)(c + r) * w;
  T* Wr = work_in_smem ? reinterpret_cast<T*>(smraw) : j.W;
  T* Wi = Wr + wplane;
  T* vr = reinterpret_cast<T*>(smraw) + (work_in_smem ? 2 * wplane : 0);   // Householder vector
  T* vi = vr + w;
  T* nrm = vi + w;                                 // remaining squared column norms, by position
  int* perm = reinterpret_cast<int*>(nrm + c);     // position -> column of Tm^T (row of Tm)
  __shared__ T red_v[8];
  __shared__ int red_i[8];
  __shared__ T sh_alpha_r, sh_alpha_i, sh_scale, sh_ref;
  __shared__ int sh_stop;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const T eps = sizeof(T) == 4 ? T(1.1920929e-7) : T(2.220446049250313e-16);
  // rows 0..c-1 of the work: the rows of Tm (columns of Tm^T); rows c..c+r-1: the rows of Y
  for (int q = warp; q < c + r; q += nw) {
    const bool isT = q < c;
    const T* sr = isT ? j.Tm + (int64_t)q * j.tld : j.Y + (int64_t)(q - c) * j.yld;
    const T* si = sr + (isT ? j.tplane : j.yplane);
    T s = 0;
    for (int t = lane; t < w; t += 32) {
      T x = sr[t], y = si[t];
      Wr[(int64_t)q * w + t] = x;
      Wi[(int64_t)q * w + t] = y;
      s += x * x + y * y;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (isT && lane == 0) { nrm[q] = s; perm[q] = q; }
  }
  const int kmax = c < w ? c : w;
  if (tid == 0) sh_stop = 0;
  __syncthreads();
  int rank = 0;
  for (int k = 0; k < kmax; ++k) {
    T best = T(-1);
    int bi = c;
    for (int q = k + tid; q < c; q += blockDim.x)
      if (nrm[q] > best) { best = nrm[q]; bi = q; }
    for (int o = 16; o > 0; o >>= 1) {
      T ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      best = red_v[0]; bi = red_i[0];
      for (int u = 1; u < nw; ++u)
        if (red_v[u] > best || (red_v[u] == best && red_i[u] < bi)) { best = red_v[u]; bi = red_i[u]; }
      T nu = sqrt(best > T(0) ? best : T(0));
      if (k == 0) sh_ref = nu;
      if (sh_ref == T(0) || nu <= T(64) * eps * sh_ref) sh_stop = 1;
      else {
        T t = nrm[k]; nrm[k] = nrm[bi]; nrm[bi] = t;
        int ti = perm[k]; perm[k] = perm[bi]; perm[bi] = ti;
      }
    }
    __syncthreads();
    if (sh_stop) break;
    T* xr = Wr + (int64_t)perm[k] * w;
    T* xi = Wi + (int64_t)perm[k] * w;
    T s2 = 0;
    for (int t = k + tid; t < w; t += blockDim.x) {
      T x = xr[t], y = xi[t];
      vr[t] = x; vi[t] = y;
      s2 += x * x + y * y;
    }
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (lane == 0) red_v[warp] = s2;
    __syncthreads();
    if (tid == 0) {
      T tot = 0;
      for (int u = 0; u < nw; ++u) tot += red_v[u];
      T nx = sqrt(tot);
      T x0r = vr[k], x0i = vi[k];
      T ax0 = sqrt(x0r * x0r + x0i * x0i);
      T phr = ax0 > T(0) ? x0r / ax0 : T(1), phi = ax0 > T(0) ? x0i / ax0 : T(0);
      T alr = -phr * nx, ali = -phi * nx;
      vr[k] = x0r - alr;
      vi[k] = x0i - ali;
      T vv = tot - (x0r * x0r + x0i * x0i) + vr[k] * vr[k] + vi[k] * vi[k];
      sh_scale = vv > T(0) ? T(2) / vv : T(0);
      sh_alpha_r = alr;
      sh_alpha_i = ali;
    }
    __syncthreads();
    for (int t = k + tid; t < w; t += blockDim.x) {
      xr[t] = t == k ? sh_alpha_r : T(0);
      xi[t] = t == k ? sh_alpha_i : T(0);
    }
    // reflect the remaining columns (positions k+1..c-1, norms updated) and every right-hand side
    const T sc = sh_scale;
    const int nrem = c - k - 1;
    for (int q = warp; q < nrem + r; q += nw) {
      const bool isT = q < nrem;
      const int row = isT ? perm[k + 1 + q] : c + (q - nrem);
      T* yr = Wr + (int64_t)row * w;
      T* yi = Wi + (int64_t)row * w;
      T dr = 0, di = 0;   // v^H y
      for (int t = k + lane; t < w; t += 32) {
        T a = vr[t], b = vi[t], p = yr[t], s = yi[t];
        dr += a * p + b * s;
        di += a * s - b * p;
      }
      for (int o = 16; o > 0; o >>= 1) {
        dr += __shfl_xor_sync(0xffffffffu, dr, o);
        di += __shfl_xor_sync(0xffffffffu, di, o);
      }
      dr *= sc;
      di *= sc;
      T s = 0;
      for (int t = k + lane; t < w; t += 32) {
        T a = vr[t], b = vi[t];
        T p = yr[t] - (a * dr - b * di);
        T u = yi[t] - (a * di + b * dr);
        yr[t] = p;
        yi[t] = u;
        if (t > k) s += p * p + u * u;
      }
      if (isT) {
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) nrm[k + 1 + q] = s;
      }
    }
    __syncthreads();
    rank = k + 1;
  }
  // R11 z = (Q^H y)[0:rank] per right-hand side (one thread each, in place), B[i][perm[b]] = z[b]
  for (int i = tid; i < r; i += blockDim.x) {
    T* yr = Wr + (int64_t)(c + i) * w;
    T* yi = Wi + (int64_t)(c + i) * w;
    for (int b = rank - 1; b >= 0; --b) {
      T accr = yr[b], acci = yi[b];
      for (int cc = b + 1; cc < rank; ++cc) {
        const int64_t pc = (int64_t)perm[cc] * w;
        T Rr = Wr[pc + b], Ri = Wi[pc + b];
        T zr = yr[cc], zi = yi[cc];
        accr -= Rr * zr - Ri * zi;
        acci -= Rr * zi + Ri * zr;
      }
      const int64_t pb = (int64_t)perm[b] * w;
      T dr = Wr[pb + b], di = Wi[pb + b];
      T den = dr * dr + di * di;
      yr[b] = (accr * dr + acci * di) / den;
      yi[b] = (acci * dr - accr * di) / den;
    }
    T* br = j.B + (int64_t)i * j.bld;
    T* bim = br + j.bplane;
    for (int b = 0; b < c; ++b) {
      br[perm[b]] = b < rank ? yr[b] : T(0);
      bim[perm[b]] = b < rank ? yi[b] : T(0);
    }
  }
}

template <typename T>
int launch_lstsq(const LstsqJob<T>* d_jobs, int njobs, int max_c, int max_r, int max_w, bool work_in_smem,
                 int32_t* status, cudaStream_t st) {
  (void)status;
  if (njobs <= 0) return 0;
  const size_t smem = lstsq_smem_bytes<T>(max_c, max_r, max_w, work_in_smem);
  if (smem > kLstsqSmemCap) return -1;
  static PerDeviceOnce attr;
  attr([] { cudaFuncSetAttribute(k_lstsq<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLstsqSmemCap); });
  count_launches(1);
  k_lstsq<T><<<njobs, 256, smem, st>>>(d_jobs, work_in_smem ? 1 : 0);
  return 0;
}

#define MF_BF_INST(T)                                                                                            \
  template int launch_row_id<T>(const IdJob<T>*, int, int, int, T, int, cudaStream_t, bool, size_t);          \
  template int launch_row_id_reg<T>(const IdJob<T>*, int, int, int, T, int, cudaStream_t);                          \
  template void launch_sketch<T>(const SketchGroup*, int, int, T*, int64_t, int, cudaStream_t);                 \
  template void launch_gather_rows<T>(const GatherJob<T>*, int, int64_t, cudaStream_t);                         \
  template void launch_front_entries<T>(const FrontEntryJob<T>*, int, int64_t, const FrontCtx<T>*, const int64_t*, \
                                        const int32_t*, const double*, cudaStream_t);                           \
  template void launch_place<T>(const PlaceJob<T>*, int, int64_t, cudaStream_t);                                \
  template int launch_small_inverse<T>(const InvJob<T>*, int, int, bool, int32_t*, cudaStream_t);                     \
  template void launch_blk2<T>(const Blk2Job<T>*, int, int64_t, cudaStream_t);                                   \
  template int launch_lstsq<T>(const LstsqJob<T>*, int, int, int, int, bool, int32_t*, cudaStream_t);

MF_BF_INST(float)
MF_BF_INST(double)

}  // namespace mf
