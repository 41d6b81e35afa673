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
template <typename T>
__global__ void __launch_bounds__(256) k_row_id(const IdJob<T>* jobs, T tol, int32_t max_rank) {
  row_id_body<T>(jobs[blockIdx.x], tol, max_rank);
}

template <typename T>
int launch_row_id(const IdJob<T>* d_jobs, int njobs, int max_m, int max_n, T tol, int max_rank, cudaStream_t st) {
  if (njobs <= 0) return 0;
  size_t sm = sizeof(T) * (2 * (size_t)max_n + max_m) + sizeof(int) * (size_t)max_m;
  if (sm > 200 * 1024) return -1;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_row_id<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  count_launches(1);
  k_row_id<T><<<njobs, 256, sm, st>>>(d_jobs, tol, max_rank);
  return 0;
}

// ---------------------------------------------------------------------------
// Counter-based complex Gaussian sketches: splitmix64 (Steele, Lea, Flood 2014)
// on the counter (key << 40) ^ (col << 24) ^ row, hashed twice (2c, 2c + 1) to
// two 53-bit uniforms in (0, 1), Box-Muller, scaled by 1/sqrt(2).
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
      double u1 = ((double)(h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      double u2 = ((double)(h2 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      double rad = sqrt(-2.0 * log(u1));
      double ang = 6.283185307179586476925286766559 * u2;
      re = (T)(rad * cos(ang) * 0.70710678118654752440);
      im = (T)(rad * sin(ang) * 0.70710678118654752440);
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
    j.dst[dof] += j.sign * j.src[so];
    j.dst[dof + j.dplane] += j.sign * j.src[so + j.splane];
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
// partial pivoting (largest modulus), computed in FP64 and stored as T.  One
// CTA per block, n <= 128.  Used for the leaf blocks D_tau of HOD-BF
// inverses (Alg. 4, "directly compute D_tau^-1").
template <typename T>
__global__ void __launch_bounds__(256) k_small_inverse(const InvJob<T>* jobs, int32_t* status) {
  const InvJob<T> j = jobs[blockIdx.x];
  const int n = j.n;
  extern __shared__ double sm_d[];
  double* Ar = sm_d;                   // n x 2n augmented [A | I]
  double* Ai = Ar + n * 2 * n;
  __shared__ int piv;
  const int w = 2 * n;
  for (int e = threadIdx.x; e < n * w; e += blockDim.x) {
    int r = e / w, c = e % w;
    if (c < n) {
      Ar[e] = (double)j.A[(int64_t)r * j.lda + c];
      Ai[e] = (double)j.A[(int64_t)r * j.lda + c + j.aplane];
    } else {
      Ar[e] = (c - n == r) ? 1.0 : 0.0;
      Ai[e] = 0.0;
    }
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      double best = -1;
      int bi = k;
      for (int r = k; r < n; ++r) {
        double m2 = Ar[r * w + k] * Ar[r * w + k] + Ai[r * w + k] * Ai[r * w + k];
        if (m2 > best) { best = m2; bi = r; }
      }
      piv = bi;
      if (!(best > 0) && status) atomicExch(status, (int32_t)DEV_ZERO_PIVOT);
    }
    __syncthreads();
    const int p = piv;
    if (p != k)
      for (int c = threadIdx.x; c < w; c += blockDim.x) {
        double t = Ar[k * w + c]; Ar[k * w + c] = Ar[p * w + c]; Ar[p * w + c] = t;
        t = Ai[k * w + c]; Ai[k * w + c] = Ai[p * w + c]; Ai[p * w + c] = t;
      }
    __syncthreads();
    double dr = Ar[k * w + k], di = Ai[k * w + k];
    double den = dr * dr + di * di;
    if (den == 0) { dr = 1; di = 0; den = 1; }
    const double ir = dr / den, ii = -di / den;
    __syncthreads();
    for (int c = threadIdx.x; c < w; c += blockDim.x) {
      double a = Ar[k * w + c], b = Ai[k * w + c];
      Ar[k * w + c] = a * ir - b * ii;
      Ai[k * w + c] = a * ii + b * ir;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * w; e += blockDim.x) {
      int r = e / w, c = e % w;
      if (r == k) continue;
      double fr = Ar[r * w + k], fi = Ai[r * w + k];
      if (c == k) continue;
      double a = Ar[k * w + c], b = Ai[k * w + c];
      Ar[e] -= fr * a - fi * b;
      Ai[e] -= fr * b + fi * a;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x)
      if (r != k) { Ar[r * w + k] = 0; Ai[r * w + k] = 0; }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int r = e / n, c = e % n;
    j.X[(int64_t)r * j.ldx + c] = (T)Ar[r * w + n + c];
    j.X[(int64_t)r * j.ldx + c + j.xplane] = (T)Ai[r * w + n + c];
  }
}

template <typename T>
int launch_small_inverse(const InvJob<T>* d_jobs, int njobs, int max_n, int32_t* status, cudaStream_t st) {
  if (njobs <= 0) return 0;
  size_t sm = sizeof(double) * 4 * (size_t)max_n * max_n;
  if (sm > 200 * 1024) return -1;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_small_inverse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  count_launches(1);
  k_small_inverse<T><<<njobs, 256, sm, st>>>(d_jobs, status);
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
    } else if (j.mode == 1) {
      const int64_t so = (int64_t)j.ridx[r] * j.sld + j.cidx[c], dof = (int64_t)r * j.dld + c;
      j.dst[dof] += j.alpha * j.src[so];
      j.dst[dof + j.dplane] += j.alpha * j.src[so + j.splane];
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
__global__ void __launch_bounds__(256) k_lstsq(const LstsqJob<T>* jobs, int32_t* status) {
  const LstsqJob<T> j = jobs[blockIdx.x];
  const int c = j.c, r = j.r, w = j.w;
  extern __shared__ double lsq[];
  double* Gr = lsq;              // c x c, Hermitian, then its Cholesky factor (lower)
  double* Gi = Gr + c * c;
  double* zr = Gi + c * c;       // per-thread-block solve vector
  double* zi = zr + c;
  const T* Tr = j.Tm;
  const T* Ti = j.Tm + j.tplane;
  // G = Tm Tm^H
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
    int a = e / c, b = e % c;
    if (b > a) continue;
    double sr = 0, si = 0;
    for (int t = 0; t < w; ++t) {
      double ar = Tr[(int64_t)a * j.tld + t], ai = Ti[(int64_t)a * j.tld + t];
      double br = Tr[(int64_t)b * j.tld + t], bi = Ti[(int64_t)b * j.tld + t];
      sr += ar * br + ai * bi;      // a * conj(b)
      si += ai * br - ar * bi;
    }
    Gr[a * c + b] = sr; Gi[a * c + b] = si;
    Gr[b * c + a] = sr; Gi[b * c + a] = -si;
  }
  __syncthreads();
  // Cholesky G = L L^H (in place, lower), by one thread per column step
  for (int k = 0; k < c; ++k) {
    if (threadIdx.x == 0) {
      double d = Gr[k * c + k];
      if (!(d > 0)) {
        if (status) atomicExch(status, (int32_t)DEV_ZERO_PIVOT);
        d = 1e-300;
      }
      Gr[k * c + k] = sqrt(d);
      Gi[k * c + k] = 0;
    }
    __syncthreads();
    const double dk = Gr[k * c + k];
    for (int i = k + 1 + threadIdx.x; i < c; i += blockDim.x) {
      Gr[i * c + k] /= dk;
      Gi[i * c + k] /= dk;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < (c - k - 1) * (c - k - 1); e += blockDim.x) {
      int i = k + 1 + e / (c - k - 1), l = k + 1 + e % (c - k - 1);
      if (l > i) continue;
      // G[i][l] -= L[i][k] conj(L[l][k])
      double ar = Gr[i * c + k], ai = Gi[i * c + k], br = Gr[l * c + k], bi = Gi[l * c + k];
      Gr[i * c + l] -= ar * br + ai * bi;
      Gi[i * c + l] -= ai * br - ar * bi;
    }
    __syncthreads();
  }
  // rows of B: b_i = h_i G^-1, h_i = y_i Tm^H ; solve G b_i^H = h_i^H
  const T* Yr = j.Y;
  const T* Yi = j.Y + j.yplane;
  for (int i = 0; i < r; ++i) {
    for (int a = threadIdx.x; a < c; a += blockDim.x) {
      double sr = 0, si = 0;   // h_i[a] = sum_t y[t] conj(T[a][t]) ; store conj -> h^H
      for (int t = 0; t < w; ++t) {
        double yr = Yr[(int64_t)i * j.yld + t], yi = Yi[(int64_t)i * j.yld + t];
        double tr = Tr[(int64_t)a * j.tld + t], ti = Ti[(int64_t)a * j.tld + t];
        sr += yr * tr + yi * ti;
        si += yi * tr - yr * ti;
      }
      zr[a] = sr;
      zi[a] = -si;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int a = 0; a < c; ++a) {          // L z = h^H
        double vr = zr[a], vi = zi[a];
        for (int b = 0; b < a; ++b) {
          double lr = Gr[a * c + b], li = Gi[a * c + b];
          vr -= lr * zr[b] - li * zi[b];
          vi -= lr * zi[b] + li * zr[b];
        }
        zr[a] = vr / Gr[a * c + a];
        zi[a] = vi / Gr[a * c + a];
      }
      for (int a = c - 1; a >= 0; --a) {     // L^H x = z
        double vr = zr[a], vi = zi[a];
        for (int b = a + 1; b < c; ++b) {
          double lr = Gr[b * c + a], li = -Gi[b * c + a];
          vr -= lr * zr[b] - li * zi[b];
          vi -= lr * zi[b] + li * zr[b];
        }
        zr[a] = vr / Gr[a * c + a];
        zi[a] = vi / Gr[a * c + a];
      }
    }
    __syncthreads();
    for (int a = threadIdx.x; a < c; a += blockDim.x) {
      j.B[(int64_t)i * j.bld + a] = (T)zr[a];
      j.B[(int64_t)i * j.bld + a + j.bplane] = (T)(-zi[a]);
    }
    __syncthreads();
  }
}

template <typename T>
int launch_lstsq(const LstsqJob<T>* d_jobs, int njobs, int max_c, int32_t* status, cudaStream_t st) {
  if (njobs <= 0) return 0;
  size_t sm = sizeof(double) * (2 * (size_t)max_c * max_c + 2 * (size_t)max_c);
  if (sm > 200 * 1024) return -1;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_lstsq<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  count_launches(1);
  k_lstsq<T><<<njobs, 256, sm, st>>>(d_jobs, status);
  return 0;
}

#define MF_BF_INST(T)                                                                                            \
  template int launch_row_id<T>(const IdJob<T>*, int, int, int, T, int, cudaStream_t);                          \
  template void launch_sketch<T>(const SketchGroup*, int, int, T*, int64_t, int, cudaStream_t);                 \
  template void launch_gather_rows<T>(const GatherJob<T>*, int, int64_t, cudaStream_t);                         \
  template void launch_front_entries<T>(const FrontEntryJob<T>*, int, int64_t, const FrontCtx<T>*, const int64_t*, \
                                        const int32_t*, const double*, cudaStream_t);                           \
  template void launch_place<T>(const PlaceJob<T>*, int, int64_t, cudaStream_t);                                \
  template int launch_small_inverse<T>(const InvJob<T>*, int, int, int32_t*, cudaStream_t);                     \
  template void launch_blk2<T>(const Blk2Job<T>*, int, int64_t, cudaStream_t);                                   \
  template int launch_lstsq<T>(const LstsqJob<T>*, int, int, int32_t*, cudaStream_t);

MF_BF_INST(float)
MF_BF_INST(double)

}  // namespace mf
