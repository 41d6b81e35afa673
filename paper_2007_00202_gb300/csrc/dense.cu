// CUDA kernels of the dense multifrontal path (Alg. 1; Sec. 2 steps 1-4) and
// of the FP64 Krylov refinement (Sec. 6: GMRES(30) preconditioned by the
// factorization).  Planar complex storage; T = float (mixed path) or double.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "kernels.h"

namespace mf {

static std::atomic<int64_t> g_launches{0};
int64_t launch_count() { return g_launches.load(); }

namespace {
std::atomic<long long> g_wait_limit{kDefaultWaitLimit};
}
void set_wait_limit(long long spins) { g_wait_limit.store(spins > 0 ? spins : kDefaultWaitLimit); }
long long wait_limit() { return g_wait_limit.load(); }
void count_launches(int k) { g_launches += k; }

// ---------------------------------------------------------------------------
// Batched SIMT complex GEMM, 64 x 64 tiles, BK = 16, 256 threads (4 x 4 per thread).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_gemm(const GemmDesc<T>* __restrict__ descs,
                                              const GemmTile* __restrict__ tiles) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ T As[2][BK][BM + 1];
  __shared__ T Bs[2][BK][BN + 1];
  const GemmTile t = tiles[blockIdx.x];
  const GemmDesc<T> d = descs[t.desc];
  const int m0 = t.tm * BM, n0 = t.tn * BN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T cr[4][4], ci[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) cr[i][j] = ci[i][j] = T(0);
  const T* Ar = d.A.re;
  const T* Ai = d.A.re + d.A.plane;
  const T* Br = d.B.re;
  const T* Bi = d.B.re + d.B.plane;
  // the next k tile is read into registers while the current one is multiplied
  T par[4], pai[4], pbr[4], pbi[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = tid + e * 256;
      int mm, kk;
      if (d.transA == 0) { mm = idx / BK; kk = idx % BK; }
      else { kk = idx / BM; mm = idx % BM; }
      int gm = m0 + mm, gk = k0 + kk;
      par[e] = pai[e] = T(0);
      if (gm < d.m && gk < d.k) {
        const int64_t off = d.transA == 0 ? (int64_t)gm * d.A.ld + gk : (int64_t)gk * d.A.ld + gm;
        par[e] = Ar[off];
        pai[e] = Ai[off];
      }
      int nn;
      if (d.transB == 0) { kk = idx / BN; nn = idx % BN; }
      else { nn = idx / BK; kk = idx % BK; }
      const int gn = n0 + nn;
      gk = k0 + kk;
      pbr[e] = pbi[e] = T(0);
      if (gn < d.n && gk < d.k) {
        const int64_t off = d.transB == 0 ? (int64_t)gk * d.B.ld + gn : (int64_t)gn * d.B.ld + gk;
        pbr[e] = Br[off];
        pbi[e] = Bi[off];
      }
    }
  };
  if (d.k > 0) load(0);
  for (int k0 = 0; k0 < d.k; k0 += BK) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = tid + e * 256;
      int mm, kk;
      if (d.transA == 0) { mm = idx / BK; kk = idx % BK; }
      else { kk = idx / BM; mm = idx % BM; }
      As[0][kk][mm] = par[e];
      As[1][kk][mm] = pai[e];
      int nn;
      if (d.transB == 0) { kk = idx / BN; nn = idx % BN; }
      else { nn = idx / BK; kk = idx % BK; }
      Bs[0][kk][nn] = pbr[e];
      Bs[1][kk][nn] = pbi[e];
    }
    __syncthreads();
    if (k0 + BK < d.k) load(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T ar[4], ai[4], br[4], bi[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { ar[i] = As[0][kk][ty + 16 * i]; ai[i] = As[1][kk][ty + 16 * i]; }
#pragma unroll
      for (int j = 0; j < 4; ++j) { br[j] = Bs[0][kk][tx + 16 * j]; bi[j] = Bs[1][kk][tx + 16 * j]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          cr[i][j] = fma(ar[i], br[j], cr[i][j]);
          cr[i][j] = fma(-ai[i], bi[j], cr[i][j]);
          ci[i][j] = fma(ar[i], bi[j], ci[i][j]);
          ci[i][j] = fma(ai[i], br[j], ci[i][j]);
        }
    }
    __syncthreads();
  }
  T* Cr = d.C.re;
  T* Ci = d.C.re + d.C.plane;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty + 16 * i;
    if (gm >= d.m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx + 16 * j;
      if (gn >= d.n) continue;
      int64_t off = (int64_t)gm * d.C.ld + gn;
      T vr = d.alpha * cr[i][j], vi = d.alpha * ci[i][j];
      if (d.beta != T(0)) { vr += d.beta * Cr[off]; vi += d.beta * Ci[off]; }
      Cr[off] = vr;
      Ci[off] = vi;
    }
  }
}

template <typename T>
void launch_gemm(const GemmDesc<T>* d_desc, const GemmTile* d_tiles, int ntiles, cudaStream_t st) {
  if (ntiles <= 0) return;
  g_launches++;
  k_gemm<T><<<ntiles, 256, 0, st>>>(d_desc, d_tiles);
}

// ---------------------------------------------------------------------------
// Assembly of A's entries into F11, F12^T and F21 (Sec. 2 step 1).  One thread per front row.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t find_sorted(const int64_t* a, int64_t n, int64_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return (lo < n && a[lo] == key) ? lo : -1;
}

template <typename T>
__global__ void k_assemble_A(FrontDev<T>* fronts, const int32_t* flist, const int64_t* rowptr, const int64_t* colind,
                             const double* vals) {
  const FrontDev<T> f = fronts[flist[blockIdx.y]];
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= f.s + f.u) return;
  const int64_t sb = f.sep_begin, se = f.sep_begin + f.s;
  int64_t g = r < f.s ? sb + r : f.upd[r - f.s];
  for (int64_t k = rowptr[g]; k < rowptr[g + 1]; ++k) {
    int64_t c = colind[k];
    T vr = (T)vals[2 * k], vi = (T)vals[2 * k + 1];
    if (r < f.s) {
      if (c >= sb && c < se) {
        int64_t off = (int64_t)r * f.ls + (c - sb);
        f.LU[off] = vr;
        f.LU[off + f.pl_ss] = vi;
      } else if (c >= se) {
        int64_t p = find_sorted(f.upd, f.u, c);
        if (p >= 0) {
          int64_t off = p * f.ls + r;
          f.F12w[off] = vr;
          f.F12w[off + f.pl_us] = vi;
        }
      }
    } else if (c >= sb && c < se) {
      int64_t off = (int64_t)(r - f.s) * f.ls + (c - sb);
      f.F21w[off] = vr;
      f.F21w[off + f.pl_us] = vi;
    }
  }
}

template <typename T>
void launch_assemble_A(FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int maxrows, const int64_t* rowptr,
                       const int64_t* colind, const double* vals, cudaStream_t st) {
  if (nf <= 0 || maxrows <= 0) return;
  dim3 grid((maxrows + 127) / 128, nf);
  g_launches++;
  k_assemble_A<T><<<grid, 128, 0, st>>>(d_fronts, d_flist, rowptr, colind, vals);
}

// ---------------------------------------------------------------------------
// Extend-add (Sec. 2 step 1): F_parent[rel(i), rel(j)] += C_child[i, j].
// One CTA per EA_TI x EA_TJ tile of a child's block: the tile's rows are read with
// 16-byte loads (when the block's rows and planes are 16-byte aligned) into shared memory,
// then scattered.  F11, F21 and C parts of the parent are row-major in the parent's column
// index, so those entries are written with lanes along the child's columns; the F12 part is
// stored transposed (row = update position), so its entries are written with lanes along the
// child's rows, which keeps consecutive lanes on consecutive addresses in both cases.  The
// two children of a front run as separate launches, so no entry is updated twice at once.
// ---------------------------------------------------------------------------
constexpr int EA_TI = 32, EA_TJ = 64;

template <typename T>
__global__ void __launch_bounds__(256) k_extend_add(const ExtendAddItem<T>* items, const FrontDev<T>* fronts,
                                                    int tiles_j) {
  const ExtendAddItem<T> it = items[blockIdx.y];
  const int ti = blockIdx.x / tiles_j, tj = blockIdx.x % tiles_j;
  const int i0 = ti * EA_TI, j0 = tj * EA_TJ;
  if (i0 >= it.uc || j0 >= it.uc) return;
  const FrontDev<T> f = fronts[it.parent];
  __shared__ T sr[EA_TI][EA_TJ + 1], si[EA_TI][EA_TJ + 1];
  __shared__ int32_t rr[EA_TI], rc[EA_TJ];
  const int tid = threadIdx.x;
  const int ni = min(EA_TI, it.uc - i0), nj = min(EA_TJ, it.uc - j0);
  if (tid < EA_TI) rr[tid] = tid < ni ? it.rel[i0 + tid] : 0;
  if (tid < EA_TJ) rc[tid] = tid < nj ? it.rel[j0 + tid] : 0;
  constexpr int V = 16 / (int)sizeof(T);
  const bool vec = ((reinterpret_cast<uintptr_t>(it.Cc) | ((uintptr_t)it.ldc * sizeof(T)) |
                     ((uintptr_t)it.plane_c * sizeof(T))) & 15) == 0;
  const T* cr = it.Cc + (int64_t)i0 * it.ldc + j0;
  const T* ci = cr + it.plane_c;
  if (vec && nj == EA_TJ) {
    constexpr int CH = EA_TI * EA_TJ / V;   // 16-byte chunks per plane
    for (int c = tid; c < 2 * CH; c += 256) {
      const int pl = c / CH, cc = c % CH, i = cc / (EA_TJ / V), jv = (cc % (EA_TJ / V)) * V;
      if (i < ni) {
        const T* src = (pl ? ci : cr) + (int64_t)i * it.ldc + jv;
        T buf[V];
        *reinterpret_cast<uint4*>(buf) = *reinterpret_cast<const uint4*>(src);
#pragma unroll
        for (int e = 0; e < V; ++e) (pl ? si : sr)[i][jv + e] = buf[e];
      }
    }
  } else {
    for (int e = tid; e < EA_TI * EA_TJ; e += 256) {
      const int i = e / EA_TJ, j = e % EA_TJ;
      if (i < ni && j < nj) {
        sr[i][j] = cr[(int64_t)i * it.ldc + j];
        si[i][j] = ci[(int64_t)i * it.ldc + j];
      }
    }
  }
  __syncthreads();
  const int s = f.s;
  // Every parent entry of the tile is distinct (rel is injective), so each thread first gathers
  // all the parent values it updates, then adds and stores them: the loads of a pass are in
  // flight together instead of one read-modify-write round trip at a time.
  constexpr int PER = EA_TI * EA_TJ / 256;   // 8 entries per thread and pass
  // pass 1, the F11, F21 and C parts: lanes along j
  {
    T* dp[PER];
    int64_t pl[PER];
    T ar[PER], ai[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = tid + 256 * q, i = e / EA_TJ, j = e % EA_TJ;
      dp[q] = nullptr;
      if (i >= ni || j >= nj) continue;
      const int ri = rr[i], rj = rc[j];
      if (ri < s) {
        if (rj >= s) continue;   // F12: pass 2
        dp[q] = f.LU + (int64_t)ri * f.ls + rj; pl[q] = f.pl_ss;
      } else if (rj < s) {
        dp[q] = f.F21w + (int64_t)(ri - s) * f.ls + rj; pl[q] = f.pl_us;
      } else {
        dp[q] = f.C + (int64_t)(ri - s) * f.lu + (rj - s); pl[q] = f.pl_uu;
      }
    }
#pragma unroll
    for (int q = 0; q < PER; ++q)
      if (dp[q]) {
        ar[q] = dp[q][0];
        ai[q] = dp[q][pl[q]];
      }
#pragma unroll
    for (int q = 0; q < PER; ++q)
      if (dp[q]) {
        const int e = tid + 256 * q, i = e / EA_TJ, j = e % EA_TJ;
        dp[q][0] = ar[q] + sr[i][j];
        dp[q][pl[q]] = ai[q] + si[i][j];
      }
  }
  // pass 2, the F12 part (stored transposed, u x s): lanes along i
  {
    T* dp[PER];
    T ar[PER], ai[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = tid + 256 * q, j = e / EA_TI, i = e % EA_TI;
      dp[q] = nullptr;
      if (i >= ni || j >= nj) continue;
      const int ri = rr[i], rj = rc[j];
      if (ri >= s || rj < s) continue;
      dp[q] = f.F12w + (int64_t)(rj - s) * f.ls + ri;
    }
#pragma unroll
    for (int q = 0; q < PER; ++q)
      if (dp[q]) {
        ar[q] = dp[q][0];
        ai[q] = dp[q][f.pl_us];
      }
#pragma unroll
    for (int q = 0; q < PER; ++q)
      if (dp[q]) {
        const int e = tid + 256 * q, j = e / EA_TI, i = e % EA_TI;
        dp[q][0] = ar[q] + sr[i][j];
        dp[q][f.pl_us] = ai[q] + si[i][j];
      }
  }
}

template <typename T>
void launch_extend_add(const ExtendAddItem<T>* d_items, int nitems, const FrontDev<T>* d_fronts, int max_uc,
                       cudaStream_t st) {
  if (nitems <= 0 || max_uc <= 0) return;
  const int tiles_i = (max_uc + EA_TI - 1) / EA_TI, tiles_j = (max_uc + EA_TJ - 1) / EA_TJ;
  dim3 grid(tiles_i * tiles_j, nitems);
  g_launches++;
  k_extend_add<T><<<grid, 256, 0, st>>>(d_items, d_fronts, tiles_j);
}

// ---------------------------------------------------------------------------
// Panel LU with partial pivoting inside F11 (Sec. 2 step 2; pivot search does
// not look at F12/F21).  Pivot: largest modulus, lowest row on ties.
// The panel (rows kb..s-1, columns kb..kb+w-1) is factored in shared memory
// when it fits (cap_rows), with the pivots' row swaps applied to the columns
// outside the panel afterwards; taller panels are factored in place in global
// memory (L2-resident for the front sizes of the dense path).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(512) k_panel_lu(FrontDev<T>* fronts, const int32_t* flist, int kb, int nb,
                                                  int cap_rows, int32_t* status) {
  FrontDev<T> f = fronts[flist[blockIdx.x]];
  const int s = f.s;
  const int ld = f.ls;
  if (kb >= s) return;
  const int w = min(nb, s - kb);
  const int rows = s - kb;
  T* Ar = f.LU;
  T* Ai = f.LU + f.pl_ss;
  __shared__ T redv[32];
  __shared__ int redi[32];
  __shared__ int piv_sh;
  __shared__ T best_sh;
  extern __shared__ unsigned char pan_raw[];
  const int tid = threadIdx.x, nt = blockDim.x;
  const bool in_smem = rows <= cap_rows;
  // panel element accessors (row q = 0..rows-1 is global row kb + q, column c = 0..w-1)
  T* Pr = reinterpret_cast<T*>(pan_raw);
  T* Pi = Pr + (size_t)cap_rows * nb;
  auto pr = [&](int q, int c) -> T& { return in_smem ? Pr[q * nb + c] : Ar[(int64_t)(kb + q) * ld + kb + c]; };
  auto pi = [&](int q, int c) -> T& { return in_smem ? Pi[q * nb + c] : Ai[(int64_t)(kb + q) * ld + kb + c]; };
  if (in_smem) {
    for (int e = tid; e < rows * w; e += nt) {
      int q = e / w, c = e % w;
      Pr[q * nb + c] = Ar[(int64_t)(kb + q) * ld + kb + c];
      Pi[q * nb + c] = Ai[(int64_t)(kb + q) * ld + kb + c];
    }
    __syncthreads();
  }
  for (int jj = 0; jj < w; ++jj) {
    T best = T(-1);
    int bi = rows;
    for (int q = jj + tid; q < rows; q += nt) {
      T a = pr(q, jj), b = pi(q, jj);
      T m2 = a * a + b * b;
      if (m2 > best) { best = m2; bi = q; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      T ob = __shfl_down_sync(0xffffffffu, best, o);
      int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if ((tid & 31) == 0) { redv[tid >> 5] = best; redi[tid >> 5] = bi; }
    __syncthreads();
    if (tid < 32) {
      int nw = nt >> 5;
      best = tid < nw ? redv[tid] : T(-1);
      bi = tid < nw ? redi[tid] : rows;
      for (int o = 16; o > 0; o >>= 1) {
        T ob = __shfl_down_sync(0xffffffffu, best, o);
        int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        piv_sh = bi < rows ? bi : jj;
        best_sh = best;
        f.piv[kb + jj] = kb + piv_sh;
        if (!(best > T(0)) && status) atomicExch(status, (int32_t)DEV_ZERO_PIVOT);
      }
    }
    __syncthreads();
    const int p = piv_sh;
    if (p != jj) {
      if (in_smem) {
        for (int c = tid; c < w; c += nt) {
          T t0 = Pr[jj * nb + c]; Pr[jj * nb + c] = Pr[p * nb + c]; Pr[p * nb + c] = t0;
          t0 = Pi[jj * nb + c]; Pi[jj * nb + c] = Pi[p * nb + c]; Pi[p * nb + c] = t0;
        }
      } else {
        for (int c = tid; c < s; c += nt) {
          int64_t o1 = (int64_t)(kb + jj) * ld + c, o2 = (int64_t)(kb + p) * ld + c;
          T t0 = Ar[o1]; Ar[o1] = Ar[o2]; Ar[o2] = t0;
          t0 = Ai[o1]; Ai[o1] = Ai[o2]; Ai[o2] = t0;
        }
      }
    }
    __syncthreads();
    T dr = pr(jj, jj), di = pi(jj, jj);
    T den = dr * dr + di * di;
    if (den == T(0)) { dr = T(1); di = T(0); den = T(1); }
    const T invr = dr / den, invi = -di / den;
    for (int q = jj + 1 + tid; q < rows; q += nt) {
      T ar = pr(q, jj), ai = pi(q, jj);
      T lr = ar * invr - ai * invi, li = ar * invi + ai * invr;
      pr(q, jj) = lr;
      pi(q, jj) = li;
      for (int c = jj + 1; c < w; ++c) {
        T ur = pr(jj, c), ui = pi(jj, c);
        pr(q, c) -= lr * ur - li * ui;
        pi(q, c) -= lr * ui + li * ur;
      }
    }
    __syncthreads();
  }
  if (in_smem) {
    for (int e = tid; e < rows * w; e += nt) {
      int q = e / w, c = e % w;
      Ar[(int64_t)(kb + q) * ld + kb + c] = Pr[q * nb + c];
      Ai[(int64_t)(kb + q) * ld + kb + c] = Pi[q * nb + c];
    }
    // the panel's row swaps on the columns outside the panel, in pivot order
    for (int c = tid; c < s; c += nt) {
      if (c >= kb && c < kb + w) continue;
      for (int jj = 0; jj < w; ++jj) {
        int p = f.piv[kb + jj];
        if (p != kb + jj) {
          int64_t o1 = (int64_t)(kb + jj) * ld + c, o2 = (int64_t)p * ld + c;
          T t0 = Ar[o1]; Ar[o1] = Ar[o2]; Ar[o2] = t0;
          t0 = Ai[o1]; Ai[o1] = Ai[o2]; Ai[o2] = t0;
        }
      }
    }
  }
}

template <typename T>
void launch_panel_lu(FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int kb, int nb, int max_rows,
                     int32_t* status, cudaStream_t st) {
  if (nf <= 0) return;
  constexpr size_t budget = 192 * 1024;
  int cap = (int)(budget / (2 * sizeof(T) * (size_t)nb));
  if (max_rows < cap) cap = max_rows;
  size_t sm = 2 * sizeof(T) * (size_t)nb * cap;
  static PerDeviceOnce attr;
  attr([] { cudaFuncSetAttribute(k_panel_lu<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget); });
  g_launches++;
  k_panel_lu<T><<<nf, 512, sm, st>>>(d_fronts, d_flist, kb, nb, cap, status);
}

// U12 <- L11^-1 A12 for the panel rows [kb, kb+w) and columns [kb+w, s).
template <typename T>
__global__ void k_panel_trsm(FrontDev<T>* fronts, const int32_t* flist, int kb, int nb) {
  FrontDev<T> f = fronts[flist[blockIdx.y]];
  const int s = f.s;
  const int ld = f.ls;
  if (kb >= s) return;
  const int w = min(nb, s - kb);
  __shared__ T Lr[64][65], Li[64][65];
  T* Ar = f.LU;
  T* Ai = f.LU + f.pl_ss;
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
    int r = e / w, c = e % w;
    Lr[r][c] = Ar[(int64_t)(kb + r) * ld + kb + c];
    Li[r][c] = Ai[(int64_t)(kb + r) * ld + kb + c];
  }
  __syncthreads();
  int col = kb + w + blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= s) return;
  T xr[64], xi[64];
#pragma unroll 1
  for (int r = 0; r < w; ++r) {
    T vr = Ar[(int64_t)(kb + r) * ld + col], vi = Ai[(int64_t)(kb + r) * ld + col];
    for (int t = 0; t < r; ++t) {
      vr -= Lr[r][t] * xr[t] - Li[r][t] * xi[t];
      vi -= Lr[r][t] * xi[t] + Li[r][t] * xr[t];
    }
    xr[r] = vr;
    xi[r] = vi;
    Ar[(int64_t)(kb + r) * ld + col] = vr;
    Ai[(int64_t)(kb + r) * ld + col] = vi;
  }
}

template <typename T>
void launch_panel_trsm(FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int kb, int nb, int max_s,
                       cudaStream_t st) {
  if (nf <= 0 || max_s - kb - 1 <= 0) return;
  dim3 grid((max_s + 127) / 128, nf);
  g_launches++;
  k_panel_trsm<T><<<grid, 128, 0, st>>>(d_fronts, d_flist, kb, nb);
}

// ---------------------------------------------------------------------------
// After the LU: U^T, gather permutation, pivots applied to F12^T.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_transpose_U(FrontDev<T>* fronts, const int32_t* flist) {
  FrontDev<T> f = fronts[flist[blockIdx.z]];
  const int s = f.s;
  const int ld = f.ls;
  __shared__ T tr[32][33], ti[32][33];
  int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  if (r0 >= s || c0 >= s) return;
  int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    int r = r0 + k, c = c0 + tx;
    T vr = T(0), vi = T(0);
    if (r < s && c < s && c >= r) {
      vr = f.LU[(int64_t)r * ld + c];
      vi = f.LU[(int64_t)r * ld + c + f.pl_ss];
    }
    tr[k][tx] = vr;
    ti[k][tx] = vi;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    int r = c0 + k, c = r0 + tx;   // UT[r][c] = U[c][r]
    if (r < s && c < s) {
      f.UT[(int64_t)r * ld + c] = tr[tx][k];
      f.UT[(int64_t)r * ld + c + f.pl_ss] = ti[tx][k];
    }
  }
}

template <typename T>
__global__ void k_piv_to_perm(FrontDev<T>* fronts, const int32_t* flist, int nf) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nf) return;
  FrontDev<T> f = fronts[flist[q]];
  for (int k = 0; k < f.s; ++k) f.perm[k] = k;
  for (int k = 0; k < f.s; ++k) {
    int p = f.piv[k];
    int t = f.perm[k]; f.perm[k] = f.perm[p]; f.perm[p] = t;
  }
}

template <typename T>
__global__ void k_permute_F12(FrontDev<T>* fronts, const int32_t* flist) {
  FrontDev<T> f = fronts[flist[blockIdx.y]];
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)f.u * f.s) return;
  int64_t j = e / f.s, k = e % f.s;
  int64_t dst = j * f.ls + k;
  int64_t src = j * f.ls + f.perm[k];
  f.F12p[dst] = f.F12w[src];
  f.F12p[dst + f.pl_us] = f.F12w[src + f.pl_us];
}

template <typename T>
void launch_post_lu(FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int max_s, int max_u, cudaStream_t st) {
  if (nf <= 0) return;
  dim3 g1((max_s + 31) / 32, (max_s + 31) / 32, nf);
  g_launches++;
  k_transpose_U<T><<<g1, dim3(32, 8), 0, st>>>(d_fronts, d_flist);
  g_launches++;
  k_piv_to_perm<T><<<(nf + 127) / 128, 128, 0, st>>>(d_fronts, d_flist, nf);
  int64_t mx = (int64_t)max_s * max_u;
  if (mx > 0) {
    dim3 g2((unsigned)((mx + 255) / 256), nf);
    g_launches++;
    k_permute_F12<T><<<g2, 256, 0, st>>>(d_fronts, d_flist);
  }
}

// ---------------------------------------------------------------------------
// Inverses of the 64 x 64 diagonal blocks of a lower triangular matrix.
// which = 0: T = unit lower part of LU -> Linv; which = 1: T = UT -> UinvT.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_trinv_diag(FrontDev<T>* fronts, const int32_t* flist, int which) {
  FrontDev<T> f = fronts[flist[blockIdx.y]];
  const int s = f.s;
  const int ld = f.ls;
  const int b0 = blockIdx.x * 64;
  if (b0 >= s) return;
  const int w = min(64, s - b0);
  extern __shared__ unsigned char smem_raw[];
  T* Tr = reinterpret_cast<T*>(smem_raw);      // 64 x 65
  T* Ti = Tr + 64 * 65;
  T* Xr = Ti + 64 * 65;
  T* Xi = Xr + 64 * 65;
  const T* src = which == 0 ? f.LU : f.UT;
  T* dst = which == 0 ? f.Linv : f.UinvT;
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
    int r = e / w, c = e % w;
    T vr = T(0), vi = T(0);
    if (c < r || (c == r && which == 1)) {
      vr = src[(int64_t)(b0 + r) * ld + b0 + c];
      vi = src[(int64_t)(b0 + r) * ld + b0 + c + f.pl_ss];
    } else if (c == r) {
      vr = T(1);
    }
    Tr[r * 65 + c] = vr;
    Ti[r * 65 + c] = vi;
  }
  __syncthreads();
  const int c = threadIdx.x;
  if (c < w) {
    // column c of the inverse: forward substitution on e_c
    for (int r = 0; r < c; ++r) { Xr[r * 65 + c] = T(0); Xi[r * 65 + c] = T(0); }
    for (int r = c; r < w; ++r) {
      T vr = (r == c) ? T(1) : T(0), vi = T(0);
      for (int t = c; t < r; ++t) {
        T ar = Tr[r * 65 + t], ai = Ti[r * 65 + t];
        T xr = Xr[t * 65 + c], xi = Xi[t * 65 + c];
        vr -= ar * xr - ai * xi;
        vi -= ar * xi + ai * xr;
      }
      T dr = Tr[r * 65 + r], di = Ti[r * 65 + r];
      T den = dr * dr + di * di;
      if (den == T(0)) den = T(1);
      Xr[r * 65 + c] = (vr * dr + vi * di) / den;
      Xi[r * 65 + c] = (vi * dr - vr * di) / den;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
    int r = e / w, cc = e % w;
    dst[(int64_t)(b0 + r) * ld + b0 + cc] = Xr[r * 65 + cc];
    dst[(int64_t)(b0 + r) * ld + b0 + cc + f.pl_ss] = Xi[r * 65 + cc];
  }
}

template <typename T>
void launch_trinv_diag(FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int max_s, int which, T* const*,
                       cudaStream_t st) {
  if (nf <= 0) return;
  size_t sm = 4 * 64 * 65 * sizeof(T);
  static PerDeviceOnce attr;
  attr([sm] { cudaFuncSetAttribute(k_trinv_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); });
  dim3 grid((max_s + 63) / 64, nf);
  g_launches++;
  k_trinv_diag<T><<<grid, 64, sm, st>>>(d_fronts, d_flist, which);
}

// ---------------------------------------------------------------------------
// Right-hand-side movement for the solve (row-major N x nrhs planar vectors).
// ---------------------------------------------------------------------------
// tmp[k][c] = X[sep_begin + perm[k]][c]   (P^T b_s)
template <typename T>
__global__ void k_fwd_gather(const FrontDev<T>* fronts, const int32_t* flist, const T* X, int64_t xpl, int nrhs,
                             T* const* tmp) {
  const FrontDev<T> f = fronts[flist[blockIdx.y]];
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= f.s * nrhs) return;
  int k = e / nrhs, c = e % nrhs;
  T* d = tmp[blockIdx.y];
  int64_t src = (f.sep_begin + f.perm[k]) * nrhs + c;
  int64_t tpl = (int64_t)f.s * nrhs;
  d[e] = X[src];
  d[e + tpl] = X[src + xpl];
}

template <typename T>
__global__ void k_scatter_sep(const FrontDev<T>* fronts, const int32_t* flist, T* X, int64_t xpl, int nrhs,
                              T* const* srcs) {
  const FrontDev<T> f = fronts[flist[blockIdx.y]];
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= f.s * nrhs) return;
  const T* s = srcs[blockIdx.y];
  int64_t tpl = (int64_t)f.s * nrhs;
  int64_t dst = f.sep_begin * nrhs + e;
  X[dst] = s[e];
  X[dst + xpl] = s[e + tpl];
}

template <typename T>
__global__ void k_gather_sep(const FrontDev<T>* fronts, const int32_t* flist, const T* X, int64_t xpl, int nrhs,
                             T* const* dsts) {
  const FrontDev<T> f = fronts[flist[blockIdx.y]];
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= f.s * nrhs) return;
  T* d = dsts[blockIdx.y];
  int64_t tpl = (int64_t)f.s * nrhs;
  int64_t src = f.sep_begin * nrhs + e;
  d[e] = X[src];
  d[e + tpl] = X[src + xpl];
}

template <typename T>
__global__ void k_scatter_add_upd(const FrontDev<T>* fronts, const int32_t* flist, T* X, int64_t xpl, int nrhs,
                                  T* const* srcs) {
  const FrontDev<T> f = fronts[flist[blockIdx.y]];
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= f.u * nrhs) return;
  int j = e / nrhs, c = e % nrhs;
  const T* s = srcs[blockIdx.y];
  int64_t tpl = (int64_t)f.u * nrhs;
  int64_t dst = f.upd[j] * nrhs + c;
  atomicAdd(&X[dst], s[e]);
  atomicAdd(&X[dst + xpl], s[e + tpl]);
}

template <typename T>
__global__ void k_gather_upd(const FrontDev<T>* fronts, const int32_t* flist, const T* X, int64_t xpl, int nrhs,
                             T* const* dsts) {
  const FrontDev<T> f = fronts[flist[blockIdx.y]];
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= f.u * nrhs) return;
  int j = e / nrhs, c = e % nrhs;
  T* d = dsts[blockIdx.y];
  int64_t tpl = (int64_t)f.u * nrhs;
  int64_t src = f.upd[j] * nrhs + c;
  d[e] = X[src];
  d[e + tpl] = X[src + xpl];
}

template <typename T>
void launch_fwd_gather(const FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int max_s, const T* X, int64_t xpl,
                       int nrhs, T* const* d_tmp, cudaStream_t st) {
  if (nf <= 0 || max_s <= 0) return;
  dim3 g((max_s * nrhs + 255) / 256, nf);
  g_launches++;
  k_fwd_gather<T><<<g, 256, 0, st>>>(d_fronts, d_flist, X, xpl, nrhs, d_tmp);
}
template <typename T>
void launch_scatter_sep(const FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int max_s, T* X, int64_t xpl,
                        int nrhs, T* const* d_src, cudaStream_t st) {
  if (nf <= 0 || max_s <= 0) return;
  dim3 g((max_s * nrhs + 255) / 256, nf);
  g_launches++;
  k_scatter_sep<T><<<g, 256, 0, st>>>(d_fronts, d_flist, X, xpl, nrhs, d_src);
}
template <typename T>
void launch_gather_sep(const FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int max_s, const T* X,
                       int64_t xpl, int nrhs, T* const* d_dst, cudaStream_t st) {
  if (nf <= 0 || max_s <= 0) return;
  dim3 g((max_s * nrhs + 255) / 256, nf);
  g_launches++;
  k_gather_sep<T><<<g, 256, 0, st>>>(d_fronts, d_flist, X, xpl, nrhs, d_dst);
}
template <typename T>
void launch_scatter_add_upd(const FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int max_u, T* X,
                            int64_t xpl, int nrhs, T* const* d_src, cudaStream_t st) {
  if (nf <= 0 || max_u <= 0) return;
  dim3 g((max_u * nrhs + 255) / 256, nf);
  g_launches++;
  k_scatter_add_upd<T><<<g, 256, 0, st>>>(d_fronts, d_flist, X, xpl, nrhs, d_src);
}
template <typename T>
void launch_gather_upd(const FrontDev<T>* d_fronts, const int32_t* d_flist, int nf, int max_u, const T* X,
                       int64_t xpl, int nrhs, T* const* d_dst, cudaStream_t st) {
  if (nf <= 0 || max_u <= 0) return;
  dim3 g((max_u * nrhs + 255) / 256, nf);
  g_launches++;
  k_gather_upd<T><<<g, 256, 0, st>>>(d_fronts, d_flist, X, xpl, nrhs, d_dst);
}

// ---------------------------------------------------------------------------
// Conversions: interleaved complex128 column-major (original numbering)
// <-> planar T row-major (new numbering).  perm[new] = old.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_to_planar(const double* src, int64_t ld, int64_t n, int nrhs, const int64_t* perm, T* dst,
                            int64_t pl, int pld) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * nrhs) return;
  int64_t i = e / nrhs;
  int c = (int)(e % nrhs);
  int64_t o = perm ? perm[i] : i;
  dst[i * pld + c] = (T)src[2 * (o + c * ld)];
  dst[i * pld + c + pl] = (T)src[2 * (o + c * ld) + 1];
}

template <typename T>
__global__ void k_from_planar(const T* src, int64_t pl, int64_t n, int nrhs, const int64_t* perm, double* dst,
                              int64_t ld, int pld) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * nrhs) return;
  int64_t i = e / nrhs;
  int c = (int)(e % nrhs);
  int64_t o = perm ? perm[i] : i;
  dst[2 * (o + c * ld)] = (double)src[i * pld + c];
  dst[2 * (o + c * ld) + 1] = (double)src[i * pld + c + pl];
}

template <typename T>
void launch_to_planar(const double* src, int64_t ld, int64_t n, int nrhs, const int64_t* perm, T* dst, int64_t pl,
                      cudaStream_t st, int pld) {
  if (pld <= 0) pld = nrhs;
  int64_t tot = n * nrhs;
  if (tot <= 0) return;
  g_launches++;
  k_to_planar<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(src, ld, n, nrhs, perm, dst, pl, pld);
}
template <typename T>
void launch_from_planar(const T* src, int64_t pl, int64_t n, int nrhs, const int64_t* perm, double* dst, int64_t ld,
                        cudaStream_t st, int pld) {
  if (pld <= 0) pld = nrhs;
  int64_t tot = n * nrhs;
  if (tot <= 0) return;
  g_launches++;
  k_from_planar<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(src, pl, n, nrhs, perm, dst, ld, pld);
}

// ---------------------------------------------------------------------------
// FP64 sparse products and Krylov vector operations (interleaved complex128).
// ---------------------------------------------------------------------------
__global__ void k_spmv(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* vals, const double* x,
                       const double* b, double* y, int nrhs, int64_t ld) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * nrhs) return;
  int64_t i = e % n;
  int c = (int)(e / n);
  const double* xc = x + 2 * c * ld;
  double ar = 0, ai = 0;
  for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
    double vr = vals[2 * k], vi = vals[2 * k + 1];
    int64_t j = colind[k];
    double xr = xc[2 * j], xi = xc[2 * j + 1];
    ar += vr * xr - vi * xi;
    ai += vr * xi + vi * xr;
  }
  double* yc = y + 2 * c * ld;
  if (b) {
    const double* bc = b + 2 * c * ld;
    yc[2 * i] = bc[2 * i] - ar;
    yc[2 * i + 1] = bc[2 * i + 1] - ai;
  } else {
    yc[2 * i] = ar;
    yc[2 * i + 1] = ai;
  }
}

void launch_spmv_residual(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* vals,
                          const double* x, const double* b, double* r, int nrhs, int64_t ld, cudaStream_t st) {
  int64_t tot = n * nrhs;
  g_launches++;
  k_spmv<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, rowptr, colind, vals, x, b, r, nrhs, ld);
}
void launch_spmv(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* vals, const double* x,
                 double* y, int nrhs, int64_t ld, cudaStream_t st) {
  int64_t tot = n * nrhs;
  g_launches++;
  k_spmv<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, rowptr, colind, vals, x, nullptr, y, nrhs, ld);
}

// per-column complex dot conj(V)^T W: grid (blocks, nrhs), atomics into out
__global__ void k_coldot(int64_t n, const double* V, int64_t ldv, const double* W, int64_t ldw, double* out) {
  int c = blockIdx.y;
  const double* v = V + 2 * c * ldv;
  const double* w = W + 2 * c * ldw;
  double sr = 0, si = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double vr = v[2 * i], vi = v[2 * i + 1], wr = w[2 * i], wi = w[2 * i + 1];
    sr += vr * wr + vi * wi;
    si += vr * wi - vi * wr;
  }
  __shared__ double rr[32], ri[32];
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, o);
    si += __shfl_down_sync(0xffffffffu, si, o);
  }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { rr[wid] = sr; ri[wid] = si; }
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    sr = lane < nw ? rr[lane] : 0;
    si = lane < nw ? ri[lane] : 0;
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_down_sync(0xffffffffu, sr, o);
      si += __shfl_down_sync(0xffffffffu, si, o);
    }
    if (lane == 0) {
      atomicAdd(&out[2 * c], sr);
      atomicAdd(&out[2 * c + 1], si);
    }
  }
}

void launch_coldot(int64_t n, int nrhs, const double* V, int64_t ldv, const double* W, int64_t ldw, double* out,
                   cudaStream_t st) {
  cudaMemsetAsync(out, 0, sizeof(double) * 2 * nrhs, st);
  int blocks = (int)((n + 255) / 256);
  if (blocks > 304) blocks = 304;
  g_launches++;
  k_coldot<<<dim3(blocks, nrhs), 256, 0, st>>>(n, V, ldv, W, ldw, out);
}

__global__ void k_colaxpy(int64_t n, const double* h, const double* V, int64_t ldv, double* W, int64_t ldw,
                          double sign) {
  int c = blockIdx.y;
  double hr = sign * h[2 * c], hi = sign * h[2 * c + 1];
  const double* v = V + 2 * c * ldv;
  double* w = W + 2 * c * ldw;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double vr = v[2 * i], vi = v[2 * i + 1];
    w[2 * i] -= hr * vr - hi * vi;
    w[2 * i + 1] -= hr * vi + hi * vr;
  }
}

void launch_colaxpy(int64_t n, int nrhs, const double* h, const double* V, int64_t ldv, double* W, int64_t ldw,
                    double sign, cudaStream_t st) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 1216) blocks = 1216;
  g_launches++;
  k_colaxpy<<<dim3(blocks, nrhs), 256, 0, st>>>(n, h, V, ldv, W, ldw, sign);
}

__global__ void k_colscale(int64_t n, const double* s, const double* X, int64_t ldx, double* Y, int64_t ldy) {
  int c = blockIdx.y;
  double sr = s[2 * c], si = s[2 * c + 1];
  const double* x = X + 2 * c * ldx;
  double* y = Y + 2 * c * ldy;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double xr = x[2 * i], xi = x[2 * i + 1];
    y[2 * i] = sr * xr - si * xi;
    y[2 * i + 1] = sr * xi + si * xr;
  }
}

void launch_colscale(int64_t n, int nrhs, const double* s, const double* X, int64_t ldx, double* Y, int64_t ldy,
                     cudaStream_t st) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 1216) blocks = 1216;
  g_launches++;
  k_colscale<<<dim3(blocks, nrhs), 256, 0, st>>>(n, s, X, ldx, Y, ldy);
}

__global__ void k_colnorm2(int64_t n, const double* X, int64_t ldx, double* out) {
  int c = blockIdx.y;
  const double* x = X + 2 * c * ldx;
  double s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += x[2 * i] * x[2 * i] + x[2 * i + 1] * x[2 * i + 1];
  __shared__ double r[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) r[wid] = s;
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    s = lane < nw ? r[lane] : 0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) atomicAdd(&out[c], s);
  }
}

void launch_colnorm2(int64_t n, int nrhs, const double* X, int64_t ldx, double* out, cudaStream_t st) {
  cudaMemsetAsync(out, 0, sizeof(double) * nrhs, st);
  int blocks = (int)((n + 255) / 256);
  if (blocks > 304) blocks = 304;
  g_launches++;
  k_colnorm2<<<dim3(blocks, nrhs), 256, 0, st>>>(n, X, ldx, out);
}

// ---------------------------------------------------------------------------
// explicit instantiations
// ---------------------------------------------------------------------------
#define MF_INST(T)                                                                                                  \
  template void launch_gemm<T>(const GemmDesc<T>*, const GemmTile*, int, cudaStream_t);                           \
  template void launch_assemble_A<T>(FrontDev<T>*, const int32_t*, int, int, const int64_t*, const int64_t*,     \
                                     const double*, cudaStream_t);                                               \
  template void launch_extend_add<T>(const ExtendAddItem<T>*, int, const FrontDev<T>*, int, cudaStream_t);        \
  template void launch_panel_lu<T>(FrontDev<T>*, const int32_t*, int, int, int, int, int32_t*, cudaStream_t);     \
  template void launch_panel_trsm<T>(FrontDev<T>*, const int32_t*, int, int, int, int, cudaStream_t);             \
  template void launch_post_lu<T>(FrontDev<T>*, const int32_t*, int, int, int, cudaStream_t);                     \
  template void launch_trinv_diag<T>(FrontDev<T>*, const int32_t*, int, int, int, T* const*, cudaStream_t);       \
  template void launch_fwd_gather<T>(const FrontDev<T>*, const int32_t*, int, int, const T*, int64_t, int,        \
                                     T* const*, cudaStream_t);                                                    \
  template void launch_scatter_sep<T>(const FrontDev<T>*, const int32_t*, int, int, T*, int64_t, int, T* const*,  \
                                      cudaStream_t);                                                              \
  template void launch_gather_sep<T>(const FrontDev<T>*, const int32_t*, int, int, const T*, int64_t, int,        \
                                     T* const*, cudaStream_t);                                                    \
  template void launch_scatter_add_upd<T>(const FrontDev<T>*, const int32_t*, int, int, T*, int64_t, int,         \
                                          T* const*, cudaStream_t);                                               \
  template void launch_gather_upd<T>(const FrontDev<T>*, const int32_t*, int, int, const T*, int64_t, int,        \
                                     T* const*, cudaStream_t);                                                    \
  template void launch_to_planar<T>(const double*, int64_t, int64_t, int, const int64_t*, T*, int64_t,            \
                                    cudaStream_t, int);                                                           \
  template void launch_from_planar<T>(const T*, int64_t, int64_t, int, const int64_t*, double*, int64_t,          \
                                      cudaStream_t, int);

MF_INST(float)
MF_INST(double)

}  // namespace mf
