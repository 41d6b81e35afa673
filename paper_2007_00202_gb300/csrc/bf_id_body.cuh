// Device bodies of the batched row interpolative decomposition (Sec. 3): row_id_body (one CTA
// per matrix, shared by the batched kernel and its fixed-scratch variant; dynamic shared memory
// of row_id_smem_bytes(m, n, work_in_smem): the QR work matrix (2 m n values) sits there too
// when work_in_smem, else in jb.work), row_id_body_reg (rows in registers, m, n <= 128) and
// row_id_body_cluster (a thread-block cluster per large matrix, work in jb.work).
//
// Row ID of M (m x n): column-pivoted Householder QR of M^T, truncated at the
// first k with |R_{k+1,k+1}| <= tol |R_11| (or k = kmax), then
// U = P [I; (R11^-1 R12)^T].  The columns of M^T are the rows of M, which are
// contiguous: every reflection updates each remaining row with one dot product
// and one axpy (a group of 4 to 32 lanes per row, sized to the row length), and
// the remaining row norms are recomputed in the same pass.  Pivot: largest remaining norm, lowest position on ties.
#pragma once
#include <cooperative_groups.h>

#include "bf_kernels.h"

namespace mf {

template <typename T>
__device__ __forceinline__ void row_id_body(const IdJob<T>& jb, T tol, int32_t max_rank, bool work_in_smem) {
  const int m = jb.m, n = jb.n;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Wr = work_in_smem ? reinterpret_cast<T*>(smraw) : jb.work;
  T* Wi = work_in_smem ? Wr + (int64_t)m * n : jb.work + jb.wplane;
  T* vr = reinterpret_cast<T*>(smraw) + (work_in_smem ? 2 * (int64_t)m * n : 0);   // Householder vector (re, im)
  T* vi = vr + n;
  T* nrm = vi + n;                           // remaining squared norms, by position
  int* perm = reinterpret_cast<int*>(nrm + m);
  __shared__ T red_v[32];
  __shared__ int red_i[32];
  __shared__ T sh_alpha_r, sh_alpha_i, sh_scale, sh_ref;
  __shared__ int sh_p, sh_stop;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  int G = 32;   // lanes per row in the reflection updates: about 12 or more columns per lane
  while (G > 4 && (G >> 1) * 12 >= n) G >>= 1;
  const int gid = tid / G, glane = tid % G, ngrp = (int)blockDim.x / G;
  // copy M to the work matrix (ld = n) and compute the row norms
  for (int r = warp; r < m; r += nw) {
    const T* mr = jb.M + (int64_t)r * jb.ld;
    const T* mi = mr + jb.plane;
    T s = 0;
    for (int c = lane; c < n; c += 32) {
      T a = mr[c], b = mi[c];
      Wr[(int64_t)r * n + c] = a;
      Wi[(int64_t)r * n + c] = b;
      s += a * a + b * b;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) { nrm[r] = s; perm[r] = r; }
  }
  int kmax = m < n ? m : n;
  if (max_rank > 0 && max_rank < kmax) kmax = max_rank;
  if (tid == 0) sh_stop = 0;
  __syncthreads();
  int rank = 0;
  for (int k = 0; k < kmax; ++k) {
    // pivot: largest remaining norm among positions k..m-1
    T best = T(-1);
    int bi = m;
    for (int q = k + tid; q < m; q += blockDim.x)
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
      for (int w = 1; w < nw; ++w)
        if (red_v[w] > best || (red_v[w] == best && red_i[w] < bi)) { best = red_v[w]; bi = red_i[w]; }
      T nu = sqrt(best > T(0) ? best : T(0));
      if (k == 0) sh_ref = nu;
      if (sh_ref == T(0) || nu <= tol * sh_ref) sh_stop = 1;
      else {
        sh_p = bi;
        T t = nrm[k]; nrm[k] = nrm[bi]; nrm[bi] = t;
        int ti = perm[k]; perm[k] = perm[bi]; perm[bi] = ti;
      }
    }
    __syncthreads();
    if (sh_stop) break;
    // Householder vector from the pivot row's coordinates k..n-1
    const int pr = perm[k];
    T* xr = Wr + (int64_t)pr * n;
    T* xi = Wi + (int64_t)pr * n;
    for (int c = k + tid; c < n; c += blockDim.x) {
      vr[c] = xr[c];
      vi[c] = xi[c];
    }
    __syncthreads();
    if (tid == 0) {
      const T tot = nrm[k];   // the pivot row's squared norm over coordinates k.. (independent of blockDim)
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
    // reflected pivot row: alpha e_k
    for (int c = k + tid; c < n; c += blockDim.x) {
      xr[c] = c == k ? sh_alpha_r : T(0);
      xi[c] = c == k ? sh_alpha_i : T(0);
    }
    // apply H to the remaining rows, recompute their norms beyond coordinate k: groups of G
    // lanes per row (G sized to the row length), all groups of a warp in lockstep
    const T sc = sh_scale;
    for (int base = k + 1; base < m; base += ngrp) {
      const int q = base + gid;
      const bool act = q < m;
      T* yr = Wr + (int64_t)(act ? perm[q] : 0) * n;
      T* yi = Wi + (int64_t)(act ? perm[q] : 0) * n;
      T dr = 0, di = 0;   // v^H y
      if (act)
#pragma unroll 4
        for (int c = k + glane; c < n; c += G) {
          T a = vr[c], b = vi[c], p = yr[c], r = yi[c];
          dr += a * p + b * r;
          di += a * r - b * p;
        }
      for (int o = G >> 1; o > 0; o >>= 1) {
        dr += __shfl_xor_sync(0xffffffffu, dr, o);
        di += __shfl_xor_sync(0xffffffffu, di, o);
      }
      dr *= sc;
      di *= sc;
      T s = 0;
      if (act)
#pragma unroll 4
        for (int c = k + glane; c < n; c += G) {
          T a = vr[c], b = vi[c];
          T p = yr[c] - (a * dr - b * di);
          T r = yi[c] - (a * di + b * dr);
          yr[c] = p;
          yi[c] = r;
          if (c > k) s += p * p + r * r;
        }
      for (int o = G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (act && glane == 0) nrm[q] = s;
    }
    __syncthreads();
    rank = k + 1;
  }
  __syncthreads();
  // outputs: rank, skeleton (first rank pivots), U = P [I; (R11^-1 R12)^T]
  const int r = rank;
  if (tid == 0) *jb.rank = r;
  for (int b = tid; b < r; b += blockDim.x) jb.sk[b] = perm[b];
  const int ldu = jb.ldu;

  T* Ur = jb.U;
  T* Ui = jb.U + jb.uplane;
  // identity rows
  for (int e = tid; e < r * r; e += blockDim.x) {
    int b = e / r, c = e % r;
    Ur[(int64_t)perm[b] * ldu + c] = b == c ? T(1) : T(0);
    Ui[(int64_t)perm[b] * ldu + c] = T(0);
  }
  // non-pivot rows: back substitution with R11 (R11[a][b] = work[perm[b]][a], a <= b), in place
  // in the row's first r work entries (its R12 column), then copied out to U
  for (int j = r + tid; j < m; j += blockDim.x) {
    const int q = perm[j];
    T* yr = Wr + (int64_t)q * n;
    T* yi = Wi + (int64_t)q * n;
    for (int b = r - 1; b >= 0; --b) {
      T accr = yr[b], acci = yi[b];
      for (int c = b + 1; c < r; ++c) {
        const int pc = perm[c];
        T Rr = Wr[(int64_t)pc * n + b], Ri = Wi[(int64_t)pc * n + b];
        T tr = yr[c], ti = yi[c];
        accr -= Rr * tr - Ri * ti;
        acci -= Rr * ti + Ri * tr;
      }
      const int pb = perm[b];
      T dr = Wr[(int64_t)pb * n + b], di = Wi[(int64_t)pb * n + b];
      T den = dr * dr + di * di;
      if (den == T(0)) den = T(1);
      yr[b] = (accr * dr + acci * di) / den;
      yi[b] = (acci * dr - accr * di) / den;
    }
  }
  __syncthreads();
  for (int e = tid; e < (m - r) * r; e += blockDim.x) {
    const int q = perm[r + e / r], c = e % r;
    Ur[(int64_t)q * ldu + c] = Wr[(int64_t)q * n + c];
    Ui[(int64_t)q * ldu + c] = Wi[(int64_t)q * n + c];
  }
}


}  // namespace mf

namespace mf {

// Register-resident variant for m <= 128 rows of n <= 8 RC columns (the randomized
// construction's sketch blocks): 1024 threads, 8 lanes per row, each lane keeping its RC
// columns (c = lane8 + 8 j) of the row in registers for the whole factorization.  A step
// costs two barriers: the pivot row's owners publish it in shared memory, every thread
// derives the reflection from it, updates its own columns, and the lanes of a row reduce
// the dot product and the new norm with shuffles; each warp leaves its largest norm for the
// next step's pivot.  The final rows go to shared memory for the back substitution.
// Same result contract as row_id_body; pivot: largest remaining norm, lowest row on ties.
template <typename T, int RC>
__device__ __forceinline__ void row_id_body_reg(const IdJob<T>& jb, T tol, int32_t max_rank) {
  constexpr int LPR = 8;
  const int m = jb.m, n = jb.n;
  const int kw = m < n ? m : n;   // columns kept for the back substitution (>= any rank)
  extern __shared__ __align__(16) unsigned char smraw[];
  T* pr = reinterpret_cast<T*>(smraw);   // pivot row (n values, re / im)
  T* pi = pr + n;
  T* Wr = pi + n;                         // m x kw, after the factorization
  T* Wi = Wr + (int64_t)m * kw;
  int* piv = reinterpret_cast<int*>(Wi + (int64_t)m * kw);
  __shared__ T wbest_v[2][32];
  __shared__ int wbest_i[2][32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int row = tid / LPR, l8 = tid % LPR;
  const bool mine = row < m;
  auto better = [](T v, int i, T ov, int oi) { return ov > v || (ov == v && oi < i); };
  T yr[RC], yi[RC];
  bool done = !mine;
  {
    T s = 0;
#pragma unroll
    for (int j = 0; j < RC; ++j) {
      const int c = l8 + LPR * j;
      T a = 0, b = 0;
      if (mine && c < n) {
        a = jb.M[(int64_t)row * jb.ld + c];
        b = jb.M[(int64_t)row * jb.ld + c + jb.plane];
      }
      yr[j] = a;
      yi[j] = b;
      s += a * a + b * b;
    }
    for (int o = LPR >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    T bv = mine ? s : T(-1);
    int bi = mine ? row : m;
    for (int o = 16; o >= LPR; o >>= 1) {
      T ov = __shfl_xor_sync(0xffffffffu, bv, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (better(bv, bi, ov, oi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { wbest_v[0][warp] = bv; wbest_i[0][warp] = bi; }
  }
  int kmax = kw;
  if (max_rank > 0 && max_rank < kmax) kmax = max_rank;
  __syncthreads();
  int rank = 0;
  T ref = T(0);
  const int nw = blockDim.x >> 5;
  for (int k = 0; k < kmax; ++k) {
    const int cb = k & 1, nb = cb ^ 1;
    T best = lane < nw ? wbest_v[cb][lane] : T(-1);   // the warps' candidates, reduced in every warp
    int q = lane < nw ? wbest_i[cb][lane] : m;
    for (int o = 16; o > 0; o >>= 1) {
      T ov = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, q, o);
      if (better(best, q, ov, oi)) { best = ov; q = oi; }
    }
    if (q >= m) break;
    const T nu = sqrt(best > T(0) ? best : T(0));
    if (k == 0) ref = nu;
    if (ref == T(0) || nu <= tol * ref) break;
    if (tid == 0) piv[k] = q;
    if (row == q) {   // publish the pivot row's coordinates k.. and take its place in R
#pragma unroll
      for (int j = 0; j < RC; ++j) {
        const int c = l8 + LPR * j;
        if (c >= k && c < n) { pr[c] = yr[j]; pi[c] = yi[j]; }
      }
    }
    __syncthreads();
    const T x0r = pr[k], x0i = pi[k];
    const T ax0 = sqrt(x0r * x0r + x0i * x0i);
    const T phr = ax0 > T(0) ? x0r / ax0 : T(1), phi = ax0 > T(0) ? x0i / ax0 : T(0);
    const T alr = -phr * nu, ali = -phi * nu;
    const T v0r = x0r - alr, v0i = x0i - ali;
    const T vv = best - (x0r * x0r + x0i * x0i) + v0r * v0r + v0i * v0i;
    const T sc = vv > T(0) ? T(2) / vv : T(0);
    if (row == q) {
      done = true;
#pragma unroll
      for (int j = 0; j < RC; ++j) {
        const int c = l8 + LPR * j;
        if (c >= k) { yr[j] = c == k ? alr : T(0); yi[j] = c == k ? ali : T(0); }
      }
    }
    T dr = 0, di = 0;   // v^H y over this lane's columns
    if (!done) {
#pragma unroll
      for (int j = 0; j < RC; ++j) {
        const int c = l8 + LPR * j;
        if (c >= k && c < n) {
          const T a = c == k ? v0r : pr[c], b = c == k ? v0i : pi[c];
          dr += a * yr[j] + b * yi[j];
          di += a * yi[j] - b * yr[j];
        }
      }
    }
    for (int o = LPR >> 1; o > 0; o >>= 1) {
      dr += __shfl_xor_sync(0xffffffffu, dr, o);
      di += __shfl_xor_sync(0xffffffffu, di, o);
    }
    dr *= sc;
    di *= sc;
    T s = 0;
    if (!done) {
#pragma unroll
      for (int j = 0; j < RC; ++j) {
        const int c = l8 + LPR * j;
        if (c >= k && c < n) {
          const T a = c == k ? v0r : pr[c], b = c == k ? v0i : pi[c];
          yr[j] -= a * dr - b * di;
          yi[j] -= a * di + b * dr;
          if (c > k) s += yr[j] * yr[j] + yi[j] * yi[j];
        }
      }
    }
    for (int o = LPR >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    T bv = done ? T(-1) : s;
    int bi = done ? m : row;
    for (int o = 16; o >= LPR; o >>= 1) {
      T ov = __shfl_xor_sync(0xffffffffu, bv, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (better(bv, bi, ov, oi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { wbest_v[nb][warp] = bv; wbest_i[nb][warp] = bi; }
    rank = k + 1;
    __syncthreads();
  }
  // rows to shared memory (first kw columns: R of the pivots, R12 of the others)
  if (mine) {
#pragma unroll
    for (int j = 0; j < RC; ++j) {
      const int c = l8 + LPR * j;
      if (c < kw) { Wr[(int64_t)row * kw + c] = yr[j]; Wi[(int64_t)row * kw + c] = yi[j]; }
    }
  }
  __syncthreads();
  const int r = rank;
  if (tid == 0) *jb.rank = r;
  for (int b = tid; b < r; b += blockDim.x) jb.sk[b] = piv[b];
  const int ldu = jb.ldu;
  T* Ur = jb.U;
  T* Ui = jb.U + jb.uplane;
  for (int e = tid; e < r * r; e += blockDim.x) {
    int b = e / r, c = e % r;
    Ur[(int64_t)piv[b] * ldu + c] = b == c ? T(1) : T(0);
    Ui[(int64_t)piv[b] * ldu + c] = T(0);
  }
  // non-pivot rows (the row's own lanes know whether it is done): back substitution in place
  if (mine && !done && l8 == 0) {
    T* wr = Wr + (int64_t)row * kw;
    T* wi = Wi + (int64_t)row * kw;
    for (int b = r - 1; b >= 0; --b) {
      T accr = wr[b], acci = wi[b];
      for (int c = b + 1; c < r; ++c) {
        const int pc = piv[c];
        T Rr = Wr[(int64_t)pc * kw + b], Ri = Wi[(int64_t)pc * kw + b];
        accr -= Rr * wr[c] - Ri * wi[c];
        acci -= Rr * wi[c] + Ri * wr[c];
      }
      const int pb = piv[b];
      T dr2 = Wr[(int64_t)pb * kw + b], di2 = Wi[(int64_t)pb * kw + b];
      T den = dr2 * dr2 + di2 * di2;
      if (den == T(0)) den = T(1);
      wr[b] = (accr * dr2 + acci * di2) / den;
      wi[b] = (acci * dr2 - accr * di2) / den;
    }
  }
  __syncthreads();
  // copy the non-pivot rows' coefficients out (the lanes of a row, columns strided)
  if (mine && !done)
    for (int c = l8; c < r; c += LPR) {
      Ur[(int64_t)row * ldu + c] = Wr[(int64_t)row * kw + c];
      Ui[(int64_t)row * ldu + c] = Wi[(int64_t)row * kw + c];
    }
}

}  // namespace mf

namespace mf {

// Cluster variant for the large matrices whose QR work stays in global memory: the C CTAs of a
// thread-block cluster share one matrix, CTA c owning the rows r with r % C == c.  Every CTA
// keeps the same position order (perm / pos).  A step exchanges each CTA's best candidate
// through distributed shared memory (cluster barrier 1), every CTA derives the same reflection
// from the pivot row in global memory, the pivot row's owner writes the reflected row once all
// have read it (cluster barrier 2), and each CTA updates its own rows.  Per row the arithmetic is
// row_id_body's (same group width, same order), so the results are identical; pivot: largest
// remaining norm, lowest position on ties.  Rows of other CTAs are read through L2 (ld.global.cg).
template <typename T, int C>
__device__ __forceinline__ void row_id_body_cluster(const IdJob<T>& jb, T tol, int32_t max_rank) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank();
  const int m = jb.m, n = jb.n;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Wr = jb.work;
  T* Wi = jb.work + jb.wplane;
  T* vr = reinterpret_cast<T*>(smraw);   // Householder vector (re, im)
  T* vi = vr + n;
  T* nrm = vi + n;                        // remaining squared norms, by row (own rows)
  int* perm = reinterpret_cast<int*>(nrm + m);   // position -> row
  int* pos = perm + m;                            // row -> position
  __shared__ T red_v[32];
  __shared__ int red_i[32];
  __shared__ T cand_v[2];   // this CTA's best candidate of steps k (k & 1)
  __shared__ int cand_p[2];
  __shared__ T sh_alpha_r, sh_alpha_i, sh_scale, sh_ref, sh_tot;
  __shared__ int sh_stop;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  int G = 32;   // lanes per row in the reflection updates (as in row_id_body)
  while (G > 4 && (G >> 1) * 12 >= n) G >>= 1;
  const int gid = tid / G, glane = tid % G, ngrp = (int)blockDim.x / G;
  const int nown = m > crank ? (m - crank + C - 1) / C : 0;   // own rows: crank + C t
  auto better = [](T v, int p, T ov, int op) { return ov > v || (ov == v && op < p); };
  for (int t = warp; t < nown; t += nw) {
    const int r = crank + C * t;
    const T* mr = jb.M + (int64_t)r * jb.ld;
    const T* mi = mr + jb.plane;
    T s = 0;
    for (int c = lane; c < n; c += 32) {
      T a = mr[c], b = mi[c];
      Wr[(int64_t)r * n + c] = a;
      Wi[(int64_t)r * n + c] = b;
      s += a * a + b * b;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) nrm[r] = s;
  }
  for (int q = tid; q < m; q += blockDim.x) {
    perm[q] = q;
    pos[q] = q;
  }
  int kmax = m < n ? m : n;
  if (max_rank > 0 && max_rank < kmax) kmax = max_rank;
  if (tid == 0) sh_stop = 0;
  __syncthreads();
  int rank = 0;
  for (int k = 0; k < kmax; ++k) {
    const int sl = k & 1;
    T best = T(-1);
    int bp = m;
    for (int t = tid; t < nown; t += blockDim.x) {
      const int r = crank + C * t, p = pos[r];
      if (p >= k && better(best, bp, nrm[r], p)) { best = nrm[r]; bp = p; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      T ob = __shfl_xor_sync(0xffffffffu, best, o);
      int op = __shfl_xor_sync(0xffffffffu, bp, o);
      if (better(best, bp, ob, op)) { best = ob; bp = op; }
    }
    if (lane == 0) { red_v[warp] = best; red_i[warp] = bp; }
    __syncthreads();
    if (tid == 0) {
      best = red_v[0]; bp = red_i[0];
      for (int w = 1; w < nw; ++w)
        if (better(best, bp, red_v[w], red_i[w])) { best = red_v[w]; bp = red_i[w]; }
      cand_v[sl] = best;
      cand_p[sl] = bp;
    }
    cl.sync();   // 1: every CTA's candidate, and the rows of the previous step, are published
    if (tid == 0) {
      T gb = T(-1);
      int gp = m;
      for (int c = 0; c < C; ++c) {
        const T ov = cl.map_shared_rank(cand_v, c)[sl];
        const int op = cl.map_shared_rank(cand_p, c)[sl];
        if (better(gb, gp, ov, op)) { gb = ov; gp = op; }
      }
      T nu = sqrt(gb > T(0) ? gb : T(0));
      if (k == 0) sh_ref = nu;
      if (gp >= m || sh_ref == T(0) || nu <= tol * sh_ref) sh_stop = 1;
      else {
        sh_tot = gb;   // the pivot row's squared norm over coordinates k..
        const int rk = perm[k], rp = perm[gp];
        perm[k] = rp; perm[gp] = rk;
        pos[rp] = k; pos[rk] = gp;
      }
    }
    __syncthreads();
    if (sh_stop) break;
    const int pr = perm[k];
    T* xr = Wr + (int64_t)pr * n;
    T* xi = Wi + (int64_t)pr * n;
    for (int c = k + tid; c < n; c += blockDim.x) {
      vr[c] = __ldcg(xr + c);
      vi[c] = __ldcg(xi + c);
    }
    __syncthreads();
    if (tid == 0) {
      const T tot = sh_tot;
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
    cl.sync();   // 2: every CTA holds the pivot row (and its reflection data)
    if (pr % C == crank)
      for (int c = k + tid; c < n; c += blockDim.x) {
        xr[c] = c == k ? sh_alpha_r : T(0);
        xi[c] = c == k ? sh_alpha_i : T(0);
      }
    const T sc = sh_scale;
    for (int base = 0; base < nown; base += ngrp) {
      const int t = base + gid;
      const int r = crank + C * t;
      const bool act = t < nown && pos[r] > k;
      T* yr = Wr + (int64_t)(act ? r : 0) * n;
      T* yi = Wi + (int64_t)(act ? r : 0) * n;
      T dr = 0, di = 0;   // v^H y
      if (act)
#pragma unroll 4
        for (int c = k + glane; c < n; c += G) {
          T a = vr[c], b = vi[c], p = yr[c], q = yi[c];
          dr += a * p + b * q;
          di += a * q - b * p;
        }
      for (int o = G >> 1; o > 0; o >>= 1) {
        dr += __shfl_xor_sync(0xffffffffu, dr, o);
        di += __shfl_xor_sync(0xffffffffu, di, o);
      }
      dr *= sc;
      di *= sc;
      T s = 0;
      if (act)
#pragma unroll 4
        for (int c = k + glane; c < n; c += G) {
          T a = vr[c], b = vi[c];
          T p = yr[c] - (a * dr - b * di);
          T q = yi[c] - (a * di + b * dr);
          yr[c] = p;
          yi[c] = q;
          if (c > k) s += p * p + q * q;
        }
      for (int o = G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (act && glane == 0) nrm[r] = s;
    }
    __syncthreads();
    rank = k + 1;
  }
  cl.sync();   // 3: the last reflected pivot row is visible; no CTA reads another's candidates after this
  const int r = rank;
  if (crank == 0) {
    if (tid == 0) *jb.rank = r;
    for (int b = tid; b < r; b += blockDim.x) jb.sk[b] = perm[b];
  }
  const int ldu = jb.ldu;
  T* Ur = jb.U;
  T* Ui = jb.U + jb.uplane;
  // identity rows of the own pivots
  for (int e = tid; e < nown * r; e += blockDim.x) {
    const int t = e / r, c = e % r, row = crank + C * t, b = pos[row];
    if (b >= r) continue;
    Ur[(int64_t)row * ldu + c] = b == c ? T(1) : T(0);
    Ui[(int64_t)row * ldu + c] = T(0);
  }
  // own non-pivot rows: back substitution with R11 (R11[a][b] = work[perm[b]][a], a <= b)
  for (int t = tid; t < nown; t += blockDim.x) {
    const int q = crank + C * t;
    if (pos[q] < r) continue;
    T* yr = Wr + (int64_t)q * n;
    T* yi = Wi + (int64_t)q * n;
    for (int b = r - 1; b >= 0; --b) {
      T accr = yr[b], acci = yi[b];
      for (int c = b + 1; c < r; ++c) {
        const int pc = perm[c];
        T Rr = __ldcg(Wr + (int64_t)pc * n + b), Ri = __ldcg(Wi + (int64_t)pc * n + b);
        T tr = yr[c], ti = yi[c];
        accr -= Rr * tr - Ri * ti;
        acci -= Rr * ti + Ri * tr;
      }
      const int pb = perm[b];
      T dr = __ldcg(Wr + (int64_t)pb * n + b), di = __ldcg(Wi + (int64_t)pb * n + b);
      T den = dr * dr + di * di;
      if (den == T(0)) den = T(1);
      yr[b] = (accr * dr + acci * di) / den;
      yi[b] = (acci * dr - accr * di) / den;
    }
  }
  __syncthreads();
  for (int e = tid; e < nown * r; e += blockDim.x) {
    const int t = e / r, c = e % r, q = crank + C * t;
    if (pos[q] < r) continue;
    Ur[(int64_t)q * ldu + c] = Wr[(int64_t)q * n + c];
    Ui[(int64_t)q * ldu + c] = Wi[(int64_t)q * n + c];
  }
}

}  // namespace mf
