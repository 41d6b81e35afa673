// Batched planar complex GEMM for narrow products, C = alpha op(A) B + beta C with
// n <= 128, in column tiles of NB = 16 or 32: the solve's front products (n = number of right-hand
// sides, Alg. 1's last line) and the butterfly level products with blocks of vectors
// (Sec. 3).  These stream op(A) once and are bound by HBM (or, for n >= 16, by the
// FP32 FMA rate), not by a square tile's reuse.
//
// One CTA (4 warps) owns 32 rows and NB columns of C (tile {desc, tm, tn}).  K advances in
// tiles of 32: the A tile (32 x 32, stored k-major) and the B tile (32 x NB) are copied to
// shared memory with cp.async, four tiles in flight; each warp takes 8 of the tile's k, lane = row, with the
// B row broadcast from shared memory.  The four warps' partial sums are added in
// shared memory.  When there are few row tiles, K is also split over the CTAs of a
// thread-block cluster (gridDim.y = split, cluster 1 x split): every CTA reduces its
// own k-range and the leader adds the others' partial tiles through distributed
// shared memory, in rank order (deterministic), and applies alpha / beta.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace mf {

namespace {

constexpr int NR_BM = 32, NR_BK = 32, NR_WARPS = 4, NR_STAGES = 4;

template <typename T, int NB>
struct NrSmem {
  T ar[NR_BK][NR_BM + 1], ai[NR_BK][NR_BM + 1];   // A tile, k-major (padded: conflict-free)
  T br[NR_BK][NB], bi[NR_BK][NB];                 // B tile
};

// one element global -> shared, asynchronous; src_bytes = 0 fills zeros (out-of-range elements)
template <typename T>
__device__ __forceinline__ void cp_elem(T* dst, const T* src, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? (int)sizeof(T) : 0;
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(src), "r"(n));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(src), "r"(n));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <typename T, int NB, bool TWO>
__global__ void __launch_bounds__(128) k_gemm_nrhs(const GemmDesc<T>* __restrict__ descs,
                                                   const GemmTile* __restrict__ tiles) {
  constexpr int AE = NR_BM * NR_BK / 128;   // A elements per thread and plane (8)
  constexpr int BE = NR_BK * NB / 128;      // B elements per thread and plane (NB / 4)
  constexpr int BSTEP = 128 / NB;           // k rows between a thread's B elements (transB = 0)
  extern __shared__ __align__(16) unsigned char nr_raw[];
  NrSmem<T, NB>* S = reinterpret_cast<NrSmem<T, NB>*>(nr_raw);   // NR_STAGES tiles in flight
  const GemmTile t = tiles[blockIdx.x];
  const GemmDesc<T> d = descs[t.desc];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m0 = t.tm * NR_BM, n0 = t.tn * NB;
  const int nkt = (d.k + NR_BK - 1) / NR_BK;
  const int ks = gridDim.y, kr = blockIdx.y;
  const int kt0 = (int)((int64_t)nkt * kr / ks), kt1 = (int)((int64_t)nkt * (kr + 1) / ks);
  const int k1 = d.k1 > 0 ? d.k1 : d.k;   // reduction indices of the first term
  // this thread's A elements: (mm, kk) = (tid / 32 + 4 e, tid % 32) for transA = 0 (k-contiguous
  // rows), (tid % 32, tid / 32 + 4 e) for transA = 1 (m-contiguous rows of the stored A)
  const int a_fast = tid & 31, a_slow = tid >> 5;
  const int a_mm = d.transA == 0 ? a_slow : a_fast, a_kk = d.transA == 0 ? a_fast : a_slow;
  const int a_dm = d.transA == 0 ? 4 : 0, a_dk = d.transA == 0 ? 0 : 4;
  const int b_nn = d.transB == 0 ? tid % NB : tid >> 5, b_kk = d.transB == 0 ? tid / NB : tid & 31;
  const int b_dn = d.transB == 0 ? 0 : 4, b_dk = d.transB == 0 ? BSTEP : 0;
  // copies of k tile kt into stage slot (one cp.async per element, zero-filled outside)
  auto issue = [&](int kt, int slot) {
    NrSmem<T, NB>& Sm = S[slot];
    const int k0 = kt * NR_BK;
#pragma unroll
    for (int e = 0; e < AE; ++e) {
      const int gm = m0 + a_mm + a_dm * e, gk = k0 + a_kk + a_dk * e;
      const bool ok = gm < d.m && gk < d.k;
      const bool s2 = TWO && gk >= k1;   // second term of a two-term product
      const T* a = s2 ? d.A2.re : d.A.re;
      const int64_t apl = s2 ? d.A2.plane : d.A.plane, ald = s2 ? d.A2.ld : d.A.ld;
      const int kk2 = s2 ? gk - k1 : gk;
      const int64_t off = d.transA == 0 ? (int64_t)gm * ald + kk2 : (int64_t)kk2 * ald + gm;
      const T* src = ok ? a + off : d.A.re;   // nothing is read when !ok (zero fill)
      cp_elem(&Sm.ar[a_kk + a_dk * e][a_mm + a_dm * e], src, ok);
      cp_elem(&Sm.ai[a_kk + a_dk * e][a_mm + a_dm * e], ok ? src + apl : src, ok);
    }
#pragma unroll
    for (int e = 0; e < BE; ++e) {
      const int nn = n0 + b_nn + b_dn * e, gk = k0 + b_kk + b_dk * e;
      const bool ok = nn < d.n && gk < d.k;
      const bool s2 = TWO && gk >= k1;
      const T* b = s2 ? d.B2.re : d.B.re;
      const int64_t bpl = s2 ? d.B2.plane : d.B.plane, bld = s2 ? d.B2.ld : d.B.ld;
      const int kk2 = s2 ? gk - k1 : gk;
      const int64_t off = d.transB == 0 ? (int64_t)kk2 * bld + nn : (int64_t)nn * bld + kk2;
      const T* src = ok ? b + off : d.B.re;
      cp_elem(&Sm.br[b_kk + b_dk * e][b_nn + b_dn * e], src, ok);
      cp_elem(&Sm.bi[b_kk + b_dk * e][b_nn + b_dn * e], ok ? src + bpl : src, ok);
    }
  };
  T cr[NB], ci[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) cr[j] = ci[j] = T(0);
  // pipeline: NR_STAGES - 1 tiles in flight ahead of the one being multiplied (one commit group per
  // tile, empty groups past the end keep the wait counts uniform)
#pragma unroll
  for (int s0 = 0; s0 < NR_STAGES - 1; ++s0) {
    if (kt0 + s0 < kt1) issue(kt0 + s0, s0);
    cp_commit();
  }
  for (int kt = kt0; kt < kt1; ++kt) {
    cp_wait<NR_STAGES - 2>();   // tile kt has landed (this thread's copies)
    __syncthreads();            // ... everyone's; and every reader of the slot refilled below is done
    const int nxt = kt + NR_STAGES - 1;
    if (nxt < kt1) issue(nxt, (nxt - kt0) % NR_STAGES);
    cp_commit();
    const NrSmem<T, NB>& Sm = S[(kt - kt0) % NR_STAGES];
#pragma unroll 2
    for (int q = 0; q < NR_BK / NR_WARPS; ++q) {
      const int kk = warp * (NR_BK / NR_WARPS) + q;
      const T a_r = Sm.ar[kk][lane], a_i = Sm.ai[kk][lane];
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const T b_r = Sm.br[kk][j], b_i = Sm.bi[kk][j];
        cr[j] = fma(a_r, b_r, cr[j]);
        cr[j] = fma(-a_i, b_i, cr[j]);
        ci[j] = fma(a_r, b_i, ci[j]);
        ci[j] = fma(a_i, b_r, ci[j]);
      }
    }
  }
  cp_wait<0>();
  // the four warps' partial sums -> part (32 x NB complex) in the front of the shared memory
  __syncthreads();
  T* red = reinterpret_cast<T*>(nr_raw);   // [warp][2][NB][32]
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    red[((warp * 2 + 0) * NB + j) * NR_BM + lane] = cr[j];
    red[((warp * 2 + 1) * NB + j) * NR_BM + lane] = ci[j];
  }
  __syncthreads();
  T* part = red + NR_WARPS * 2 * NB * NR_BM;   // [2][NB][32]
  for (int e = tid; e < 2 * NB * NR_BM; e += 128) {
    T s = T(0);
#pragma unroll
    for (int w = 0; w < NR_WARPS; ++w) s += red[w * 2 * NB * NR_BM + e];
    part[e] = s;
  }
  if (ks > 1) {
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();   // every CTA's part is complete
    if (cl.block_rank() == 0) {
      for (int r = 1; r < ks; ++r) {
        const T* other = cl.map_shared_rank(part, r);
        for (int e = tid; e < 2 * NB * NR_BM; e += 128) part[e] += other[e];
      }
    }
    cl.sync();   // the others' shared memory stays alive until the leader has read it
    if (cl.block_rank() != 0) return;
  }
  __syncthreads();
  T* Cr = d.C.re;
  T* Ci = d.C.re + d.C.plane;
  for (int e = tid; e < NB * NR_BM; e += 128) {
    const int j = e / NR_BM, r = e % NR_BM;
    const int gm = m0 + r;
    if (gm >= d.m || n0 + j >= d.n) continue;
    const int64_t off = (int64_t)gm * d.C.ld + n0 + j;
    T vr = d.alpha * part[j * NR_BM + r], vi = d.alpha * part[(NB + j) * NR_BM + r];
    if (d.beta != T(0)) {
      vr += d.beta * Cr[off];
      vi += d.beta * Ci[off];
    }
    Cr[off] = vr;
    Ci[off] = vi;
  }
}

template <typename T, int NB, bool TWO>
void launch_nb(const GemmDesc<T>* d_desc, const GemmTile* d_tiles, int ntiles, int ksplit, cudaStream_t st) {
  const size_t red = (size_t)(NR_WARPS + 1) * 2 * NB * NR_BM * sizeof(T);
  const size_t stages = NR_STAGES * sizeof(NrSmem<T, NB>);
  const size_t smem = stages > red ? stages : red;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemm_nrhs<T, NB, TWO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_gemm_nrhs<T, NB, TWO>, cudaFuncAttributeNonPortableClusterSizeAllowed, 0);
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ntiles, (unsigned)ksplit, 1);
  cfg.blockDim = dim3(128, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 1;
  at[0].val.clusterDim.y = (unsigned)ksplit;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = ksplit > 1 ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k_gemm_nrhs<T, NB, TWO>, d_desc, d_tiles);
}

template <typename T, int NB>
void launch_nb2(const GemmDesc<T>* d_desc, const GemmTile* d_tiles, int ntiles, int ksplit, bool two, cudaStream_t st) {
  if (two) launch_nb<T, NB, true>(d_desc, d_tiles, ntiles, ksplit, st);
  else launch_nb<T, NB, false>(d_desc, d_tiles, ntiles, ksplit, st);
}

}  // namespace

int gemm_nrhs_width(int max_n, size_t elem) {
  (void)elem;
  if (max_n <= 16) return 16;
  if (max_n <= 32) return 32;
  if (max_n > 128) return 0;
  return (max_n + 15) / 16 * 16 < (max_n + 31) / 32 * 32 ? 16 : 32;   // column tiles of 16 or 32
}

int gemm_nrhs_split(int ntiles, int max_k) {
  int ks = 1;
  while (ks < 8 && (int64_t)ntiles * ks < 2 * 152 && max_k / (2 * ks) >= 2 * NR_BK) ks *= 2;
  return ks;
}

template <typename T>
void launch_gemm_nrhs(const GemmDesc<T>* d_desc, const GemmTile* d_tiles, int ntiles, int nb, int ksplit,
                      cudaStream_t st, bool two) {
  if (ntiles <= 0) return;
  if (ksplit < 1) ksplit = 1;
  count_launches(1);
  if (nb <= 16) launch_nb2<T, 16>(d_desc, d_tiles, ntiles, ksplit, two, st);
  else if (nb <= 32 || sizeof(T) != 4) launch_nb2<T, 32>(d_desc, d_tiles, ntiles, ksplit, two, st);
  else launch_nb2<T, (sizeof(T) == 4 ? 64 : 32)>(d_desc, d_tiles, ntiles, ksplit, two, st);
}

template void launch_gemm_nrhs<float>(const GemmDesc<float>*, const GemmTile*, int, int, int, cudaStream_t, bool);
template void launch_gemm_nrhs<double>(const GemmDesc<double>*, const GemmTile*, int, int, int, cudaStream_t, bool);

}  // namespace mf
