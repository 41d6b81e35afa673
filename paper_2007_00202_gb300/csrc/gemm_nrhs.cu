// Batched planar complex GEMM for narrow products, C = alpha op(A) B + beta C with
// n <= 128, in column tiles of NB = 16 or 32: the solve's front products (n = number of right-hand
// sides, Alg. 1's last line) and the butterfly level products with blocks of vectors
// (Sec. 3).  These stream op(A) once and are bound by HBM (or, for n >= 16, by the
// FP32 FMA rate), not by a square tile's reuse.
//
// One CTA (4 warps) owns 32 rows and NB columns of C (tile {desc, tm, tn}).  K advances in
// tiles of 32 (a two-term product multiplies the first term's tiles, then the second's): the A
// tile (32 x 32, k-major, real and imaginary parts interleaved) and the B tile (32 x NB, planar)
// are copied to shared memory with cp.async (element-wise for A; 16-byte chunks for B when its
// rows and planes are aligned), up to four tiles in flight (the pipeline depth is sized to the
// launch's largest K).  Each warp takes 8 of the tile's k (none past the tile's valid rows),
// lane = row, with NB columns of B broadcast from shared memory in 16-byte loads.  The four
// warps' partial sums are added in shared memory.  When there are few row tiles, K is also split
// over the CTAs of a thread-block cluster (gridDim.y = split, cluster 1 x split): every CTA
// reduces its own k-range and the leader adds the others' partial tiles through distributed
// shared memory, in rank order (deterministic), applies alpha / beta and writes C rows.
#include <cooperative_groups.h>
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace mf {

namespace {

constexpr int NR_BM = 32, NR_BK = 32, NR_WARPS = 4, NR_MAX_STAGES = 4;
constexpr int NR_STAGE_BUDGET = 51200;   // bytes of stage buffers per CTA: 4 CTAs per SM

template <typename T> struct Cx2;
template <> struct Cx2<float> { using type = float2; };
template <> struct Cx2<double> { using type = double2; };
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

// One pipeline slot: the A tile k-major with (re, im) interleaved (one 8- or 16-byte load gives a
// lane its complex element), padded rows; the B tile planar (broadcast 16-byte loads of 16 / sizeof(T)
// columns).
template <typename T, int NB>
struct NrSlot {
  typename Cx2<T>::type a[NR_BK][NR_BM + 1];
  T br[NR_BK][NB], bi[NR_BK][NB];
};
static_assert(sizeof(NrSlot<float, 16>) % 16 == 0 && sizeof(NrSlot<float, 32>) % 16 == 0, "slot alignment");
static_assert(sizeof(NrSlot<double, 16>) % 16 == 0 && sizeof(NrSlot<double, 32>) % 16 == 0, "slot alignment");

template <typename T, int NB>
constexpr int nr_max_slots() {
  return NR_STAGE_BUDGET / (int)sizeof(NrSlot<T, NB>) < 2 ? 2
         : NR_STAGE_BUDGET / (int)sizeof(NrSlot<T, NB>) > NR_MAX_STAGES ? NR_MAX_STAGES
                                                                         : NR_STAGE_BUDGET / (int)sizeof(NrSlot<T, NB>);
}
// partial sums of the four warps, [warp][plane][column][row], rows padded (conflict-free both ways)
template <typename T, int NB>
constexpr size_t nr_red_bytes() { return (size_t)NR_WARPS * 2 * NB * (NR_BM + 1) * sizeof(T); }

// global -> shared, asynchronous: one element, or a 16-byte chunk of which the first `bytes` are
// copied and the rest zero-filled
template <typename T>
__device__ __forceinline__ void cp_elem(unsigned dst, const T* src) {
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_chunk(unsigned dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// This thread's share of the copies of one operand term: element e of a tile starting at reduction
// index k0 comes from p + k0 * ks + e * es (+ plane for the imaginary part); it is wanted when bit e
// of `mask` is set and its tile-local reduction index kx + e * kd is below the tile's valid count.
template <typename T>
struct TermSrc {
  const T* p;
  int64_t pl;
  int es, ks;
  unsigned mask;
  int kx, kd;
  int vec;   // B only: 16-byte chunks (transB = 0, aligned planes and rows)
};

template <typename T, int NB, bool TWO>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 2) k_gemm_nrhs(const GemmDesc<T>* __restrict__ descs,
                                                      const GemmTile* __restrict__ tiles, int nslots) {
  using C2 = typename Cx2<T>::type;
  using V16 = typename Vec16<T>::type;
  constexpr int V = 16 / (int)sizeof(T);      // elements of one 16-byte chunk
  constexpr int AE = NR_BM * NR_BK / 128;     // A elements per thread (8)
  constexpr int BE = NR_BK * NB / 128;        // B elements per thread, element-wise copies
  constexpr int BC = NR_BK * NB / V / 128;    // B chunks per thread, 16-byte copies
  constexpr int KW = NR_BK / NR_WARPS;        // reduction indices of a tile per warp
  static_assert(BC >= 1 && BE >= 1, "tile shape");
  extern __shared__ __align__(16) unsigned char nr_raw[];
  NrSlot<T, NB>* S = reinterpret_cast<NrSlot<T, NB>*>(nr_raw);
  // programmatic dependent launch: the next kernel of the stream may start its own set-up now; it
  // waits (griddepcontrol.wait) for this grid's completion before it reads anything this grid writes
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  const GemmTile t = tiles[blockIdx.x];   // descriptors and tile lists are written before the launch
  const GemmDesc<T>& d = descs[t.desc];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = d.m, n = d.n, k = d.k, transA = d.transA, transB = d.transB;
  const int m0 = t.tm * NR_BM, n0 = t.tn * NB;
  const int k1 = TWO && d.k1 > 0 ? d.k1 : k;   // reduction indices of the first term
  const int nt1 = (k1 + NR_BK - 1) / NR_BK;
  const int nkt = nt1 + (TWO ? (k - k1 + NR_BK - 1) / NR_BK : 0);   // tiles: first term's, then second's
  const int ks = gridDim.y, kr = blockIdx.y;
  const int kt0 = (int)((int64_t)nkt * kr / ks), kt1 = (int)((int64_t)nkt * (kr + 1) / ks);
  const int P = nslots;   // pipeline depth (2 .. 4)

  // per-thread copy plans.  A, transA = 0 (rows k-contiguous): element e = (row a_slow + 4e, k lane);
  // transA = 1 (stored k x m): element e = (row lane, k a_slow + 4e).
  const int a_slow = tid >> 5;
  auto a_plan = [&](const PMat<T>& A) {
    TermSrc<T> s;
    s.es = 4 * (int)A.ld;
    s.pl = A.plane;
    if (transA == 0) {
      s.p = A.re + (int64_t)(m0 + a_slow) * A.ld + lane;
      s.ks = 1;
      s.mask = 0;
#pragma unroll
      for (int e = 0; e < AE; ++e) s.mask |= (m0 + a_slow + 4 * e < m ? 1u : 0u) << e;
      s.kx = lane;
      s.kd = 0;
    } else {
      s.p = A.re + (int64_t)a_slow * A.ld + m0 + lane;
      s.ks = (int)A.ld;
      s.mask = m0 + lane < m ? 0xffu : 0u;
      s.kx = a_slow;
      s.kd = 4;
    }
    s.vec = 0;
    return s;
  };
  const int a_d0 = transA == 0 ? lane * (NR_BM + 1) + a_slow : a_slow * (NR_BM + 1) + lane;
  const int a_dd = transA == 0 ? 4 : 4 * (NR_BM + 1);
  // B, transB = 0 (stored k x n): chunk c = tid + 128 e covers row c / (NB / V), columns
  // (c % (NB / V)) V ..; element-wise: element e = (row tid / NB + (128 / NB) e, column tid % NB).
  // transB = 1 (stored n x k): element e = (row lane, column a_slow + 4e).
  auto b_plan = [&](const PMat<T>& B) {
    TermSrc<T> s;
    s.pl = B.plane;
    s.vec = transB == 0 && B.ld % V == 0 && B.plane % V == 0 && ((uintptr_t)B.re & 15) == 0;
    if (s.vec) {
      const int c = tid, row = c / (NB / V), col = (c % (NB / V)) * V;
      s.p = B.re + (int64_t)row * B.ld + n0 + col;
      s.es = (128 / (NB / V)) * (int)B.ld;
      s.ks = (int)B.ld;
      s.mask = 0;
      s.kx = row;
      s.kd = 128 / (NB / V);
    } else if (transB == 0) {
      s.p = B.re + (int64_t)(tid / NB) * B.ld + n0 + tid % NB;
      s.es = (128 / NB) * (int)B.ld;
      s.ks = (int)B.ld;
      s.mask = n0 + tid % NB < n ? 0xffffffffu : 0u;
      s.kx = tid / NB;
      s.kd = 128 / NB;
    } else {
      s.p = B.re + (int64_t)(n0 + a_slow) * B.ld + lane;
      s.es = 4 * (int)B.ld;
      s.ks = 1;
      s.mask = 0;
#pragma unroll
      for (int e = 0; e < BE; ++e) s.mask |= (n0 + a_slow + 4 * e < n ? 1u : 0u) << e;
      s.kx = lane;
      s.kd = 0;
    }
    return s;
  };
  const TermSrc<T> pa1 = a_plan(d.A), pb1 = b_plan(d.B);
  TermSrc<T> pa2 = pa1, pb2 = pb1;
  if (TWO && nkt > nt1) {
    pa2 = a_plan(d.A2);
    pb2 = b_plan(d.B2);
  }
  const unsigned sbase = (unsigned)__cvta_generic_to_shared(nr_raw);
  // operands and C may be written by the preceding kernel: wait for it before the first copy
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  const int b_vcol = (tid % (NB / V)) * V;   // chunk column of this thread (16-byte copies)
  constexpr unsigned SBR = (unsigned)(sizeof(C2) * NR_BK * (NR_BM + 1));   // offset of br in a slot
  constexpr unsigned SBI = (unsigned)(sizeof(T) * NR_BK * NB);             // bi - br

  // copies of tile vt (of the first term, then of the second) into slot `slot`
  auto issue = [&](int vt, int slot) {
    const bool second = TWO && vt >= nt1;
    const TermSrc<T> A = second ? pa2 : pa1;   // copies (field-wise selects), not references
    const TermSrc<T> B = second ? pb2 : pb1;
    const int k0 = (second ? vt - nt1 : vt) * NR_BK;
    const int kv = min(NR_BK, (second ? k - k1 : k1) - k0);   // valid reduction indices of the tile
    const unsigned sa = sbase + (unsigned)(slot * sizeof(NrSlot<T, NB>));
    const unsigned sbr = sa + SBR, sbi = sbr + SBI;
    const T* qa = A.p + (int64_t)k0 * A.ks;
#pragma unroll
    for (int e = 0; e < AE; ++e) {
      if (((A.mask >> e) & 1u) && A.kx + A.kd * e < kv) {
        const unsigned dst = sa + (unsigned)((a_d0 + a_dd * e) * sizeof(C2));
        cp_elem(dst, qa);
        cp_elem(dst + (unsigned)sizeof(T), qa + A.pl);
      }
      qa += A.es;
    }
    const T* qb = B.p + (int64_t)k0 * B.ks;
    if (B.vec) {
      const int cnt = n - n0 - b_vcol;
      const int bytes = (cnt >= V ? V : cnt > 0 ? cnt : 0) * (int)sizeof(T);
#pragma unroll
      for (int e = 0; e < BC; ++e) {
        if (bytes > 0 && B.kx + B.kd * e < kv) {
          const unsigned off = (unsigned)((tid + 128 * e) * V * sizeof(T));
          cp_chunk(sbr + off, qb, bytes);
          cp_chunk(sbi + off, qb + B.pl, bytes);
        }
        qb += B.es;
      }
    } else {
      const int b_d0 = transB == 0 ? tid : lane * NB + a_slow;
      const int b_dd = transB == 0 ? 128 : 4;
#pragma unroll
      for (int e = 0; e < BE; ++e) {
        if (((B.mask >> e) & 1u) && B.kx + B.kd * e < kv) {
          const unsigned off = (unsigned)((b_d0 + b_dd * e) * sizeof(T));
          cp_elem(sbr + off, qb);
          cp_elem(sbi + off, qb + B.pl);
        }
        qb += B.es;
      }
    }
  };

  T cr[NB], ci[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) cr[j] = ci[j] = T(0);
  // pipeline: P - 1 tiles in flight ahead of the one being multiplied (one commit group per tile;
  // empty groups past the end keep the wait counts uniform)
  for (int s0 = 0; s0 < P - 1; ++s0) {
    if (kt0 + s0 < kt1) issue(kt0 + s0, s0);
    cp_commit();
  }
  for (int kt = kt0; kt < kt1; ++kt) {
    if (P >= 4) cp_wait<2>();   // tile kt has landed (this thread's copies)
    else if (P == 3) cp_wait<1>();
    else cp_wait<0>();
    __syncthreads();            // ... everyone's; and every reader of the slot refilled below is done
    const int nxt = kt + P - 1;
    if (nxt < kt1) issue(nxt, (nxt - kt0) % P);
    cp_commit();
    const NrSlot<T, NB>& Sm = S[(kt - kt0) % P];
    const int second = TWO && kt >= nt1;
    const int kv = min(NR_BK, (second ? k - k1 : k1) - (second ? kt - nt1 : kt) * NR_BK);
    const int kb = warp * KW, ke = min(kb + KW, kv);   // this warp's reduction indices (none past kv)
#pragma unroll 1
    for (int kk = kb; kk < ke; ++kk) {
      const C2 a = Sm.a[kk][lane];
#pragma unroll
      for (int j0 = 0; j0 < NB; j0 += V) {
        T bre[V], bim[V];
        *reinterpret_cast<V16*>(bre) = *reinterpret_cast<const V16*>(&Sm.br[kk][j0]);
        *reinterpret_cast<V16*>(bim) = *reinterpret_cast<const V16*>(&Sm.bi[kk][j0]);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          cr[j0 + v] = fma(a.x, bre[v], cr[j0 + v]);
          cr[j0 + v] = fma(-a.y, bim[v], cr[j0 + v]);
          ci[j0 + v] = fma(a.x, bim[v], ci[j0 + v]);
          ci[j0 + v] = fma(a.y, bre[v], ci[j0 + v]);
        }
      }
    }
  }
  cp_wait<0>();
  // the four warps' partial sums; warp w's go to red[w], and their sum replaces red[0] (part)
  __syncthreads();
  T* red = reinterpret_cast<T*>(nr_raw);   // [warp][2][NB][NR_BM + 1]
  constexpr int RW = 2 * NB * (NR_BM + 1);
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    red[warp * RW + j * (NR_BM + 1) + lane] = cr[j];
    red[warp * RW + (NB + j) * (NR_BM + 1) + lane] = ci[j];
  }
  __syncthreads();
  T* part = red;   // [2][NB][NR_BM + 1]
  for (int e = tid; e < 2 * NB * NR_BM; e += 128) {
    const int o = (e / NR_BM) * (NR_BM + 1) + e % NR_BM;
    T s = red[o];
#pragma unroll
    for (int w = 1; w < NR_WARPS; ++w) s += red[w * RW + o];
    part[o] = s;
  }
  if (ks > 1) {
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();   // every CTA's part is complete
    if (cl.block_rank() == 0) {
      for (int r = 1; r < ks; ++r) {
        const T* other = cl.map_shared_rank(part, r);
        for (int e = tid; e < 2 * NB * NR_BM; e += 128) {
          const int o = (e / NR_BM) * (NR_BM + 1) + e % NR_BM;
          part[o] += other[o];
        }
      }
    }
    cl.sync();   // the others' shared memory stays alive until the leader has read it
    if (cl.block_rank() != 0) return;
  }
  __syncthreads();
  // C rows are written NB columns at a time (consecutive threads, consecutive columns)
  T* Cr = d.C.re;
  T* Ci = d.C.re + d.C.plane;
  const T alpha = d.alpha, beta = d.beta;
  for (int e = tid; e < NB * NR_BM; e += 128) {
    const int r = e / NB, j = e % NB;
    const int gm = m0 + r;
    if (gm >= m || n0 + j >= n) continue;
    const int64_t off = (int64_t)gm * d.C.ld + n0 + j;
    T vr = alpha * part[j * (NR_BM + 1) + r], vi = alpha * part[(NB + j) * (NR_BM + 1) + r];
    if (beta != T(0)) {
      vr += beta * Cr[off];
      vi += beta * Ci[off];
    }
    Cr[off] = vr;
    Ci[off] = vi;
  }
}

template <typename T, int NB, bool TWO>
void launch_nb(const GemmDesc<T>* d_desc, const GemmTile* d_tiles, int ntiles, int ksplit, int max_k,
               cudaStream_t st) {
  constexpr int MS = nr_max_slots<T, NB>();
  // slots: the most tiles one CTA multiplies (bounded by the stage budget; at least 2)
  const int vt = (max_k + NR_BK - 1) / NR_BK + (TWO ? 1 : 0);
  int ns = (vt + ksplit - 1) / ksplit;
  ns = ns < 2 ? 2 : ns > MS ? MS : ns;
  const size_t stages = (size_t)ns * sizeof(NrSlot<T, NB>);
  const size_t red = nr_red_bytes<T, NB>();
  const size_t smem = stages > red ? stages : red;
  static PerDeviceOnce attr;
  attr([red] {
    const size_t most = (size_t)MS * sizeof(NrSlot<T, NB>) > red ? (size_t)MS * sizeof(NrSlot<T, NB>) : red;
    cudaFuncSetAttribute(k_gemm_nrhs<T, NB, TWO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
    cudaFuncSetAttribute(k_gemm_nrhs<T, NB, TWO>, cudaFuncAttributeNonPortableClusterSizeAllowed, 0);
  });
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ntiles, (unsigned)ksplit, 1);
  cfg.blockDim = dim3(128, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // overlap the launch with the predecessor's tail
  at[0].val.programmaticStreamSerializationAllowed = 1;
  at[1].id = cudaLaunchAttributeClusterDimension;
  at[1].val.clusterDim.x = 1;
  at[1].val.clusterDim.y = (unsigned)ksplit;
  at[1].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = ksplit > 1 ? 2 : 1;
  cudaLaunchKernelEx(&cfg, k_gemm_nrhs<T, NB, TWO>, d_desc, d_tiles, ns);
}

template <typename T, int NB>
void launch_nb2(const GemmDesc<T>* d_desc, const GemmTile* d_tiles, int ntiles, int ksplit, int max_k, bool two,
                cudaStream_t st) {
  if (two) launch_nb<T, NB, true>(d_desc, d_tiles, ntiles, ksplit, max_k, st);
  else launch_nb<T, NB, false>(d_desc, d_tiles, ntiles, ksplit, max_k, st);
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
void launch_gemm_nrhs(const GemmDesc<T>* d_desc, const GemmTile* d_tiles, int ntiles, int nb, int ksplit, int max_k,
                      cudaStream_t st, bool two) {
  if (ntiles <= 0) return;
  if (ksplit < 1) ksplit = 1;
  if (max_k < 1) max_k = 1;
  count_launches(1);
  if (nb <= 16) launch_nb2<T, 16>(d_desc, d_tiles, ntiles, ksplit, max_k, two, st);
  else launch_nb2<T, 32>(d_desc, d_tiles, ntiles, ksplit, max_k, two, st);
}

template void launch_gemm_nrhs<float>(const GemmDesc<float>*, const GemmTile*, int, int, int, int, cudaStream_t,
                                       bool);
template void launch_gemm_nrhs<double>(const GemmDesc<double>*, const GemmTile*, int, int, int, int,
                                        cudaStream_t, bool);

}  // namespace mf
