// Tensor-core planar complex GEMM for sm_103a: tcgen05.mma kind::tf32 with the
// accumulators in tensor memory.
//
//   C = alpha * A * B^T + beta * C     (complex, planar re/im planes, FP32 storage)
//   A: M x K row-major (K contiguous, lda % 4 == 0), B: N x K row-major (ldb % 4 == 0)
//
// This is the form of the Schur update C = F22 - F21 F12 (Sec. 2 step 4) with
// F12 kept transposed, and of the products F12 <- L^-1 P^T F12, F21 <- F21 U^-1.
// A complex product is four real products into two TMEM accumulators:
//   Dre += Are Bre^T ; Dre += (-Aim) Bim^T (negate-A bit) ; Dim += Are Bim^T ; Dim += Aim Bre^T.
//
// One CTA (8 warps) computes a 128 x 128 output tile.  Operand tiles of 8
// K-elements are staged in shared memory by cp.async (16-byte copies, zero
// fill past the edges) in the canonical no-swizzle K-major layout of 8 x 16-byte
// core matrices, 6 stages with copies issued 4 chunks ahead; thread 0 issues the
// MMAs and commits each stage to an mbarrier, which frees the stage.  A stage is
// refilled once the MMAs of the chunk two behind have completed, so the tensor core
// works on one chunk while the threads stage and split the next.  The epilogue
// reads TMEM with tcgen05.ld (a lane per row, half the columns per warpgroup), transposes 32 x 32 blocks
// through shared memory and writes C rows with consecutive lanes on consecutive
// columns, applying alpha / beta.
// SPLIT = true is the split-precision form: every staged value x is replaced in
// shared memory by hi = tf32(x) (round to nearest) plus a second tile lo = x - hi,
// and each product is hi*hi + hi*lo + lo*hi (three tensor-core passes), which
// brings the product close to FP32 accuracy (single TF32 pass: ~1e-3 relative).
// Every mbarrier wait is bounded: on expiry the kernel records MF status 2,
// drains its copies, frees its TMEM and returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace mf {

namespace {

constexpr int BM = 128, BN = 128, BK = 8, STAGES = 6, NT = 256;
constexpr int PREFETCH = STAGES - 2;                     // chunks whose copies are in flight
constexpr int KCH = BK / 4;                              // 16-byte K chunks per row
constexpr int TILE_BYTES = BM * BK * 4;                  // one plane tile of A (or B): 4 KB
constexpr int STAGE_BYTES = 8 * TILE_BYTES;              // Are, Aim, Bre, Bim and their lo parts
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 2048;  // + alignment slack, barriers, tmem slot
constexpr uint32_t TMEM_COLS = 256;                      // Dre (128 cols) + Dim (128 cols)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// canonical no-swizzle K-major layout: 8-row groups of KCH core matrices (8 rows x 16 B)
__device__ __forceinline__ uint32_t tile_off(int r, int kchunk) {
  return (uint32_t)((r >> 3) * (KCH * 128) + kchunk * 128 + (r & 7) * 16);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = KCH * 128;
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint32_t idesc_tf32(int neg_a) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)neg_a << 13) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait (non-blocking polls, so that the limit counts polls); returns false on expiry
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long spins) {
  for (long long i = 0; i < spins; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar) : "memory");
}

// The 16-byte chunk (row r, K chunk) of a staged tile that thread tid copies in its e-th copy.
__device__ __forceinline__ void chunk_of(int tid, int e, int& r, int& chunk) {
  const int idx = tid + e * NT;
  chunk = (idx >> 3) % KCH;               // 16-byte K chunk
  r = (idx / (8 * KCH)) * 8 + (idx & 7);  // 8-row group, row within it
}

// Stage one 128 x BK tile of a planar operand (rows r0.., K from k0) into smem.
__device__ __forceinline__ void load_tile(uint32_t dst_re, uint32_t dst_im, const float* re, int64_t plane, int64_t ld,
                                          int rows, int r0, int K, int k0, int tid) {
  // 128 rows x KCH chunks of 16 B per plane, (BM * KCH) / NT per thread
#pragma unroll
  for (int e = 0; e < (BM * KCH) / NT; ++e) {
    int r, chunk;
    chunk_of(tid, e, r, chunk);
    int gr = r0 + r, gk = k0 + chunk * 4;
    uint32_t bytes = 0;
    const float* src = re;
    if (gr < rows && gk < K) {
      int n = K - gk;
      bytes = (uint32_t)(n >= 4 ? 16 : 4 * n);
      src = re + (int64_t)gr * ld + gk;
    }
    uint32_t off = tile_off(r, chunk);
    cp_async16(dst_re + off, src, bytes);
    cp_async16(dst_im + off, bytes ? src + plane : re, bytes);
  }
}

// hi = x rounded to the 10 explicit mantissa bits of TF32 (round half away from zero, low 13 bits
// cleared explicitly, so that the MMA reads hi exactly), lo = x - hi (exact in FP32)
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  const uint32_t b = __float_as_uint(x);
  hi = __uint_as_float((b + 0x1000u) & 0xFFFFE000u);
  lo = x - hi;
}

template <bool SPLIT>
__global__ void __launch_bounds__(NT, 1) k_gemm_tc(const GemmDesc<float>* __restrict__ descs,
                                                    const GemmTile* __restrict__ tiles, int32_t* status,
                                                    long long spins) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const GemmTile t = tiles[blockIdx.x];
  const GemmDesc<float> d = descs[t.desc];
  const int m0 = t.tm * BM, n0 = t.tn * BN;
  const uint32_t sbase = (smem_u32(smem) + 1023u) & ~1023u;
  unsigned char* sgen = smem + (sbase - smem_u32(smem));
  uint64_t* bars = reinterpret_cast<uint64_t*>(sgen + STAGES * STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sgen + STAGES * STAGE_BYTES + 64);
  int* s_done = reinterpret_cast<int*>(sgen + STAGES * STAGE_BYTES + 96);
  const uint32_t bar0 = sbase + STAGES * STAGE_BYTES;

  if (tid == 0) {
    for (int s = 0; s < STAGES + 1; ++s) mbar_init(bar0 + 8 * s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const uint32_t tmem = *tmem_slot;
  (void)bars;

  const int K = d.k;
  const int nk = (K + BK - 1) / BK;
  const float* Ar = d.A.re;
  const float* Br = d.B.re;
  auto stage_addr = [&](int s, int which) { return sbase + s * STAGE_BYTES + which * TILE_BYTES; };
  auto issue_load = [&](int s, int kb) {
    load_tile(stage_addr(s, 0), stage_addr(s, 1), Ar, d.A.plane, d.A.ld, d.m, m0, K, kb * BK, tid);
    load_tile(stage_addr(s, 2), stage_addr(s, 3), Br, d.B.plane, d.B.ld, d.n, n0, K, kb * BK, tid);
  };
  bool ok = true;
  if (spins <= kProbeWaitLimit) {   // expiry test: the spare barrier (index STAGES) never completes
    if (tid == 0) *s_done = mbar_wait(bar0 + 8 * STAGES, 0u, spins) ? 1 : 0;
    __syncthreads();
    ok = *s_done != 0;
    __syncthreads();
  }
  int last = -1;   // thread 0: the last chunk whose MMAs it committed
#pragma unroll 1
  for (int s = 0; s < PREFETCH; ++s) {
    if (s < nk && ok) issue_load(s, s);
    cp_commit();
  }
  const uint32_t id_pos = idesc_tf32(0), id_neg = idesc_tf32(1);
  const uint32_t d_re = tmem, d_im = tmem + BN;
#pragma unroll 1
  const int nk_run = ok ? nk : 0;   // fixed before the loop: ok is uniform only here
  for (int kb = 0; kb < nk_run; ++kb) {
    const int s = kb % STAGES;
    const int kn = kb + PREFETCH;
    if (kn < nk) {
      const int sn = kn % STAGES;     // == (kb - 2) % STAGES: consumed by the MMAs of kb - 2
      if (kb >= 2 && ok) ok = mbar_wait(bar0 + 8 * sn, (uint32_t)(((kb - 2) / STAGES) & 1), spins);
      if (ok) issue_load(sn, kn);
    }
    cp_commit();
    cp_wait<PREFETCH>();
    if (SPLIT) {
      // the chunks this thread copied (its own copies are complete): hi in place, lo into the
      // second half of the stage; no barrier is needed before, the one below orders all of them
      // before the MMAs
#pragma unroll
      for (int e = 0; e < (BM * KCH) / NT; ++e) {
        int r, chunk;
        chunk_of(tid, e, r, chunk);
        const uint32_t off = tile_off(r, chunk);
#pragma unroll
        for (int t = 0; t < 4; ++t) {   // A re, A im, B re, B im
          float4* p = reinterpret_cast<float4*>(sgen + s * STAGE_BYTES + t * TILE_BYTES + off);
          float4* q = reinterpret_cast<float4*>(sgen + s * STAGE_BYTES + (4 + t) * TILE_BYTES + off);
          float4 x = *p, h, l;
          split_tf32(x.x, h.x, l.x);
          split_tf32(x.y, h.y, l.y);
          split_tf32(x.z, h.z, l.z);
          split_tf32(x.w, h.w, l.w);
          *p = h;
          *q = l;
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      const uint32_t a_re = stage_addr(s, 0), a_im = stage_addr(s, 1), b_re = stage_addr(s, 2), b_im = stage_addr(s, 3);
      const uint32_t lo = 4 * TILE_BYTES;   // offset of the lo tiles within the stage
#pragma unroll
      for (int kk = 0; kk < BK / 8; ++kk) {
        const uint32_t koff = kk * 256;   // 8 tf32 = 2 core matrices along K
        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
        mma_tf32(d_re, smem_desc(a_re + koff), smem_desc(b_re + koff), id_pos, acc);
        mma_tf32(d_re, smem_desc(a_im + koff), smem_desc(b_im + koff), id_neg, 1u);
        mma_tf32(d_im, smem_desc(a_re + koff), smem_desc(b_im + koff), id_pos, acc);
        mma_tf32(d_im, smem_desc(a_im + koff), smem_desc(b_re + koff), id_pos, 1u);
        if (SPLIT) {
          mma_tf32(d_re, smem_desc(a_re + koff), smem_desc(b_re + lo + koff), id_pos, 1u);
          mma_tf32(d_re, smem_desc(a_re + lo + koff), smem_desc(b_re + koff), id_pos, 1u);
          mma_tf32(d_re, smem_desc(a_im + koff), smem_desc(b_im + lo + koff), id_neg, 1u);
          mma_tf32(d_re, smem_desc(a_im + lo + koff), smem_desc(b_im + koff), id_neg, 1u);
          mma_tf32(d_im, smem_desc(a_re + koff), smem_desc(b_im + lo + koff), id_pos, 1u);
          mma_tf32(d_im, smem_desc(a_re + lo + koff), smem_desc(b_im + koff), id_pos, 1u);
          mma_tf32(d_im, smem_desc(a_im + koff), smem_desc(b_re + lo + koff), id_pos, 1u);
          mma_tf32(d_im, smem_desc(a_im + lo + koff), smem_desc(b_re + koff), id_pos, 1u);
        }
      }
      mma_commit(bar0 + 8 * s);
      last = kb;
    }
  }
  // all MMAs complete: thread 0's last commit covers every MMA it issued; every thread waits for it
  // (with the default limit even after an expired wait, so that no MMA can still write the columns
  // freed below).  The tile is written only if every chunk's MMAs were issued and no wait expired.
  if (tid == 0) *s_done = last;   // the last committed chunk, for every thread's wait below
  __syncthreads();
  const int lastc = *s_done;
  const uint32_t lbar = bar0 + 8 * (lastc < 0 ? 0 : lastc % STAGES), lpar = (uint32_t)((lastc / STAGES) & 1);
  bool done = lastc < 0 || mbar_wait(lbar, lpar, spins);   // the tile's results, within the wait limit
  // expired: still wait (default limit) until no MMA of this CTA can write the columns freed below
  if (!done && lastc >= 0) (void)mbar_wait(lbar, lpar, kDefaultWaitLimit);
  cp_wait<0>();
  ok = __syncthreads_and((ok && done && lastc == nk - 1) ? 1 : 0) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  if (!ok) {
    if (status) atomicExch(status, 2);
  } else {
    // epilogue: TMEM lane q holds row m0 + q of the tile
    const int lane = tid & 31;
    float* tb = reinterpret_cast<float*>(sgen) + warp * (2 * 32 * 33);
    // warp w reads TMEM lanes 32 (w % 4) .. +31 (its rows); the two warpgroups take half the columns each
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    float* Cr = d.C.re;
    float* Ci = d.C.re + d.C.plane;
#pragma unroll 1
    for (int c0 = (warp >> 2) * (BN / 2); c0 < (warp >> 2) * (BN / 2) + BN / 2; c0 += 32) {
      uint32_t vr[32], vi[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%"
          "19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
          : "=r"(vr[0]), "=r"(vr[1]), "=r"(vr[2]), "=r"(vr[3]), "=r"(vr[4]), "=r"(vr[5]), "=r"(vr[6]), "=r"(vr[7]),
            "=r"(vr[8]), "=r"(vr[9]), "=r"(vr[10]), "=r"(vr[11]), "=r"(vr[12]), "=r"(vr[13]), "=r"(vr[14]),
            "=r"(vr[15]), "=r"(vr[16]), "=r"(vr[17]), "=r"(vr[18]), "=r"(vr[19]), "=r"(vr[20]), "=r"(vr[21]),
            "=r"(vr[22]), "=r"(vr[23]), "=r"(vr[24]), "=r"(vr[25]), "=r"(vr[26]), "=r"(vr[27]), "=r"(vr[28]),
            "=r"(vr[29]), "=r"(vr[30]), "=r"(vr[31])
          : "r"(d_re + lane_base + c0));
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%"
          "19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
          : "=r"(vi[0]), "=r"(vi[1]), "=r"(vi[2]), "=r"(vi[3]), "=r"(vi[4]), "=r"(vi[5]), "=r"(vi[6]), "=r"(vi[7]),
            "=r"(vi[8]), "=r"(vi[9]), "=r"(vi[10]), "=r"(vi[11]), "=r"(vi[12]), "=r"(vi[13]), "=r"(vi[14]),
            "=r"(vi[15]), "=r"(vi[16]), "=r"(vi[17]), "=r"(vi[18]), "=r"(vi[19]), "=r"(vi[20]), "=r"(vi[21]),
            "=r"(vi[22]), "=r"(vi[23]), "=r"(vi[24]), "=r"(vi[25]), "=r"(vi[26]), "=r"(vi[27]), "=r"(vi[28]),
            "=r"(vi[29]), "=r"(vi[30]), "=r"(vi[31])
          : "r"(d_im + lane_base + c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      // transpose the warp's 32 x 32 block through shared memory (the stages are idle now) so
      // that the stores below run along C's rows
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        tb[lane * 33 + j] = __uint_as_float(vr[j]);
        tb[32 * 33 + lane * 33 + j] = __uint_as_float(vi[j]);
      }
      __syncwarp();
      const int col = n0 + c0 + lane;
#pragma unroll 4
      for (int r = 0; r < 32; ++r) {
        const int grow = m0 + (warp & 3) * 32 + r;
        if (grow < d.m && col < d.n) {
          const int64_t off = (int64_t)grow * d.C.ld + col;
          float xr = d.alpha * tb[r * 33 + lane];
          float xi = d.alpha * tb[32 * 33 + r * 33 + lane];
          if (d.beta != 0.f) {
            xr += d.beta * Cr[off];
            xi += d.beta * Ci[off];
          }
          Cr[off] = xr;
          Ci[off] = xi;
        }
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

}  // namespace

int gemm_tc_tile() { return BM; }

void launch_gemm_tc(const GemmDesc<float>* d_desc, const GemmTile* d_tiles, int ntiles, int32_t* status,
                    cudaStream_t st, bool split) {
  if (ntiles <= 0) return;
  static PerDeviceOnce attr;
  attr([] {
    cudaFuncSetAttribute(k_gemm_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    cudaFuncSetAttribute(k_gemm_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  });
  count_launches(1);
  if (split) k_gemm_tc<true><<<ntiles, NT, SMEM_BYTES, st>>>(d_desc, d_tiles, status, wait_limit());
  else k_gemm_tc<false><<<ntiles, NT, SMEM_BYTES, st>>>(d_desc, d_tiles, status, wait_limit());
}

}  // namespace mf
